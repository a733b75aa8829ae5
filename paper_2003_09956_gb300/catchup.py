"""Catch-up rate of the iteration on a translated polytope (the quantity the
experiments of Section 5 of Sokolinsky & Sokolinskaya 2020 report).

The polytope M of a system is translated before every iteration: at
iteration k the system is A x <= b0 + k rho A v, i.e. M(k) = M + k rho v
(Section 5: "coordinate-wise displacement", a fixed amount added to every
coordinate of M before the next iteration).  For the model system the
displacement is v = -(1, ..., 1): each coordinate moves by -rho per
iteration, away from the starting point x0 (which lies above the box); moved
the other way the box would sweep over x0 and every rate would count as
caught.  For the dense random system v is its own random unit direction.

Storage: binary64 for the systems held on the host (Algorithm 1's rate is
eps-sized, below binary32 resolution) and for the model systems in
compressed-row form, bf16 for the large dense model systems (their entries
0 and +-1 are exact; only ModAP runs there).

The catch-up rate of a rule (Algorithm 1 with relaxation lambda, Eq. 8, or
ModAP with step length lambda, Eq. 12) is the supremum of the rates rho for
which the iteration reaches eps-membership of the moving polytope (Eq. 10)
within an iteration budget K.  It is found by bracketing (doubling or
halving rho) and then bisecting on a log scale; every trial is one solve
from x0 at tick 0.  Multiplying by the measured iteration rate converts rho
per iteration into units per second, the paper's unit.

  python -m paper_2003_09956_gb300.catchup --model-n 256 4096 --dense 32768x8192
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import nsli, workloads


# --------------------------------------------------------------------------
# systems with their translation direction
# --------------------------------------------------------------------------

def model_system_translated(n: int, seed: int = 0) -> dict:
    """Model system with v = -(1, ..., 1): A v = -(row sums of A)."""
    p = workloads.model_system(n, seed)
    p["Av"] = -p["A"].sum(axis=1)
    p["v_norm"] = math.sqrt(n)
    return p


def model_system_translated_device(n: int, seed: int = 0, device=None) -> dict:
    """The same system with A built directly in device memory as binary32
    (the entries 0 and +-1 are exact in every storage format), for sizes
    whose dense host copy would be tens of gigabytes."""
    import torch

    m = 2 * n + 1
    A = torch.zeros((m, n), dtype=torch.float32, device=device)
    idx = torch.arange(n, device=device)
    A[idx, idx] = -1.0
    A[n + idx, idx] = 1.0
    A[2 * n, :] = 1.0
    b0 = np.zeros(m, np.float64)
    b0[n:2 * n] = 200.0
    b0[2 * n] = 200.0 * (n - 1) + 100.0
    Av = np.empty(m, np.float64)
    Av[:n] = 1.0
    Av[n:2 * n] = -1.0
    Av[2 * n] = -float(n)
    g = np.random.Generator(np.random.PCG64(seed))
    x0 = g.uniform(300.0, 400.0, n)
    return {"A": A, "b0": b0, "Av": Av, "x0": x0, "m": m, "n": n, "seed": seed,
            "v_norm": math.sqrt(n)}


def model_system_translated_csr(n: int, seed: int = 0) -> dict:
    """The model system in compressed-row form (3n non-zeros), same v."""
    p = workloads.model_system_csr(n, seed)
    Av = np.empty(p["m"], np.float64)
    Av[:n] = 1.0
    Av[n:2 * n] = -1.0
    Av[2 * n] = -float(n)
    p["Av"] = Av
    p["v_norm"] = math.sqrt(n)
    return p


def dense_system_translated(m: int, n: int, seed: int = 0) -> dict:
    """The dense random system; its v is already a unit vector."""
    p = workloads.dense_system(m, n, seed)
    p["v_norm"] = 1.0
    return p


# --------------------------------------------------------------------------
# the search (host logic, independent of how a trial runs)
# --------------------------------------------------------------------------

def max_rate(trial, rho0: float, steps: int = 12, limit: int = 64):
    """Bracket the largest rho with trial(rho) true.

    Assumes success is monotone in rho (a faster polytope is never easier
    to catch).  Returns (lo, hi, trials): trial(lo) succeeded (lo = 0 if
    none did), trial(hi) failed (hi = inf if none did); after bracketing,
    ``steps`` log-scale bisections shrink hi/lo to 2**(2**-steps)."""
    trials = []

    def run(r):
        ok = bool(trial(r))
        trials.append((r, ok))
        return ok

    lo, hi = (rho0, math.inf) if run(rho0) else (0.0, rho0)
    for _ in range(limit):
        if math.isinf(hi):
            r = lo * 2.0
            if run(r):
                lo = r
            else:
                hi = r
        elif lo == 0.0:
            r = hi * 0.5
            if run(r):
                lo = r
            else:
                hi = r
        else:
            break
    if lo == 0.0 or math.isinf(hi):
        return lo, hi, trials
    for _ in range(steps):
        r = math.sqrt(lo * hi)
        if run(r):
            lo = r
        else:
            hi = r
    return lo, hi, trials


# --------------------------------------------------------------------------
# trials on the GPU
# --------------------------------------------------------------------------

class GpuTrials:
    """One resident problem; trial(rho) solves from x0 at tick 0."""

    def __init__(self, p: dict, rule: str, lam: float, eps: float, max_iter: int,
                 storage: str = "f64", block_iters: int = 64):
        self.p, self.rule, self.lam = p, rule, lam
        self.eps, self.max_iter, self.block_iters = eps, max_iter, block_iters
        if "rp" in p:
            self.solver = nsli.SparseSolver(p["m"], p["n"], p["rp"], p["ci"], p["val"], p["b0"], p["x0"],
                                            Av=p["Av"], storage=storage)
        else:
            self.solver = nsli.Solver(p["A"], p["b0"], p["x0"], Av=p["Av"], storage=storage)
        self.last = None

    def close(self):
        self.solver.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __call__(self, rho: float) -> bool:
        s = self.solver
        s.set_x(self.p["x0"])
        s.update_b(None, tick=0)
        r = s.solve(lam=self.lam, rule=self.rule, stop="epsmem", eps=self.eps,
                    max_iter=self.max_iter, rho=rho, block_iters=self.block_iters)
        self.last = r
        return r["status"] == nsli.OK

    def timed(self, rho: float):
        """One solve from x0 at tick 0, synchronised: (reached, iterations,
        seconds), the seconds including the host's polls and the binary64
        confirmation of the stop (the running time of a solve)."""
        self.solver.sync()
        t0 = time.perf_counter()
        ok = self(rho)
        self.solver.sync()
        return ok, int(self.last["iters"]), time.perf_counter() - t0

    def iteration_rate(self, rho: float, min_seconds: float = 0.3) -> float:
        """Iterations per second of the same rule at the same rate, timed
        over a fixed iteration count (no stopping test)."""
        s = self.solver
        k = 64
        while True:
            s.set_x(self.p["x0"])
            s.update_b(None, tick=0)
            s.sync()
            t0 = time.perf_counter()
            s.iterate(k, lam=self.lam, rule=self.rule, rho=rho, block_iters=self.block_iters)
            s.sync()
            dt = time.perf_counter() - t0
            if dt >= min_seconds or k >= 1 << 22:
                return k / dt
            k *= 2


CURVE_FRACTIONS = (0.0, 0.25, 0.5, 0.75, 0.9, 0.97, 1.0)


def time_vs_rate(timed, rho_max: float, fractions=CURVE_FRACTIONS, repeats: int = 3) -> list:
    """Running time of a solve against the displacement rate (the kind of
    curve Section 5 reports): for rho = f rho_max, the median over `repeats`
    solves of timed(rho) -> (reached, iterations, seconds)."""
    out = []
    for f in fractions:
        rho = f * rho_max
        runs = [timed(rho) for _ in range(repeats)]
        secs = sorted(r[2] for r in runs)
        out.append({"fraction_of_rho_max": f, "rho_per_iteration": rho,
                    "reached": all(r[0] for r in runs), "iterations": runs[0][1],
                    "solve_ms": 1e3 * secs[len(secs) // 2]})
    return out


def catchup(p: dict, rule: str, lam: float, eps: float = 1e-7, max_iter: int = 20000,
            storage: str = "f64", rho0: float | None = None, steps: int = 12, curve: bool = False) -> dict:
    """Catch-up rate of one rule on one system, with the units conversion."""
    out = {"system": p.get("name", ""), "m": int(p["m"]), "n": int(p["n"]), "rule": rule,
           "lambda": lam, "eps": eps, "max_iter": max_iter, "storage": storage}
    with GpuTrials(p, rule, lam, eps, max_iter, storage) as t:
        if not t(0.0):
            out.update({"rho_max_per_iteration": 0.0, "note": "no eps-membership within "
                        "max_iter even for the stationary polytope",
                        "stationary_iterations": t.last["iters"]})
            return out
        out["stationary_iterations"] = t.last["iters"]
        if rho0 is None:
            rho0 = lam / max(p["v_norm"], 1.0) * 1e-3
        lo, hi, trials = max_rate(t, rho0, steps=steps)
        out["rho_max_per_iteration"] = lo
        out["rho_fail_per_iteration"] = hi if math.isfinite(hi) else None
        out["trials"] = len(trials)
        if lo > 0.0:
            t(lo)
            out["iterations_at_rho_max"] = t.last["iters"]
            ips = t.iteration_rate(lo)
            out["iterations_per_s"] = ips
            # speed of the polytope at the caught rate: per coordinate of v
            # (the paper's "coordinate-wise displacement") and as a vector
            out["units_per_s_per_coordinate"] = lo * ips
            out["units_per_s_total"] = lo * ips * p["v_norm"]
            if curve:
                pts = time_vs_rate(t.timed, lo)
                for q in pts:
                    q["units_per_s_per_coordinate"] = q["rho_per_iteration"] * ips
                out["time_vs_rate"] = pts
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--model-n", type=int, nargs="*", default=[256, 4096])
    ap.add_argument("--model-device-n", type=int, nargs="*", default=[],
                    help="model systems built in device memory (large n, bf16 storage)")
    ap.add_argument("--model-sparse-n", type=int, nargs="*", default=[],
                    help="model systems in compressed-row form (binary64)")
    ap.add_argument("--dense", nargs="*", default=[], help="MxN dense random systems")
    ap.add_argument("--lam-per-coordinate", type=float, nargs="+", default=[0.1, 1.0, 10.0],
                    help="ModAP step lengths, lambda = c * sqrt(n)")
    ap.add_argument("--relaxed-max-n", type=int, default=4096,
                    help="largest n for Algorithm 1 (its step shrinks like 1/n)")
    ap.add_argument("--max-iter", type=int, default=20000)
    ap.add_argument("--eps", type=float, default=1e-7)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--curve", action="store_true",
                    help="also time solves at fractions of the catch-up rate (time against rate)")
    args = ap.parse_args()
    nsli.load()
    systems = []
    for n in args.model_n:
        p = model_system_translated(n)
        p["name"] = f"model-{n}"
        systems.append((p, "f64"))
    for n in args.model_device_n:
        import torch
        p = model_system_translated_device(n, device=torch.device("cuda", torch.cuda.current_device()))
        p["name"] = f"model-{n}"
        systems.append((p, "bf16"))
    for n in args.model_sparse_n:
        p = model_system_translated_csr(n)
        p["name"] = f"model-{n}-csr"
        systems.append((p, "f64"))
    for spec in args.dense:
        m, n = (int(v) for v in spec.lower().split("x"))
        p = dense_system_translated(m, n)
        p["name"] = f"dense-{m}x{n}"
        systems.append((p, "f64"))
    for p, storage in systems:
        runs = []
        if p["n"] <= args.relaxed_max_n:
            runs.append(("relaxed", 1.0))
        for c in args.lam_per_coordinate:
            runs.append(("modap", c * math.sqrt(p["n"])))
        for rule, lam in runs:
            r = catchup(p, rule, lam, eps=args.eps, max_iter=args.max_iter, storage=storage,
                        steps=args.steps, curve=args.curve)
            print(json.dumps(r), flush=True)
        p.pop("A", None)


if __name__ == "__main__":
    main()
