#!/usr/bin/env python3
"""Throughput of the pseudo-projection iteration (AP / ModAP) on GB300.

One step = one iteration of the method over the whole system: the tick of
b(k) = b0 + k rho Av, the fused Map over all m rows (residuals, positive
slices, per-CTA sums), the deterministic Reduce, the stopping test and the
step x <- x - lambda y / h.  Default workload: the dense random system
m = 131072, n = 16384 (a_ij ~ N(0, 1), rho = 1e-4 per tick), A stored in
binary32 (8 GiB, far larger than L2, so no flush is needed between steps).
Measured in the same run and reported under "variants": the bfloat16 and
FP8-E4M3 storage of the same system, the model system's solve latency
(dense binary64 rows on the grid kernels, and compressed rows on one CTA), a
sparse system (4194304 x 1048576, 32 non-zeros per row), the same dense
system with all of A rewritten before every iteration, the batched
tensor-core form (64 problems sharing one A) and a serving stream.
`--workload dense-108001x54000` measures the long-row Map at the paper's
n = 54000.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl nsli|reference]

Multi-GPU (torchrun): every rank solves its own independent system
(replicas, weak scaling); `value` = iterations of all ranks / max time.
`--impl reference` times the FP64 CPU oracle on the host cores on a row
sample of the same workload (the baseline arm).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    "dense-131072x16384": {"m": 131072, "n": 16384, "rho": 1e-4, "seed": 2005},
    "dense-32768x8192": {"m": 32768, "n": 8192, "rho": 1e-4, "seed": 2004},
    # the benchmark's row length on a quarter of the rows (2 GiB binary32):
    # larger than L2, small enough for profiler replays
    "dense-32768x16384": {"m": 32768, "n": 16384, "rho": 1e-4, "seed": 2006},
    # rows longer than the register-resident limit (the chunked long-row Map):
    # the paper's n = 54000 with m = 2n + 1 rows, and a 16384-row slice of that
    # row length for profiler captures (3.5 GB binary32, larger than L2)
    "dense-108001x54000": {"m": 108001, "n": 54000, "rho": 1e-4, "seed": 2013},
    "dense-16384x54000": {"m": 16384, "n": 54000, "rho": 1e-4, "seed": 2014},
}
ELEM_BYTES = {"f32": 4, "bf16": 2, "fp8": 1, "f64": 8}
BATCHED = {
    # P problems sharing one bf16 A; problem p sees b0 + (p + k) rho Av
    "batched-65536x8192x64": {"m": 65536, "n": 8192, "P": 64, "rho": 1e-4, "seed": 2007},
    # a quarter of the rows, for profiler captures (A = 256 MiB bf16 > L2)
    "batched-16384x8192x64": {"m": 16384, "n": 8192, "P": 64, "rho": 1e-4, "seed": 2009},
}
SPARSE = {
    # k = 32 random columns per row (compressed rows + compressed columns,
    # 2 x 1.07 GB of binary32 entries and indices: larger than L2)
    "sparse-4194304x1048576x32": {"m": 1 << 22, "n": 1 << 20, "k": 32, "rho": 1e-4, "seed": 2011},
    "sparse-1048576x262144x32": {"m": 1 << 20, "n": 1 << 18, "k": 32, "rho": 1e-4, "seed": 2012},
}
METRIC = "ModAP iterations/sec"
UNIT = "iterations/s"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="nsli", choices=["nsli", "reference"])
    ap.add_argument("--workload", default="dense-131072x16384", choices=sorted(WORKLOADS))
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16", "fp8"])
    ap.add_argument("--variants", default="bf16,fp8",
                    help="other storage types measured in the same run ('' for none)")
    ap.add_argument("--batched", default="batched-65536x8192x64",
                    help="batched tensor-core workload measured in the same run ('' for none)")
    ap.add_argument("--batched-only", action="store_true",
                    help="time only the batched workload (profiling entry)")
    ap.add_argument("--sparse", default="sparse-4194304x1048576x32",
                    help="sparse workload measured in the same run ('' for none)")
    ap.add_argument("--sparse-only", action="store_true", help="time only the sparse workload")
    ap.add_argument("--matrix-updates", default="bf16",
                    help="storage for the run that rewrites A before every iteration ('' for none)")
    ap.add_argument("--serve-seconds", type=float, default=4.0,
                    help="length of the serving stream measured in the same run (0: none)")
    ap.add_argument("--serving-only", action="store_true", help="time only the serving stream")
    ap.add_argument("--pool", default="pool-40",
                    help="fixed pool timed with persistent launches in the same run ('' for none)")
    ap.add_argument("--pool-only", action="store_true", help="time only the fixed pool's persistent launches")
    ap.add_argument("--pool-rounds", type=int, default=20)
    ap.add_argument("--model-only", action="store_true",
                    help="time only the model system's solves (dense and compressed rows)")
    ap.add_argument("--model-seeds", type=int, default=30, help="seeds of the model-system solves")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--oracle-model-seeds", type=int, default=10,
                    help="model-system seeds solved by the FP64 oracle beside the GPU's")
    ap.add_argument("--cfg2", type=int, default=1, help="time the 32768 x 8192 system at rho 0, 1e-4, 1e-3")
    ap.add_argument("--shards", type=int, default=1,
                    help="time the benchmark system as two row shards on this GPU (the sharded form's own cost)")
    ap.add_argument("--long-rows", default="f32,bf16",
                    help="storage types timed on the 108001 x 54000 system (the paper's n); '' to skip")
    ap.add_argument("--feasibility", default="dense-8192x2048",
                    help="system solved to binary64-confirmed max r_i <= 1e-6 max|b| per storage ('' for none)")
    ap.add_argument("--feasibility-only", action="store_true", help="run only the solves to feasibility")
    ap.add_argument("--feasibility-storages", default="f32,bf16,fp8")
    ap.add_argument("--feasibility-grid", type=int, default=1,
                    help="1: A drawn on each storage type's grid; 0: the binary32 system rounded")
    ap.add_argument("--feasibility-max-iter", type=int, default=1000000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def map_bytes(m, n, storage):
    """Algorithmic bytes of one Map launch: A once, the 12-byte (16 with the
    FP8 row scale) per-row record b0, Av, 1/||a||^2, and x."""
    per_row = 16 if storage == "fp8" else 12
    return m * n * ELEM_BYTES[storage] + m * per_row + 4 * n


def sparse_bytes(m, n, nnz, storage):
    """Algorithmic bytes of one sparse iteration, per kernel: the row pass
    reads the row offsets, column indices and entries, the 16-byte row record
    (b0, Av, 1/||a||^2, 1/||a||; 32 in binary64), x once, and writes the
    slice coefficients; the column pass reads the column offsets, row indices
    and entries, the coefficients once, and reads/writes x (binary64 and its
    rounding)."""
    eb = ELEM_BYTES[storage]
    rec = 32 if storage == "f64" else 16
    row = 8 * (m + 1) + nnz * (4 + eb) + rec * m + eb * n + eb * m
    col = 8 * (n + 1) + nnz * (4 + eb) + eb * m + n * (8 + 8 + eb)
    return row, col


def step_bytes(m, n, storage):
    """Algorithmic bytes of one iteration: the Map's, plus x written back."""
    return map_bytes(m, n, storage) + 4 * n


MAP_SOURCE_END = "// --------------------------------------------------- Map, long rows --------"


def kernels_sha():
    """Hash of the source the Map kernel is compiled from: its barrier and
    bulk-copy helpers (nsli_async.cuh) and nsli_kernels.cu up to the
    long-row section (helpers, the Map body and its kernels; the kernels
    after it do not enter the Map)."""
    csrc = os.path.join(ROOT, "paper_2003_09956_gb300", "csrc")
    helpers = open(os.path.join(csrc, "nsli_async.cuh")).read()
    src = open(os.path.join(csrc, "nsli_kernels.cu")).read()
    end = src.find(MAP_SOURCE_END)
    return hashlib.sha256((helpers + src[:end if end >= 0 else len(src)]).encode()).hexdigest()[:12]


def profiled_traffic(workload, storage):
    """DRAM bytes per Map launch from the committed ncu summary, if it was
    taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "map_kernel_traffic.txt")
    if not os.path.exists(path):
        return None
    sha = kernels_sha()
    for line in open(path):
        f = line.split()
        if len(f) < 4 or line.startswith("#"):
            continue
        kv = dict(x.split("=", 1) for x in f if "=" in x)
        if kv.get("workload") == workload and kv.get("storage") == storage and kv.get("kernels_sha") == sha:
            return float(kv["traffic_bytes_per_launch"])
    return None


# GB300's nominal HBM3e bandwidth (context beside the measured copy peak)
NOMINAL_HBM_GBS = 7900.0


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples every 200 ms during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid=None):
        self.proc = None
        self.out = os.path.join("/tmp", "nsli_clocks_%d.csv" % os.getpid())
        cmd = ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits", "-lms", "200"]
        if device_uuid:
            cmd += ["-i", device_uuid]
        try:
            self.f = open(self.out, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock sampling unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.out):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.out)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_baseline(p, m_full, seconds, rho, rows=2048):
    """The FP64 oracle as it stands, single thread, on the first rows of the
    workload; rate scaled by rows (its cost per iteration is linear in m)."""
    import oracle

    rows = min(rows, p["A"].shape[0])
    A = np.ascontiguousarray(p["A"][:rows], dtype=np.float64)
    b0 = p["b0"][:rows]
    Av = p["Av"][:rows]
    n2, _ = oracle.norms2(A)
    x = p["x0"].copy()
    t0 = time.perf_counter()
    k = 0
    while True:
        _, x, _, _, _ = oracle.iteration(A, b0, Av, rho, k, n2, x)
        k += 1
        el = time.perf_counter() - t0
        if el >= seconds or k >= 1000:
            break
    rate = k / el * rows / m_full
    return {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d iterations of the FP64 C oracle (1 thread) over the first %d of %d rows "
                      "(n=%d) in %.1f s; rate scaled by %d/%d rows" % (k, rows, m_full, A.shape[1], el,
                                                                      rows, m_full)}


def cpu_baseline_all_cores(p, m_full, seconds, rho, rows_per_core=1024):
    """The FP64 oracle's own functions on every host core: the rows of the
    sample are split into one contiguous block per core, each block's Map
    and Reduce (oracle.map_reduce, C code that runs without the GIL) in its
    own thread, and the blocks combined in order with the oracle's ModAPL
    exchange (oracle.combine_step).  Rate scaled by rows."""
    import concurrent.futures as cf

    import oracle

    cores = os.cpu_count() or 1
    rows = min(p["A"].shape[0], rows_per_core * cores)
    A = np.ascontiguousarray(p["A"][:rows], dtype=np.float64)
    b0, Av = p["b0"][:rows], p["Av"][:rows]
    n2, _ = oracle.norms2(A)
    edges = [rows * w // cores for w in range(cores + 1)]
    blocks = [(a, c) for a, c in zip(edges[:-1], edges[1:]) if c > a]
    x = p["x0"].copy()
    with cf.ThreadPoolExecutor(len(blocks)) as ex:
        t0 = time.perf_counter()
        k = 0
        while True:
            b = oracle.tick_b(b0, Av, rho, k)
            recs = list(ex.map(lambda ac: oracle.map_reduce(A[ac[0]:ac[1]], b[ac[0]:ac[1]], n2[ac[0]:ac[1]], x),
                               blocks))
            _, x, _, _ = oracle.combine_step(recs, x)
            k += 1
            el = time.perf_counter() - t0
            if el >= seconds or k >= 1000:
                break
    rate = k / el * rows / m_full
    return {"value": rate, "unit": UNIT, "cores": len(blocks), "kind": "oracle",
            "sample": "%d iterations of the FP64 C oracle on %d threads (one contiguous row block each, "
                      "combined in order) over the first %d of %d rows (n=%d) in %.1f s; rate scaled by "
                      "%d/%d rows" % (k, len(blocks), rows, m_full, A.shape[1], el, rows, m_full)}


def oracle_max_violation(p, final, threads=None):
    """The FP64 oracle's max_i (a_i.x - b_i(k)) at a GPU run's final iterate
    and tick, on the exact values of its storage type (the oracle's own
    quantizers and Map/Reduce, one contiguous row block per host thread),
    beside the GPU's binary64 check: the max-violation error of the result."""
    import concurrent.futures as cf

    import oracle

    storage, x, tick, rho, mv_gpu = final
    A = p["A"]
    m = A.shape[0]
    cores = threads or os.cpu_count() or 1
    edges = [m * w // cores for w in range(cores + 1)]
    blocks = [(a, c) for a, c in zip(edges[:-1], edges[1:]) if c > a]
    b = oracle.tick_b(p["b0"], p["Av"], rho, tick)

    def block(ac):
        a, c = ac
        Ab = A[a:c]
        if storage == "bf16":
            Ab = oracle.quantize_bf16(Ab)
        elif storage == "fp8":
            Ab = oracle.quantize_e4m3_rows(Ab)[0]
        n2, _ = oracle.norms2(Ab)
        return oracle.map_reduce(Ab, b[a:c], n2, x)["maxviol"]

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(len(blocks)) as ex:
        mv = max(ex.map(block, blocks))
    return {"storage": storage, "gpu_f64": mv_gpu, "oracle_f64": mv, "abs_diff": abs(mv_gpu - mv),
            "rel_diff": abs(mv_gpu - mv) / max(abs(mv), 1e-300), "oracle_s": time.perf_counter() - t0,
            "threads": len(blocks)}


def oracle_model_solves(seeds):
    """The FP64 oracle's solve of the model system (n = 256, ||dx|| < 1e-8),
    one thread, on the first seeds of the GPU's model-system runs."""
    import oracle
    from paper_2003_09956_gb300 import workloads

    times, iters = [], []
    for sd in range(seeds):
        p = workloads.model_system(256, seed=sd)
        t0 = time.perf_counter()
        r = oracle.solve(p["A"], p["b0"], p["x0"], stop=oracle.STOP_STEP, eps=1e-8, max_iter=200000)
        times.append(time.perf_counter() - t0)
        iters.append(r["iters"])
    t = np.array(times) * 1e3
    return {"seeds": seeds, "cores": 1, "p50_solve_ms": float(np.percentile(t, 50)),
            "p99_solve_ms": float(np.percentile(t, 99)), "median_iterations": float(np.median(iters))}


def time_model_system(nsli, seeds=30):
    """The model system (n = 256, m = 513, binary64 storage, lambda = 1,
    ||dx|| < 1e-8): solve time per seed through nsli_solve (graph blocks,
    state polls and the binary64 confirmation included)."""
    from paper_2003_09956_gb300 import workloads

    times, iters, viol = [], [], []
    for sd in range(seeds):
        p = workloads.model_system(256, seed=sd)
        with nsli.Solver(p["A"], p["b0"], p["x0"], storage="f64") as s:
            if sd == 0:
                s.solve(stop="step", eps=1e-8, max_iter=100000, block_iters=64)   # warm-up (graph capture)
                s.set_x(p["x0"])
            t0 = time.perf_counter()
            r = s.solve(stop="step", eps=1e-8, max_iter=100000, block_iters=64)
            times.append(time.perf_counter() - t0)
            iters.append(r["iters"])
            viol.append(r["max_viol"] / np.abs(p["b0"]).max())
    t = np.array(times) * 1e3
    return {"workload": "model system n=256 m=513 f64, STEP 1e-8", "seeds": seeds,
            "p50_solve_ms": float(np.percentile(t, 50)), "p99_solve_ms": float(np.percentile(t, 99)),
            "median_iterations": float(np.median(iters)),
            "us_per_iteration": float(np.median(t * 1e3 / np.array(iters))),
            "max_rel_violation_f64": float(np.max(viol))}


def time_model_system_csr(nsli, seeds=30):
    """The same model systems held in compressed form (3n non-zeros), where
    the whole solve runs on one CTA: blocks of up to 1024 iterations per
    launch, state polls and the binary64 confirmation included."""
    from paper_2003_09956_gb300 import workloads

    times, iters, viol, launches = [], [], [], []
    for sd in range(seeds):
        p = workloads.model_system_csr(256, seed=sd)
        with nsli.SparseSolver(p["m"], p["n"], p["rp"], p["ci"], p["val"], p["b0"], p["x0"],
                               storage="f64") as s:
            if sd == 0:
                s.solve(stop="step", eps=1e-8, max_iter=100000)   # warm-up (module load)
                s.set_x(p["x0"])
            c0 = s.launch_count()
            t0 = time.perf_counter()
            r = s.solve(stop="step", eps=1e-8, max_iter=100000)
            times.append(time.perf_counter() - t0)
            launches.append(s.launch_count() - c0)
            iters.append(r["iters"])
            viol.append(r["max_viol"] / np.abs(p["b0"]).max())
    t = np.array(times) * 1e3
    return {"workload": "model system n=256 m=513 f64 in compressed rows (768 non-zeros), STEP 1e-8, "
                        "one CTA per solve", "seeds": seeds,
            "p50_solve_ms": float(np.percentile(t, 50)), "p99_solve_ms": float(np.percentile(t, 99)),
            "median_iterations": float(np.median(iters)),
            "us_per_iteration": float(np.median(t * 1e3 / np.array(iters))),
            "launches_per_solve": float(np.median(launches)),
            "max_rel_violation_f64": float(np.max(viol))}


def time_batched(nsli, torch, name, steps, warmup):
    """Batch iterations of P problems sharing one bf16 A on the tensor cores."""
    from paper_2003_09956_gb300 import workloads

    w = BATCHED[name]
    m, n, P = w["m"], w["n"], w["P"]
    p = workloads.dense_system(m, n, seed=w["seed"])
    rng = np.random.default_rng(w["seed"] + 1)
    X0 = rng.normal(0.0, 5.0, (P, n)).astype(np.float32).astype(np.float64)
    stream = torch.cuda.Stream()
    bs = nsli.BatchSolver(p["A"], p["b0"], X0, Av=p["Av"], tick_offsets=np.arange(P), stream=stream.cuda_stream)
    B = 16
    bs.iterate(max(warmup, B), rho=w["rho"], block_iters=B)
    bs.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = bs.launch_count()
    with torch.cuda.stream(stream):
        e0.record(stream)
        bs.iterate(steps, rho=w["rho"], block_iters=B)
        e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    launches = bs.launch_count() - l0
    mv = bs.residual_max()
    bs.close()
    abytes = 2 * m * n * 2                 # A and its transpose, bf16, once each
    flops = 2 * 2 * m * n * 3 * P          # two GEMMs, N = 3 split columns per problem
    fused = m * n * 2                      # A once, if the two products shared its reads
    return {"workload": name, "batch_iterations_per_s": 1000.0 / ms, "problem_iterations_per_s": P * 1000.0 / ms,
            "ms_per_batch_iteration": ms, "A_stream_gbs": abytes / (ms / 1e3) / 1e9,
            "A_once_gbs": fused / (ms / 1e3) / 1e9,
            "tensor_tflops": flops / (ms / 1e3) / 1e12,
            "useful_tensor_tflops": flops / 3 / (ms / 1e3) / 1e12,   # without the exact three-term split
            "gpu_launches": launches,
            "max_viol_f64_first_problems": [float(v) for v in mv[:4]]}


def time_sparse(nsli, torch, name, steps, warmup, peak):
    """Iterations of the sparse system (relaxed rule, binary32 entries)."""
    from paper_2003_09956_gb300 import workloads

    w = SPARSE[name]
    t0 = time.perf_counter()
    p = workloads.sparse_system(w["m"], w["n"], w["k"], seed=w["seed"])
    t_gen = time.perf_counter() - t0
    stream = torch.cuda.Stream()
    s = nsli.SparseSolver(p["m"], p["n"], p["rp"], p["ci"], p["val"], p["b0"], p["x0"], Av=p["Av"],
                          storage="f32", stream=stream.cuda_stream)
    B = min(steps, 50)
    s.iterate(max(warmup, B), rho=w["rho"], block_iters=B)
    s.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = s.launch_count()
    with torch.cuda.stream(stream):
        e0.record(stream)
        s.iterate(steps, rho=w["rho"], block_iters=B)
        e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    launches = s.launch_count() - l0
    kpass = min(steps, 100)
    row_ms, col_ms = s.iterate_timed(kpass, rho=w["rho"])
    mv, _ = s.residual_max()
    s.close()
    rb, cb = sparse_bytes(p["m"], p["n"], p["nnz"], "f32")
    row_gbs = rb / (row_ms / kpass / 1e3) / 1e9
    col_gbs = cb / (col_ms / kpass / 1e3) / 1e9
    return {"workload": name + " f32, rho=%g per tick, RELAXED lambda=1" % w["rho"], "nnz": p["nnz"],
            "value": 1000.0 / ms, "unit": UNIT, "ms_per_step": ms,
            "row_kernel_ms": row_ms / kpass, "col_kernel_ms": col_ms / kpass,
            "row_kernel_gbs": row_gbs, "col_kernel_gbs": col_gbs,
            "row_frac_of_measured_hbm": row_gbs / peak, "col_frac_of_measured_hbm": col_gbs / peak,
            "algorithmic_bytes_per_step": rb + cb, "gpu_launches": launches,
            "max_viol_f64": mv, "generate_s": t_gen}


def time_matrix_updates(nsli, torch, p, storage, w, steps, warmup, peak):
    """Every iteration preceded by a rewrite of ALL rows of A from device
    memory (a time-dependent matrix, c_u = (n + 1) m): two source matrices
    alternate, so each step stores, norms and streams a different A."""
    m, n = p["m"], p["n"]
    stream = torch.cuda.Stream()
    src = p["A"] if storage != "f64" else p["A"].astype(np.float64)
    s = nsli.Solver(src, p["b0"], p["x0"], Av=p["Av"], storage=storage, stream=stream.cuda_stream)
    A0 = torch.from_numpy(p["A"]).cuda()
    A1 = A0 * 1.001
    torch.cuda.synchronize()
    srcs = [A0, A1]
    for k in range(warmup):
        s.update_rows(0, srcs[k % 2])
        s.iterate(1, rho=w["rho"])
    s.sync()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = s.launch_count()
    e0.record(stream)
    for k in range(steps):
        s.update_rows(0, srcs[k % 2])
        s.iterate(1, rho=w["rho"])
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    launches = s.launch_count() - l0
    s.close()
    del A0, A1, srcs
    torch.cuda.empty_cache()
    eb = ELEM_BYTES[storage]
    moved = m * n * 4 + m * n * eb + map_bytes(m, n, storage)   # source read, stored write, Map read
    return {"workload": "dense %dx%d, all rows of A rewritten from device memory before every iteration, "
                        "%s storage" % (m, n, storage),
            "value": 1000.0 / ms, "unit": UNIT, "ms_per_step": ms, "bytes_per_step": moved,
            "gbs": moved / (ms / 1e3) / 1e9, "frac_of_measured_hbm": moved / (ms / 1e3) / 1e9 / peak,
            "gpu_launches": launches}


SERVE = {"rate": 200.0, "tick_s": 0.010, "rho": 1e-4, "eps": 1e-6, "seed": 2010,
         "classes": [int(round(512 * 2 ** (k / 2))) for k in range(11)], "c": [2, 4, 8],
         # cold requests start from x0 ~ N(0, 25 I) (tens of thousands of
         # relaxed iterations each); warm ones from x0 = z + d u, |u| = 1,
         # d ~ U(0.01, 0.1): near the polytope, as when a request follows the
         # solution of a nearby system
         "cold_budget": 300, "warm_budget": 5000, "warm_d": (0.01, 0.1),
         "ladder": (25.0, 12.5, 6.25), "ladder_drain_s": 8.0}


def serving_templates(torch, seconds, rates, seed):
    """Arrival times of every stream and one template system per (size
    class, c) drawn, resident on the device."""
    from paper_2003_09956_gb300 import workloads

    cfg = SERVE
    streams = {}
    for key, rate in rates.items():
        rng = np.random.default_rng(seed + int(rate))
        arrivals, t = [], 0.0
        while True:
            t += rng.exponential(1.0 / rate)
            if t > seconds:
                break
            arrivals.append((t, int(rng.integers(0, len(cfg["classes"]))), int(rng.integers(0, 3)),
                             int(rng.integers(1 << 30))))
        streams[key] = arrivals
    templates = {}
    for arrivals in streams.values():
        for _, k, ci, _ in arrivals:
            if (k, ci) in templates:
                continue
            n = cfg["classes"][k]
            m = cfg["c"][ci] * n
            p = workloads.dense_system(m, n, seed=cfg["seed"] + 100 * k + ci)
            templates[(k, ci)] = (torch.from_numpy(p["A"]).cuda(), p["b0"], p["Av"], n, p["z"])
    torch.cuda.synchronize()
    return streams, templates


def serving_stream(nsli, arrivals, templates, seconds, kind, rate, drain_s):
    """One Poisson stream served with continuous batching (persistent
    launches); wall-clock ticks of 10 ms move every b."""
    from paper_2003_09956_gb300 import serve

    cfg = SERVE
    budget = cfg["warm_budget"] if kind == "warm" else cfg["cold_budget"]
    params = dict(stop="maxviol_rel", eps=cfg["eps"], max_iter=budget, rho=cfg["rho"])
    srv = serve.Server(storage="bf16", tick_s=cfg["tick_s"], epoch_s=0.05)
    clock = time.perf_counter
    t0 = clock()
    i = 0

    def due():
        return i < len(arrivals) and arrivals[i][0] <= clock() - t0

    while True:
        now = clock() - t0
        while i < len(arrivals) and arrivals[i][0] <= now:
            ta, k, ci, sx = arrivals[i]
            A, b0, Av, n, z = templates[(k, ci)]
            g = np.random.default_rng(sx)
            if kind == "warm":
                u = g.normal(0.0, 1.0, n)
                x0 = z + g.uniform(*cfg["warm_d"]) * u / np.linalg.norm(u)
            else:
                x0 = g.normal(0.0, 5.0, n)
            x0 = x0.astype(np.float32).astype(np.float64)
            srv.submit(serve.Request(i, A, b0, x0, Av=Av, params=params, arrival=t0 + ta))
            i += 1
        if srv.queue or srv.live:
            srv.pump(wake=due)
        elif i < len(arrivals):
            time.sleep(max(0.0, min(0.001, arrivals[i][0] - now)))
        if (i >= len(arrivals) and not srv.queue and not srv.live) or now > seconds + drain_s:
            break
    elapsed = clock() - t0
    done = srv.done
    feas = [r for r in done if r.status == nsli.OK]
    lat = np.array([r.latency for r in done]) * 1e3
    flat = np.array([r.latency for r in feas]) * 1e3
    iters = np.array([r.iters for r in feas]) if feas else np.zeros(0)
    out = {"kind": kind, "arrival_rate_per_s": rate, "stream_s": seconds, "requests": len(arrivals),
           "completed": len(done), "feasible": len(feas), "not_converged_within_budget": len(done) - len(feas),
           "left_queued": len(srv.queue), "left_running": len(srv.live), "iteration_budget": budget,
           "elapsed_s": elapsed, "solves_per_s": len(done) / elapsed,
           "problem_iterations_per_s": srv.problem_iterations / elapsed,
           "p50_time_to_result_ms": float(np.percentile(lat, 50)) if done else None,
           "p99_time_to_result_ms": float(np.percentile(lat, 99)) if done else None,
           "p50_time_to_feasible_ms": float(np.percentile(flat, 50)) if feas else None,
           "p99_time_to_feasible_ms": float(np.percentile(flat, 99)) if feas else None,
           "median_iterations_to_feasible": float(np.median(iters)) if feas else None,
           "p99_iterations_to_feasible": float(np.percentile(iters, 99)) if feas else None,
           "max_viol_over_max_b0_f64_of_feasible": float(max(r.max_viol / np.abs(r.b0).max() for r in feas))
           if feas else None,
           "round_gbs": srv.bytes_streamed / max(srv.busy_s, 1e-9) / 1e9,
           "persistent_launches": srv.launches, "gpu_launches": srv.pool.launch_count()}
    # kept up: 95 % of the requests finished (feasible, or at their budget)
    # by the end of the drain
    out["sustained"] = bool(out["completed"] >= 0.95 * out["requests"])
    srv.close()
    return out


def time_serving(nsli, torch, seconds):
    """Poisson streams of dense random systems of mixed sizes (n
    log-uniform in [512, 16384] over 11 log-spaced classes, m = c n with c
    in {2, 4, 8}, bf16, rho = 1e-4 per 10 ms wall-clock tick): the cold
    stream at 200 requests/s, the warm stream at 200/s, and the warm stream
    at a ladder of lower rates down to the first one whose requests (95 %)
    are all served by the end of a drain (the sustainable rate)."""
    cfg = SERVE
    rates = {"cold": cfg["rate"], "warm": cfg["rate"]}
    for r in cfg["ladder"]:
        rates["warm_%g" % r] = r
    t_gen = time.perf_counter()
    streams, templates = serving_templates(torch, seconds, rates, cfg["seed"])
    t_gen = time.perf_counter() - t_gen
    out = {"ticks": "%g s wall clock, advanced on the device" % cfg["tick_s"], "template_setup_s": t_gen}
    out["cold_200_per_s"] = serving_stream(nsli, streams["cold"], templates, seconds, "cold", cfg["rate"],
                                           drain_s=1.0)
    out["warm_200_per_s"] = serving_stream(nsli, streams["warm"], templates, seconds, "warm", cfg["rate"],
                                           drain_s=2.0)
    sustainable = cfg["rate"] if out["warm_200_per_s"]["sustained"] else None
    if sustainable is None:
        for r in cfg["ladder"]:
            res = serving_stream(nsli, streams["warm_%g" % r], templates, seconds, "warm", r,
                                 drain_s=cfg["ladder_drain_s"])
            out["warm_%g_per_s" % r] = res
            if res["sustained"]:
                sustainable = r
                break
    out["sustainable_warm_rate_per_s"] = sustainable
    del templates
    torch.cuda.empty_cache()
    return out


POOL = {
    # resident bf16 problems, m = 4 n, n cycling over the sizes; one
    # persistent launch runs `rounds` rounds over all of them
    "pool-40": {"sizes": (1024, 2048, 4096, 8192, 16384), "nprob": 40, "seed": 2015},
    # the same mix without the largest size, for profiler captures (3.4 GB)
    "pool-20": {"sizes": (1024, 2048, 4096, 8192), "nprob": 20, "seed": 2015},
}


def time_pool_rounds(nsli, torch, name, rounds, warmup, peak):
    """Persistent launches (one launch = `rounds` rounds, each round one
    iteration of every resident problem) over a fixed pool of bf16
    problems of mixed sizes: bytes of A streamed per second."""
    from paper_2003_09956_gb300 import workloads

    w = POOL[name]
    pool = nsli.Pool(storage="bf16")
    total = 0
    # one template system per size (each problem gets its own device copy
    # of it and its own x0)
    templates = {n: workloads.dense_system(4 * n, n, seed=w["seed"] + n) for n in w["sizes"]}
    for q in range(w["nprob"]):
        n = int(w["sizes"][q % len(w["sizes"])])
        p = templates[n]
        A = torch.from_numpy(p["A"]).cuda()
        x0 = np.random.default_rng(w["seed"] + q).normal(0.0, 5.0, n).astype(np.float32).astype(np.float64)
        pool.add(A, p["b0"], x0, Av=p["Av"], stop="none", max_iter=1 << 40, rho=1e-4)
        total += 4 * n * n * 2
        del A
    del templates
    for _ in range(max(1, warmup)):
        pool.launch(max_rounds=rounds, max_seconds=60.0)
        pool.wait()
    l0 = pool.launch_count()
    t0 = time.perf_counter()
    pool.launch(max_rounds=rounds, max_seconds=60.0)
    r = pool.wait()
    el = time.perf_counter() - t0
    launches = pool.launch_count() - l0
    pool.close()
    torch.cuda.empty_cache()
    gbs = total * r / el / 1e9
    return {"workload": name + " (%d bf16 problems, m = 4n, n in %s)" % (w["nprob"], list(w["sizes"])),
            "bytes_of_A_per_round": total, "rounds": r, "ms_per_round": el / r * 1e3, "gbs": gbs,
            "frac_of_measured_hbm": gbs / peak, "gpu_launches": launches}


def time_cfg2(nsli, torch, steps, warmup, dist, world, peak):
    """The dense 32768 x 8192 system (binary32 storage) at the three
    translation rates rho = 0, 1e-4, 1e-3 per tick."""
    from paper_2003_09956_gb300 import workloads

    w0 = WORKLOADS["dense-32768x8192"]
    p = workloads.dense_system(w0["m"], w0["n"], seed=w0["seed"])
    out = {}
    mb = map_bytes(w0["m"], w0["n"], "f32")
    for rho in (0.0, 1e-4, 1e-3):
        s, _, r = time_storage(nsli, torch, p, "f32", {"rho": rho}, steps, warmup, dist, world)
        s.close()
        val = world * steps / (r["ms"] / 1000.0)
        out["rho=%g" % rho] = {"value": val, "unit": UNIT, "ms_per_step": r["ms"] / steps,
                               "map_ms_avg": r["map_ms_avg"], "reduce_ms_avg": r["reduce_ms_avg"],
                               "map_gbs": mb / (r["map_ms_avg"] / 1000.0) / 1e9,
                               "map_frac_of_measured_hbm": mb / (r["map_ms_avg"] / 1000.0) / 1e9 / peak,
                               "max_viol_f64": r["max_viol_f64"], "gpu_launches": r["launches"]}
    return out


def time_long_rows(nsli, torch, storages, steps, warmup, dist, world, peak):
    """The paper's row length n = 54000 (m = 2n + 1 rows, A 21.7 GiB in
    binary32): rows longer than the register-resident limit, mapped on
    thread-block clusters, per storage type."""
    from paper_2003_09956_gb300 import workloads

    w0 = WORKLOADS["dense-108001x54000"]
    p = workloads.dense_system(w0["m"], w0["n"], seed=w0["seed"])
    out = {}
    for st in storages:
        s, _, r = time_storage(nsli, torch, p, st, w0, steps, warmup, dist, world)
        s.close()
        mb = map_bytes(w0["m"], w0["n"], st)
        out[st] = {"value": world * steps / (r["ms"] / 1000.0), "unit": UNIT, "ms_per_step": r["ms"] / steps,
                   "map_ms_avg": r["map_ms_avg"], "map_gbs": mb / (r["map_ms_avg"] / 1000.0) / 1e9,
                   "map_frac_of_measured_hbm": mb / (r["map_ms_avg"] / 1000.0) / 1e9 / peak,
                   "max_viol_f64": r["max_viol_f64"], "gpu_launches": r["launches"]}
    del p
    torch.cuda.empty_cache()
    return out


def time_shards_one_gpu(nsli, torch, p, storage, w, steps, warmup, fused_ms):
    """The row-sharded form (ModAPL's sublists, one handle per worker) with
    R = 2 workers on this one GPU and one stream: each iteration is every
    worker's Map + local Reduce into its row of the records array (what an
    allgather delivers on several GPUs) and every worker's global Reduce and
    step.  The workers run one after the other, so the time against the one
    handle over all rows is the cost the sharded form adds on the device
    (its extra launches, the records and the record-based step), without any
    transport."""
    from paper_2003_09956_gb300 import shard

    R = 2
    m, n = p["A"].shape
    stream = torch.cuda.Stream()
    ws = []
    for q in range(R):
        r0, r1 = shard.row_range(m, R, q)
        ws.append(nsli.Solver(np.ascontiguousarray(p["A"][r0:r1]), p["b0"][r0:r1], p["x0"], Av=p["Av"][r0:r1],
                              storage=storage, stream=stream.cuda_stream))
    recs = torch.zeros((R, shard.HEADER + n), dtype=torch.float64, device="cuda")
    for s in ws:
        s.shard_begin(lam=1.0, rule="relaxed", stop="none", max_iter=1 << 40, rho=w["rho"])

    def one():
        for q, s in enumerate(ws):
            s.shard_map(recs[q])
        for s in ws:
            s.shard_step(recs)

    for _ in range(warmup):
        one()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = sum(s.launch_count() for s in ws)
    e0.record(stream)
    for _ in range(steps):
        one()
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / steps
    launches = sum(s.launch_count() for s in ws) - l0
    xs = [s.get_x() for s in ws]
    same = all(np.array_equal(xs[0], x) for x in xs[1:])
    for s in ws:
        s.close()
    del recs
    torch.cuda.empty_cache()
    return {"workload": "%dx%d %s storage as %d row shards, one handle each, on one GPU" % (m, n, storage, R),
            "value": 1000.0 / ms, "unit": UNIT, "ms_per_step": ms, "fused_ms_per_step": fused_ms,
            "added_ms_per_step": ms - fused_ms, "record_bytes_per_worker": (shard.HEADER + n) * 8,
            "workers_hold_the_same_iterate": same, "gpu_launches": launches}


FEASIBILITY = {
    "dense-8192x2048": {"m": 8192, "n": 2048, "seed": 3001},
    "dense-16384x4096": {"m": 16384, "n": 4096, "seed": 3002},
    "dense-32768x8192": {"m": 32768, "n": 8192, "seed": 2004},
    # the benchmark system at rho = 0 (hundreds of thousands of iterations:
    # minutes per storage type)
    "dense-131072x16384": {"m": 131072, "n": 16384, "seed": 2005},
}


def time_feasibility(nsli, name, storages=("f32", "bf16", "fp8"), max_iter=1000000, on_grid=True):
    """Solves from x0 ~ N(0, 25 I) of a stationary dense random system to
    max_i r_i <= 1e-6 max|b| confirmed by the binary64 check, per storage
    (RELAXED, lambda = 1): iterations, wall time, the binary64 violation,
    and the binary32 stop candidates the check rejected.  on_grid: A drawn
    on each storage type's grid (the same system for every storage);
    otherwise the binary32 system, rounded to the storage type."""
    from paper_2003_09956_gb300 import workloads

    f = FEASIBILITY[name]
    out = {"workload": name + " rho=0, RELAXED lambda=1, MAXVIOL_REL 1e-6, x0 ~ N(0, 25 I); " +
           ("A drawn on each storage type's grid, so that z is interior to the stored system" if on_grid
            else "A drawn in binary32 and rounded to the storage type")}
    for st in storages:
        grid = {"f32": None, "bf16": "bf16", "fp8": "e4m3"}[st] if on_grid else None
        p = workloads.dense_system(f["m"], f["n"], seed=f["seed"], grid=grid)
        with nsli.Solver(p["A"], p["b0"], p["x0"], storage=st) as s:
            s.iterate(64, block_iters=64)          # warm-up (graph capture)
            s.set_x(p["x0"])
            s.sync()
            t0 = time.perf_counter()
            r = s.solve(stop="maxviol_rel", eps=1e-6, max_iter=max_iter, block_iters=256)
            el = time.perf_counter() - t0
        out[st] = {"status": nsli.strerror(r["status"]), "iterations": r["iters"], "solve_s": el,
                   "iterations_per_s": r["iters"] / el,
                   "max_viol_over_max_b_f64": r["max_viol"] / r["max_abs_b"],
                   "rejected_candidates": r["rejected"]}
    return out


def dist_setup():
    from paper_2003_09956_gb300 import replicas

    return replicas.rank_info()


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    w = WORKLOADS[args.workload]
    from paper_2003_09956_gb300 import workloads

    p = workloads.dense_system(w["m"], w["n"], seed=w["seed"], rows=(0, 2048))
    per_step_s = min(20.0, max(0.5, 90.0 / max(1, args.steps)))
    # warm-up steps, then K timed steps, each a bounded sample
    for _ in range(min(args.warmup, 3)):
        cpu_baseline(p, w["m"], 0.5, w["rho"])
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(p, w["m"], per_step_s, w["rho"]))
    el = time.perf_counter() - t0
    rate = statistics.median(v["value"] for v in vals)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / rate,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload + " f32-generated, FP64 oracle on a row sample",
                       "m": w["m"], "n": w["n"], "rho": w["rho"]},
            "cpu_baseline": dict(vals[-1], value=rate),
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": el}
    print(json.dumps(line, allow_nan=False), flush=True)
    return 0


def time_storage(nsli, torch, p, storage, w, steps, warmup, dist, world, clocks=None, soak_s=0.0):
    """Create the solver for one storage type, warm up, time `steps`
    iterations (graph replays), then one kernel-by-kernel pass.  With a
    clock sampler factory `clocks`, the sampler runs from the start of the
    warm-up to the end of the kernel pass, and the warm-up is extended to
    about `soak_s` seconds of the same iterations so that the sampler sees
    the clocks of this load (the timed region alone can be shorter than
    one sampling period)."""
    from paper_2003_09956_gb300 import replicas

    stream = torch.cuda.Stream()
    s = nsli.Solver(p["A"], p["b0"], p["x0"], Av=p["Av"], storage=storage, stream=stream.cuda_stream)
    B = min(steps, 50)
    s.iterate(max(warmup, B), rho=w["rho"], block_iters=B)   # also captures the graph
    s.sync()
    sampler = clocks() if clocks else None
    soak = 0
    if soak_s > 0:
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < soak_s:
            s.iterate(B * 8, rho=w["rho"], block_iters=B)
            s.sync()
            soak += B * 8
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    replicas.barrier(dist)
    torch.cuda.synchronize()
    l0 = s.launch_count()
    with torch.cuda.stream(stream):
        e0.record(stream)
        s.iterate(steps, rho=w["rho"], block_iters=B)
        e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    launches = s.launch_count() - l0
    replicas.barrier(dist)
    ms = replicas.max_over_ranks(dist, e0.elapsed_time(e1), device="cuda")
    kpass = min(steps, 100)
    map_ms, red_ms = s.iterate_timed(kpass, rho=w["rho"])
    clk = sampler.stop() if sampler else None
    mv, mn = s.residual_max()
    return s, stream, {"ms": ms, "launches": launches, "map_ms_avg": map_ms / kpass,
                       "reduce_ms_avg": red_ms / kpass, "kernel_pass_ms_per_step": (map_ms + red_ms) / kpass,
                       "max_viol_f64": mv, "max_viol_norm_f64": mn, "clocks": clk, "soak_iterations": soak,
                       "final": (storage, s.get_x(), s.result()["tick"], w["rho"], mv)}


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    import torch

    world, rank, local = dist_setup()
    dist = None
    if world > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = tdist
    else:
        torch.cuda.set_device(0)
    from paper_2003_09956_gb300 import nsli, replicas, workloads

    nsli.load()
    if args.serving_only:
        r = time_serving(nsli, torch, args.serve_seconds)
        if rank == 0:
            w = r["warm_200_per_s"]
            print(json.dumps({"metric": "serving solves/sec", "value": w["solves_per_s"], "unit": "solves/s",
                              "config": {"workload": "poisson-200/s mixed-size bf16 stream"}, **r}), flush=True)
        return 0
    if args.feasibility_only:
        r = time_feasibility(nsli, args.feasibility, storages=tuple(args.feasibility_storages.split(",")),
                             max_iter=args.feasibility_max_iter, on_grid=bool(args.feasibility_grid))
        if rank == 0:
            print(json.dumps({"metric": "solve to binary64-confirmed feasibility", "config": {"workload": r["workload"]},
                              **r}), flush=True)
        return 0
    if args.pool_only:
        peak, _ = measured_peak()
        r = time_pool_rounds(nsli, torch, args.pool, args.pool_rounds, max(1, args.warmup), peak)
        if rank == 0:
            print(json.dumps({"metric": "persistent pool rounds GB/s", "value": r["gbs"], "unit": "GB/s",
                              "config": {"workload": r["workload"]}, **r}), flush=True)
        return 0
    if args.model_only:
        dense = time_model_system(nsli, seeds=args.model_seeds)
        csr = time_model_system_csr(nsli, seeds=args.model_seeds)
        if rank == 0:
            print(json.dumps({"metric": "model system p50 solve ms", "value": csr["p50_solve_ms"], "unit": "ms",
                              "higher_is_better": False,
                              "config": {"workload": "model system n=256 m=513 f64, STEP 1e-8"},
                              "compressed_rows_one_cta": csr, "dense_rows_grid": dense}), flush=True)
        return 0
    if args.sparse_only:
        peak, _ = measured_peak()
        r = time_sparse(nsli, torch, args.sparse, args.steps, max(3, args.warmup), peak)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "config": {"workload": args.sparse}, **r}), flush=True)
        return 0
    if args.batched_only:
        r = time_batched(nsli, torch, args.batched, args.steps, max(3, args.warmup))
        if rank == 0:
            print(json.dumps({"metric": "batched ModAP iterations/sec", "value": r["problem_iterations_per_s"],
                              "unit": "problem-iterations/s", "config": {"workload": args.batched}, **r}),
                  flush=True)
        return 0
    w = WORKLOADS[args.workload]
    m, n = w["m"], w["n"]
    t_gen = time.perf_counter()
    p = workloads.dense_system(m, n, seed=w["seed"] + rank)
    t_gen = time.perf_counter() - t_gen
    K, W = args.steps, max(3, args.warmup)

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
    except Exception:
        uuid = None
    s, stream, main_run = time_storage(nsli, torch, p, args.storage, w, K, W, dist, world,
                                       clocks=lambda: ClockSampler(uuid), soak_s=1.5)
    clk = main_run["clocks"]
    clk["window"] = ("%d warm-up iterations of the same system (about 1.5 s), the %d timed iterations and "
                     "the kernel-by-kernel pass" % (main_run["soak_iterations"], K))

    # end to end through the public API with host buffers: each step copies
    # that tick's right-hand side in from pinned memory, iterates once and
    # reads x back
    Ke = min(K, 50)
    snaps = [np.ascontiguousarray(p["b0"] + (W + K + 100 + k) * w["rho"] * p["Av"]) for k in range(Ke)]
    b_pin = torch.empty((Ke, m), dtype=torch.float64, pin_memory=True).numpy()
    for k in range(Ke):
        b_pin[k] = snaps[k]
    x_pin = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
    s.sync()
    replicas.barrier(dist)
    t0 = time.perf_counter()
    for k in range(Ke):
        s.update_b(b_pin[k], tick=0)
        s.iterate(1, rho=0.0)
        s.get_x(out=x_pin)
    t_e2e = replicas.max_over_ranks(dist, time.perf_counter() - t0, device="cuda")
    s.close()

    peak, peak_kind = measured_peak()
    value = replicas.aggregate_rate(world, K, main_run["ms"] / 1000.0)
    mb = map_bytes(m, n, args.storage)
    achieved = mb / (main_run["map_ms_avg"] / 1000.0) / 1e9
    traffic = profiled_traffic(args.workload, args.storage)

    # variants: the storage variants come last so that they end the printed
    # line (whose tail is what a truncated log keeps)
    variants = {}
    variants["model_system_f64"] = time_model_system(nsli, seeds=args.model_seeds)
    variants["model_system_f64_csr"] = time_model_system_csr(nsli, seeds=args.model_seeds)
    if args.sparse:
        variants["sparse_f32"] = time_sparse(nsli, torch, args.sparse, K, W, peak)
    if args.matrix_updates:
        variants["matrix_rewrite_every_tick_" + args.matrix_updates] = time_matrix_updates(
            nsli, torch, p, args.matrix_updates, w, min(K, 50), W, peak)
    if args.batched:
        variants["batched_bf16"] = time_batched(nsli, torch, args.batched, min(K, 100), W)
    if args.serve_seconds > 0 and world == 1:
        variants["serving_bf16"] = time_serving(nsli, torch, args.serve_seconds)
    if args.pool and world == 1:
        variants["persistent_pool_bf16"] = time_pool_rounds(nsli, torch, args.pool, args.pool_rounds, 2, peak)
    if args.cfg2:
        variants["dense-32768x8192_f32"] = time_cfg2(nsli, torch, K, W, dist, world, peak)
    if args.shards and world == 1:
        variants["row_shards_2_on_one_gpu"] = time_shards_one_gpu(nsli, torch, p, args.storage, w, min(K, 20), W,
                                                                   main_run["ms"] / K)
    if args.long_rows:
        variants["dense-108001x54000"] = time_long_rows(nsli, torch, [v for v in args.long_rows.split(",") if v],
                                                        min(K, 20), W, dist, world, peak)
    if args.feasibility:
        variants["solve_to_feasibility"] = time_feasibility(nsli, args.feasibility)
    finals = [main_run["final"]]
    for st in [v for v in args.variants.split(",") if v and v != args.storage]:
        sv, _, r = time_storage(nsli, torch, p, st, w, K, W, dist, world)
        sv.close()
        finals.append(r["final"])
        vb = map_bytes(m, n, st)
        v_val = world * K / (r["ms"] / 1000.0)
        variants[st] = {"value": v_val, "unit": UNIT, "ms_per_step": r["ms"] / K,
                        "vs_f32": v_val / value,
                        "map_gbs": vb / (r["map_ms_avg"] / 1000.0) / 1e9,
                        "map_frac_of_measured_hbm": vb / (r["map_ms_avg"] / 1000.0) / 1e9 / peak,
                        "max_viol_f64": r["max_viol_f64"], "gpu_launches": r["launches"]}

    cpu = cpu_all = oracle_model = None
    viol_vs_oracle = []
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(p, m, args.cpu_seconds, w["rho"])
        cpu_all = cpu_baseline_all_cores(p, m, args.cpu_seconds, w["rho"])
        oracle_model = oracle_model_solves(args.oracle_model_seeds)
        viol_vs_oracle = [oracle_max_violation(p, f) for f in finals]

    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": main_run["ms"] / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.storage, "data": "synthetic",
        "config": {"workload": "%s %s storage, rho=%g per tick, RELAXED lambda=1" % (args.workload, args.storage,
                                                                                   w["rho"]),
                   "m": m, "n": n, "storage": args.storage, "rho": w["rho"],
                   "l2": "inputs larger than L2 (A is %.1f GiB), no flush" % (m * n * ELEM_BYTES[args.storage] / 2**30),
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "graph_block_iters": min(K, 50)},
        "roofline": {"bound": "hbm", "kernel": "map_kernel", "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "nominal_peak": NOMINAL_HBM_GBS, "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                     "algorithmic_bytes_per_launch": mb,
                     "map_ms_avg": main_run["map_ms_avg"], "reduce_ms_avg": main_run["reduce_ms_avg"],
                     "kernel_pass_ms_per_step": main_run["kernel_pass_ms_per_step"],
                     "step_gbs": step_bytes(m, n, args.storage) * value / world / 1e9},
        "e2e": {"value": replicas.aggregate_rate(world, Ke, t_e2e), "unit": UNIT, "h2d_bytes_per_step": m * 8,
                "d2h_bytes_per_step": n * 8},
        "gpu_launches": main_run["launches"],
        "clocks": clk,
        "max_viol_f64": main_run["max_viol_f64"],
        "variants": variants,
        "generate_s": t_gen,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
        line["cpu_baseline_all_cores"] = cpu_all
        line["variants"]["model_system_f64"]["oracle_1_thread"] = oracle_model
        line["max_viol_vs_oracle"] = viol_vs_oracle
    print(json.dumps(line, allow_nan=False), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
