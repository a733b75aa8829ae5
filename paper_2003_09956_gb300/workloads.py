"""Seeded synthetic inputs for the pseudo-projection solver.

This module only draws problem data (matrices, right-hand sides, starting
points, translation directions).  It holds none of the method's arithmetic,
imports nothing from the CUDA binding and nothing from the oracle, so the
tests can feed byte-identical inputs to both.

Workload families (the paper's own test system of Section 5 is a figure that
did not survive; these stand in for it):

* ``model_system(n)``: the scalable cube-with-a-cut-corner system
  0 <= x_j <= 200, sum_j x_j <= 200 (n - 1) + 100  (m = 2n + 1 rows), started
  outside the cut corner at x0 ~ U[300, 400]^n.
* ``dense_system(m, n)``: a_ij ~ N(0, 1), an interior point z ~ U(-1, 1)^n,
  b0 = A z + U(0.1, 1.0), a unit translation direction v = g / ||g||,
  Av = A v (both in FP64) and x0 ~ N(0, 25 I) rounded to binary32.
  ``grid="bf16"`` or ``grid="e4m3"`` first rounds A onto the bfloat16 grid, or
  onto a per-row power-of-two-scaled FP8 E4M3 grid, with torch's own
  conversions, so that the system is exactly representable in that storage
  format; b0 and Av are then computed from the rounded A.
* ``small_polytope(n, m)``: a small random system around a known interior
  point, for brute-force checks.
* ``sparse_system(m, n, k)``: the dense system's recipe with k non-zeros per
  row at random distinct columns (compressed-row form), or row lengths given
  per row; ``model_system_csr(n)``: the model system in compressed-row form.

Large matrices are drawn in fixed row chunks, each from its own
``SeedSequence`` child, so the bytes do not depend on the thread count.
"""
from __future__ import annotations

import concurrent.futures as _cf
import os

import numpy as np

_CHUNK_ROWS = 2048


def _chunk_rngs(seed: int, m: int):
    nchunks = (m + _CHUNK_ROWS - 1) // _CHUNK_ROWS
    children = np.random.SeedSequence(seed).spawn(nchunks + 1)
    return children[:nchunks], np.random.Generator(np.random.PCG64(children[-1]))


def _threads() -> int:
    return max(1, min(32, os.cpu_count() or 1))


def gaussian_matrix(m: int, n: int, seed: int, rows: tuple[int, int] | None = None) -> np.ndarray:
    """m x n float32 matrix with N(0, 1) entries, drawn in row chunks.

    ``rows=(r0, r1)`` returns only rows r0..r1-1 of that same matrix (r0 a
    multiple of the chunk size), without drawing the others."""
    r_lo, r_hi = (0, m) if rows is None else rows
    if r_lo % _CHUNK_ROWS:
        raise ValueError("row window must start on a chunk boundary")
    A = np.empty((r_hi - r_lo, n), np.float32)
    seqs, _ = _chunk_rngs(seed, m)

    def fill(c):
        r0 = c * _CHUNK_ROWS
        r1 = min(r_hi, r0 + _CHUNK_ROWS)
        g = np.random.Generator(np.random.PCG64(seqs[c]))
        if r1 - r0 == _CHUNK_ROWS or r1 == min(m, r0 + _CHUNK_ROWS):
            g.standard_normal((r1 - r0, n), dtype=np.float32, out=A[r0 - r_lo:r1 - r_lo])
        else:
            A[r0 - r_lo:r1 - r_lo] = g.standard_normal((min(m, r0 + _CHUNK_ROWS) - r0, n),
                                                       dtype=np.float32)[:r1 - r0]

    with _cf.ThreadPoolExecutor(_threads()) as ex:
        list(ex.map(fill, range(r_lo // _CHUNK_ROWS, (r_hi + _CHUNK_ROWS - 1) // _CHUNK_ROWS)))
    return A


def round_to_grid(A: np.ndarray, grid: str | None) -> np.ndarray:
    """Round A (float32) onto a storage grid with torch's conversions."""
    if grid is None or grid == "f32":
        return A
    import torch

    if grid == "bf16":
        out = np.empty_like(A)
        for r0 in range(0, A.shape[0], 8192):
            t = torch.from_numpy(A[r0:r0 + 8192])
            out[r0:r0 + 8192] = t.to(torch.bfloat16).to(torch.float32).numpy()
        return out
    if grid == "e4m3":
        out = np.empty_like(A)
        for r0 in range(0, A.shape[0], 8192):
            blk = A[r0:r0 + 8192]
            amax = np.abs(blk).max(axis=1).astype(np.float64)
            f, e2 = np.frexp(amax)
            # smallest power of two 2^e with amax / 2^e <= 448 = 0.875 * 2^9
            e = np.where(f <= 0.875, e2 - 9, e2 - 8)
            e = np.where(amax > 0, e, 0)
            s = np.ldexp(1.0, e).astype(np.float32)[:, None]
            t = torch.from_numpy(np.ascontiguousarray(blk / s))
            q = t.to(torch.float8_e4m3fn).to(torch.float32).numpy()
            out[r0:r0 + 8192] = q * s
        return out
    raise ValueError("unknown grid %r" % (grid,))


def _matvec_f64(A: np.ndarray, v: np.ndarray) -> np.ndarray:
    out = np.empty(A.shape[0], np.float64)
    step = 4096

    def part(r0):
        out[r0:r0 + step] = A[r0:r0 + step].astype(np.float64) @ v

    with _cf.ThreadPoolExecutor(_threads()) as ex:
        list(ex.map(part, range(0, A.shape[0], step)))
    return out


def dense_system(m: int, n: int, seed: int, grid: str | None = None,
                 x0_std: float = 5.0, rows: tuple[int, int] | None = None) -> dict:
    """The non-stationary dense random system (see the module docstring).

    ``rows=(r0, r1)`` gives the same system restricted to rows r0..r1-1
    (A, b0, Av sliced; z, v, x0 unchanged)."""
    A = round_to_grid(gaussian_matrix(m, n, seed, rows=rows), grid)
    _, g = _chunk_rngs(seed, m)
    z = g.uniform(-1.0, 1.0, n)
    slack = g.uniform(0.1, 1.0, m)
    dirn = g.standard_normal(n)
    v = dirn / np.sqrt(np.sum(dirn * dirn))
    x0 = g.normal(0.0, x0_std, n).astype(np.float32).astype(np.float64)
    if rows is not None:
        slack = slack[rows[0]:rows[1]]
    b0 = _matvec_f64(A, z) + slack
    Av = _matvec_f64(A, v)
    return {"A": A, "b0": b0, "Av": Av, "x0": x0, "z": z, "v": v,
            "m": m, "n": n, "seed": seed, "grid": grid}


def model_system(n: int, seed: int) -> dict:
    """0 <= x_j <= 200 and sum x_j <= 200(n-1)+100, x0 ~ U[300, 400]^n."""
    m = 2 * n + 1
    A = np.zeros((m, n), np.float64)
    b0 = np.zeros(m, np.float64)
    idx = np.arange(n)
    A[idx, idx] = -1.0           # -x_j <= 0
    A[n + idx, idx] = 1.0        #  x_j <= 200
    b0[n:2 * n] = 200.0
    A[2 * n, :] = 1.0            #  sum_j x_j <= 200(n-1) + 100
    b0[2 * n] = 200.0 * (n - 1) + 100.0
    g = np.random.Generator(np.random.PCG64(seed))
    x0 = g.uniform(300.0, 400.0, n)
    z = np.full(n, 100.0)        # strictly interior point
    return {"A": A, "b0": b0, "Av": None, "x0": x0, "z": z, "m": m, "n": n,
            "seed": seed}


def small_polytope(n: int, m: int, seed: int, spread: float = 3.0) -> dict:
    """Small random bounded system around an interior point z.

    Rows: the 2n box faces |x_j - z_j| <= 2 plus m - 2n random rows
    a ~ N(0, 1) with b = a.z + U(0.1, 1).  z is strictly interior."""
    g = np.random.Generator(np.random.PCG64(seed))
    z = g.uniform(-1.0, 1.0, n)
    rows, rhs = [], []
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        rows.append(e.copy())
        rhs.append(z[j] + 2.0)
        rows.append(-e)
        rhs.append(-z[j] + 2.0)
    for _ in range(max(0, m - 2 * n)):
        a = g.standard_normal(n)
        rows.append(a)
        rhs.append(float(a @ z) + g.uniform(0.1, 1.0))
    A = np.array(rows, np.float64)
    b0 = np.array(rhs, np.float64)
    x0 = z + g.normal(0.0, spread, n) * 3.0
    return {"A": A, "b0": b0, "Av": None, "x0": x0, "z": z, "m": A.shape[0],
            "n": n, "seed": seed}


def _csr_rows_dot(rp: np.ndarray, ci: np.ndarray, val: np.ndarray, v: np.ndarray) -> np.ndarray:
    """sum_e val[e] v[ci[e]] per row, binary64 (input construction only)."""
    m = rp.size - 1
    prod = val * v[ci]
    out = np.add.reduceat(prod, rp[:-1]) if prod.size else np.zeros(m)
    out[rp[:-1] == rp[1:]] = 0.0
    return out


def sparse_system(m: int, n: int, k: int, seed: int, x0_std: float = 5.0,
                  lengths: np.ndarray | None = None, dense_cols: int = 0) -> dict:
    """Sparse non-stationary random system in compressed-row form.

    Row i has k non-zeros (or ``lengths[i]``) at distinct columns, ascending;
    the entries are N(0, 1) rounded to binary32.  As for ``dense_system``:
    z ~ U(-1, 1)^n, b0 = A z + U(0.1, 1.0), v = g / ||g||, Av = A v (binary64),
    x0 ~ N(0, x0_std^2 I) rounded to binary32.  With a fixed k the columns of
    a row are a sorted sample with replacement from [0, n - k] plus 0..k-1
    (distinct by construction); with ``lengths`` each row is a uniform
    sample without replacement, and ``dense_cols`` > 0 puts columns
    0 .. dense_cols-1 into every row (counted in its length)."""
    g = np.random.Generator(np.random.PCG64(seed))
    if lengths is None:
        if not 1 <= k <= n:
            raise ValueError("need 1 <= k <= n")
        rp = np.arange(0, m * k + 1, k, dtype=np.int64)
        ci = np.empty(m * k, np.int32)
        val = np.empty(m * k, np.float64)
        step = 1 << 18
        for r0 in range(0, m, step):
            r1 = min(m, r0 + step)
            c = g.integers(0, n - k + 1, size=(r1 - r0, k), dtype=np.int64)
            c.sort(axis=1)
            c += np.arange(k, dtype=np.int64)
            ci[r0 * k:r1 * k] = c.reshape(-1)
            val[r0 * k:r1 * k] = g.standard_normal((r1 - r0) * k, dtype=np.float32)
    else:
        lengths = np.asarray(lengths, dtype=np.int64)
        if lengths.shape != (m,) or lengths.min() < max(1, dense_cols) or lengths.max() > n:
            raise ValueError("lengths must hold m values in [max(1, dense_cols), n]")
        rp = np.zeros(m + 1, np.int64)
        np.cumsum(lengths, out=rp[1:])
        ci = np.empty(int(rp[-1]), np.int32)
        head = np.arange(dense_cols)
        for i in range(m):
            rest = g.choice(n - dense_cols, int(lengths[i]) - dense_cols, replace=False) + dense_cols
            ci[rp[i]:rp[i + 1]] = np.concatenate([head, np.sort(rest)])
        val = g.standard_normal(ci.size, dtype=np.float32).astype(np.float64)
    z = g.uniform(-1.0, 1.0, n)
    slack = g.uniform(0.1, 1.0, m)
    dirn = g.standard_normal(n)
    v = dirn / np.sqrt(np.sum(dirn * dirn))
    x0 = g.normal(0.0, x0_std, n).astype(np.float32).astype(np.float64)
    b0 = _csr_rows_dot(rp, ci, val, z) + slack
    Av = _csr_rows_dot(rp, ci, val, v)
    return {"rp": rp, "ci": ci, "val": val, "b0": b0, "Av": Av, "x0": x0, "z": z, "v": v,
            "m": m, "n": n, "nnz": int(ci.size), "seed": seed}


def model_system_csr(n: int, seed: int) -> dict:
    """``model_system(n)`` in compressed-row form (3n non-zeros)."""
    m = 2 * n + 1
    idx = np.arange(n, dtype=np.int64)
    rp = np.concatenate([np.arange(0, 2 * n + 1, dtype=np.int64), [3 * n]])
    ci = np.concatenate([idx, idx, idx]).astype(np.int32)
    val = np.concatenate([-np.ones(n), np.ones(n), np.ones(n)])
    b0 = np.zeros(m, np.float64)
    b0[n:2 * n] = 200.0
    b0[2 * n] = 200.0 * (n - 1) + 100.0
    g = np.random.Generator(np.random.PCG64(seed))
    x0 = g.uniform(300.0, 400.0, n)
    return {"rp": rp, "ci": ci, "val": val, "b0": b0, "Av": None, "x0": x0,
            "z": np.full(n, 100.0), "m": m, "n": n, "nnz": 3 * n, "seed": seed}


def csr_to_dense(rp: np.ndarray, ci: np.ndarray, val: np.ndarray, n: int) -> np.ndarray:
    """Dense binary64 copy of a compressed-row matrix (small sizes)."""
    m = rp.size - 1
    A = np.zeros((m, n), np.float64)
    rows = np.repeat(np.arange(m), np.diff(rp))
    A[rows, ci] = val
    return A


def drifted_matrix(A0: np.ndarray, k: int, seed: int, amp: float = 0.05) -> np.ndarray:
    """A(k) = A0 + amp G_k, G_k ~ N(0, 1) drawn for tick k, rounded to
    binary32: a matrix whose every entry changes at every tick (Eq. 1 with a
    time-dependent A)."""
    G = gaussian_matrix(A0.shape[0], A0.shape[1], seed * 1000003 + k)
    return (A0.astype(np.float32) + np.float32(amp) * G).astype(np.float32)
