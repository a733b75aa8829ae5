"""FP64 CPU oracle for the pseudo-projection method (AP / ModAP).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, double-precision
restatement of the method that the CUDA path is checked against.  Only the
tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import it; the product package never does, and this package imports
nothing from the product package.

The arithmetic lives in ``nsli_oracle.c`` (plain C, sequential loops, IEEE
double, ``-ffp-contract=off``); this module compiles it with gcc on first use
and marshals numpy arrays through ctypes.

Paper: Sokolinsky & Sokolinskaya, "Scalable Parallel Algorithm for Solving
Non-stationary Systems of Linear Inequalities" (2020).
  - positive slice of the reflection vector: Eq. 7 (Section 2)
  - phi = y / h, h = number of non-zero slices: Eq. 8
  - eps-membership stopping test: Eq. 10
  - ModAP fixed-length step psi = lambda * y / ||y||: Eq. 12
  - Map / Reduce list form: Eq. 13 and the ModAP-on-lists description (Section 3)
  - ModAPL's split of the list among workers and the global Reduce of their
    partial results (Section 3): combine_step

Every function here is pinned by the ``-m "not gpu"`` tests against closed
forms, brute force on small systems, invariants and library routines.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nsli_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libnsli_oracle.so")
_lock = threading.Lock()
_lib = None
_override = None


@contextlib.contextmanager
def library(path: str):
    """Test support: run the oracle's functions on another build of
    nsli_oracle.c (used to check that the pins catch planted mistakes)."""
    global _lib, _override
    old_lib, old_override = _lib, _override
    _lib, _override = None, path
    try:
        yield
    finally:
        _lib, _override = old_lib, old_override

RULE_RELAXED = 0
RULE_MODAP = 1
STOP_NONE = 0
STOP_STEP = 1
STOP_EPSMEM = 2
STOP_MAXVIOL_REL = 3
IT_STEPPED = 0
IT_CONVERGED = 1
IT_STEP_STOP = 2
OK = 0
NOT_CONVERGED = 1


def compile_source(src: str, out: str) -> str:
    """Compile an oracle source file into a shared library (same flags)."""
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", out, src, "-lm"]
    subprocess.run(cmd, check=True)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build`` (idempotent)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
        compile_source(_SRC, tmp)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(_override if _override else build())
        i64, dbl, ip = ctypes.c_int64, ctypes.c_double, ctypes.c_int
        P = ctypes.c_void_p
        lib.oracle_norms2.argtypes = [i64, i64, P, P]
        lib.oracle_norms2.restype = i64
        lib.oracle_tick_b.argtypes = [i64, P, P, dbl, i64, P]
        lib.oracle_tick_b.restype = None
        lib.oracle_map_reduce.argtypes = [i64, i64, P, P, P, P, P, P, P, P, P, P]
        lib.oracle_map_reduce.restype = None
        lib.oracle_iteration.argtypes = [i64, i64, P, P, P, dbl, i64, P, P, dbl,
                                         ip, ip, dbl, ip, P, P, P, P]
        lib.oracle_iteration.restype = ip
        lib.oracle_solve.argtypes = [i64, i64, P, P, P, dbl, i64, P, P, dbl, ip,
                                     ip, dbl, i64, P, P]
        lib.oracle_solve.restype = None
        lib.oracle_combine_step.argtypes = [i64, i64, P, P, P, P, P, P, dbl, ip, ip, dbl, ip,
                                            P, P]
        lib.oracle_combine_step.restype = ip
        lib.oracle_map_reduce_f32.argtypes = [i64, i64, P, P, P, P, P, P, P, P, P, P]
        lib.oracle_map_reduce_f32.restype = None
        lib.oracle_norms2_f32.argtypes = [i64, i64, P, P]
        lib.oracle_norms2_f32.restype = i64
        lib.oracle_quantize_bf16.argtypes = [i64, P, P]
        lib.oracle_quantize_bf16.restype = None
        lib.oracle_quantize_e4m3_rows.argtypes = [i64, i64, P, P, P]
        lib.oracle_quantize_e4m3_rows.restype = None
        lib.oracle_map_reduce_csr.argtypes = [i64, i64, P, P, P, P, P, P, P, P, P, P, P, P]
        lib.oracle_map_reduce_csr.restype = None
        lib.oracle_norms2_csr.argtypes = [i64, P, P, P]
        lib.oracle_norms2_csr.restype = i64
        _lib = lib
        return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def norms2(A) -> tuple[np.ndarray, int]:
    """||a_i||^2 per row in FP64 and the number of zero rows (Section 2).
    A float32 matrix is read as binary32 and widened entry by entry."""
    if isinstance(A, np.ndarray) and A.dtype == np.float32:
        A = np.ascontiguousarray(A)
        m, n = A.shape
        n2 = np.empty(m, np.float64)
        zero = _load().oracle_norms2_f32(m, n, _ptr(A), _ptr(n2))
        return n2, int(zero)
    A = _f64(A)
    m, n = A.shape
    n2 = np.empty(m, np.float64)
    zero = _load().oracle_norms2(m, n, _ptr(A), _ptr(n2))
    return n2, int(zero)


def tick_b(b0, Av, rho: float, k: int) -> np.ndarray:
    """b(k) = b0 + k * rho * Av (translation of the polytope, Section 5)."""
    b0 = _f64(b0)
    Av = None if Av is None else _f64(Av)
    out = np.empty_like(b0)
    _load().oracle_tick_b(b0.shape[0], _ptr(b0), _ptr(Av), float(rho), int(k), _ptr(out))
    return out


def map_reduce(A, b, n2, x) -> dict:
    """Map (Eq. 13 / Eq. 7) then Reduce(+) at x with right-hand side b.
    A float32 matrix is read as binary32 and widened entry by entry."""
    if isinstance(A, np.ndarray) and A.dtype == np.float32:
        A = np.ascontiguousarray(A)
        fn = _load().oracle_map_reduce_f32
    else:
        A = _f64(A)
        fn = _load().oracle_map_reduce
    b, n2, x = _f64(b), _f64(n2), _f64(x)
    m, n = A.shape
    y = np.empty(n, np.float64)
    r = np.empty(m, np.float64)
    h = ctypes.c_int64()
    mv, mn, mb = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    fn(m, n, _ptr(A), _ptr(b), _ptr(n2), _ptr(x), _ptr(y),
                              ctypes.byref(h), ctypes.byref(mv), ctypes.byref(mn),
                              ctypes.byref(mb), _ptr(r))
    return {"y": y, "h": int(h.value), "maxviol": mv.value, "maxnorm": mn.value,
            "maxb": mb.value, "r": r}


def norms2_csr(rp, val) -> tuple[np.ndarray, int]:
    """||a_i||^2 per compressed row in FP64 and the number of zero rows."""
    rp = np.ascontiguousarray(rp, dtype=np.int64)
    val = _f64(val)
    m = rp.size - 1
    n2 = np.empty(m, np.float64)
    zero = _load().oracle_norms2_csr(m, _ptr(rp), _ptr(val), _ptr(n2))
    return n2, int(zero)


def map_reduce_csr(rp, ci, val, n, b, n2, x) -> dict:
    """map_reduce for A in compressed-row form (row_ptr, col_idx, val)."""
    rp = np.ascontiguousarray(rp, dtype=np.int64)
    ci = np.ascontiguousarray(ci, dtype=np.int32)
    val, b, n2, x = _f64(val), _f64(b), _f64(n2), _f64(x)
    m = rp.size - 1
    y = np.empty(n, np.float64)
    r = np.empty(m, np.float64)
    h = ctypes.c_int64()
    mv, mn, mb = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _load().oracle_map_reduce_csr(m, int(n), _ptr(rp), _ptr(ci), _ptr(val), _ptr(b), _ptr(n2),
                                  _ptr(x), _ptr(y), ctypes.byref(h), ctypes.byref(mv),
                                  ctypes.byref(mn), ctypes.byref(mb), _ptr(r))
    return {"y": y, "h": int(h.value), "maxviol": mv.value, "maxnorm": mn.value,
            "maxb": mb.value, "r": r}


def iteration(A, b0, Av, rho, k, n2, x, lam=1.0, rule=RULE_RELAXED,
              stop=STOP_NONE, eps=0.0, force_step=False):
    """One iteration at tick k.  Returns (code, x_new, stats, y, r)."""
    A, b0, n2 = _f64(A), _f64(b0), _f64(n2)
    Av = None if Av is None else _f64(Av)
    x = np.array(x, dtype=np.float64, copy=True)
    m, n = A.shape
    y = np.empty(n, np.float64)
    bk = np.empty(m, np.float64)
    r = np.empty(m, np.float64)
    stats = np.zeros(6, np.float64)
    code = _load().oracle_iteration(m, n, _ptr(A), _ptr(b0), _ptr(Av), float(rho),
                                    int(k), _ptr(n2), _ptr(x), float(lam), int(rule),
                                    int(stop), float(eps), int(bool(force_step)),
                                    _ptr(y), _ptr(bk), _ptr(r), _ptr(stats))
    st = {"h": int(stats[0]), "maxviol": stats[1], "maxnorm": stats[2],
          "maxb": stats[3], "dx_norm": stats[4], "y_norm": stats[5]}
    return int(code), x, st, y, r


def combine_step(records, x, lam=1.0, rule=RULE_RELAXED, stop=STOP_NONE, eps=0.0,
                 force_step=False):
    """The exchange of ModAPL (Section 3): the per-worker Map/Reduce outputs
    ``records`` (a list, in worker order, of dicts with y, h, maxviol,
    maxnorm, maxb as map_reduce returns them) are combined in worker order,
    then the decision and step of one iteration are taken at x.
    Returns (code, x_new, stats, y)."""
    R = len(records)
    x = np.array(x, dtype=np.float64, copy=True)
    n = x.shape[0]
    ys = np.ascontiguousarray(np.stack([_f64(r["y"]) for r in records]) if R else
                              np.zeros((0, n)))
    hs = np.ascontiguousarray([int(r["h"]) for r in records], dtype=np.int64)
    mvs = _f64([r["maxviol"] for r in records])
    mns = _f64([r["maxnorm"] for r in records])
    mbs = _f64([r["maxb"] for r in records])
    y = np.empty(n, np.float64)
    stats = np.zeros(6, np.float64)
    code = _load().oracle_combine_step(R, n, _ptr(ys), _ptr(hs), _ptr(mvs), _ptr(mns), _ptr(mbs),
                                       _ptr(x), float(lam), int(rule), int(stop), float(eps),
                                       int(bool(force_step)), _ptr(y), _ptr(stats))
    st = {"h": int(stats[0]), "maxviol": stats[1], "maxnorm": stats[2],
          "maxb": stats[3], "dx_norm": stats[4], "y_norm": stats[5]}
    return int(code), x, st, y


def solve(A, b0, x0, Av=None, rho=0.0, k0=0, n2=None, lam=1.0,
          rule=RULE_RELAXED, stop=STOP_STEP, eps=1e-8, max_iter=100000) -> dict:
    """Run the method until the stopping rule holds or max_iter updates."""
    A, b0 = _f64(A), _f64(b0)
    Av = None if Av is None else _f64(Av)
    m, n = A.shape
    if n2 is None:
        n2, zero = norms2(A)
        if zero:
            raise ValueError("zero row in A: the method assumes a_i != 0")
    n2 = _f64(n2)
    x = np.array(x0, dtype=np.float64, copy=True)
    work = np.empty(n + m, np.float64)
    out = np.zeros(8, np.float64)
    _load().oracle_solve(m, n, _ptr(A), _ptr(b0), _ptr(Av), float(rho), int(k0),
                         _ptr(n2), _ptr(x), float(lam), int(rule), int(stop),
                         float(eps), int(max_iter), _ptr(work), _ptr(out))
    return {"status": int(out[0]), "iters": int(out[1]), "tick": int(out[2]),
            "h": int(out[3]), "maxviol": out[4], "maxnorm": out[5], "maxb": out[6],
            "last_dx": out[7], "x": x}


def quantize_bf16(a) -> np.ndarray:
    """Values of a binary32 array rounded to bfloat16 (RNE), as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    out = np.empty_like(a)
    _load().oracle_quantize_bf16(a.size, _ptr(a), _ptr(out))
    return out


def quantize_e4m3_rows(A) -> tuple[np.ndarray, np.ndarray]:
    """Per-row power-of-two-scaled FP8 E4M3 values of A (float32) and scales."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    m, n = A.shape
    out = np.empty_like(A)
    scale = np.empty(m, np.float32)
    _load().oracle_quantize_e4m3_rows(m, n, _ptr(A), _ptr(out), _ptr(scale))
    return out, scale
