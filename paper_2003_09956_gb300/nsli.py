"""Python binding of the C ABI in ``include/nsli.h`` (argument marshalling only).

Every step of the method runs in ``libnsli.so`` (CUDA, sm_103a).  The binding
never computes any part of the method; when the library is missing it raises
instead of falling back to anything else.

Functions carry the C names (``nsli_create``, ``nsli_update_b``,
``nsli_iterate``, ``nsli_solve``, ``nsli_residual_max``, ...).  ``Solver``
wraps a handle for numpy arrays (host memory) or CUDA torch tensors (device
memory); the library detects which from the pointer.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

F64, F32, BF16, FP8E4M3 = 0, 1, 2, 3
RULE_RELAXED, RULE_MODAP = 0, 1
STOP_NONE, STOP_STEP, STOP_EPSMEM, STOP_MAXVIOL_REL = 0, 1, 2, 3
OK, NOT_CONVERGED, RUNNING, CANDIDATE = 0, 1, 2, 3
ERR_ARG, ERR_ZERO_ROW, ERR_NONFINITE, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED = (
    -1, -2, -3, -4, -5, -6, -7)

STORAGE = {"f64": F64, "f32": F32, "bf16": BF16, "fp8": FP8E4M3, "e4m3": FP8E4M3}
RULES = {"relaxed": RULE_RELAXED, "modap": RULE_MODAP}
STOPS = {"none": STOP_NONE, "step": STOP_STEP, "epsmem": STOP_EPSMEM,
         "maxviol_rel": STOP_MAXVIOL_REL}


class nsli_params(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("rule", ctypes.c_int32),
                ("stop", ctypes.c_int32), ("eps", ctypes.c_double),
                ("max_iter", ctypes.c_int64), ("block_iters", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("rho", ctypes.c_double)]


class nsli_result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64), ("tick", ctypes.c_int64),
                ("status", ctypes.c_int32), ("rejected", ctypes.c_int32),
                ("h", ctypes.c_int64), ("max_viol", ctypes.c_double),
                ("max_viol_norm", ctypes.c_double), ("max_abs_b", ctypes.c_double),
                ("last_step_norm", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class NsliError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        msg = "%s failed: %s (%d)" % (where, strerror(code), code)
        if detail:
            msg += ": " + detail
        super().__init__(msg)


_lib = None
_lock = threading.Lock()
EXPORTS = ["nsli_create", "nsli_create_csr", "nsli_update_b", "nsli_update_rows", "nsli_iterate", "nsli_iterate_timed", "nsli_solve",
           "nsli_residual_max", "nsli_map_reduce", "nsli_get_x", "nsli_set_x",
           "nsli_get_stored_rows", "nsli_get_norms2", "nsli_test_inject_timeout",
           "nsli_get_result", "nsli_launch_count", "nsli_sync", "nsli_destroy",
           "nsli_strerror", "nsli_last_error", "nsli_map_reduce_noalloc",
           "nsli_shard_begin", "nsli_shard_map", "nsli_shard_step",
           "nsli_batch_create", "nsli_batch_iterate", "nsli_batch_map_reduce", "nsli_batch_get_x",
           "nsli_batch_residual_max", "nsli_batch_launch_count", "nsli_batch_sync",
           "nsli_batch_destroy", "nsli_batch_last_error",
           "nsli_pool_create", "nsli_pool_add", "nsli_pool_step", "nsli_pool_set_ticks",
           "nsli_pool_poll", "nsli_pool_get_x", "nsli_pool_residual_max", "nsli_pool_remove",
           "nsli_pool_live", "nsli_pool_bytes_used", "nsli_pool_launch_count", "nsli_pool_sync",
           "nsli_pool_destroy", "nsli_pool_last_error",
           "nsli_pool_launch", "nsli_pool_yield", "nsli_pool_stopped", "nsli_pool_wait"]


def library_path() -> str:
    return _build.LIB_PATH


def load(path: str | None = None):
    """Load libnsli.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or _build.LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(
                "libnsli.so is not built (%s); run `python -c \"import __graft_entry__ as g; "
                "g.build()\"` first -- there is no fallback" % p)
        lib = ctypes.CDLL(p)
        P, i32, i64, d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        H = ctypes.c_void_p
        lib.nsli_create.argtypes = [ctypes.POINTER(H), i64, i64, i32, i32, P, i64, P, P, P, P, P]
        lib.nsli_create.restype = ctypes.c_int
        lib.nsli_create_csr.argtypes = [ctypes.POINTER(H), i64, i64, i32, i64, P, P, P, P, P, P, P, P]
        lib.nsli_create_csr.restype = ctypes.c_int
        lib.nsli_update_rows.argtypes = [H, i64, i64, i32, P, i64, P]
        lib.nsli_update_rows.restype = ctypes.c_int
        lib.nsli_update_b.argtypes = [H, P, i64]
        lib.nsli_update_b.restype = ctypes.c_int
        lib.nsli_iterate.argtypes = [H, ctypes.POINTER(nsli_params), i64]
        lib.nsli_iterate.restype = ctypes.c_int
        lib.nsli_iterate_timed.argtypes = [H, ctypes.POINTER(nsli_params), i64, P]
        lib.nsli_iterate_timed.restype = ctypes.c_int
        lib.nsli_solve.argtypes = [H, ctypes.POINTER(nsli_params), ctypes.POINTER(nsli_result)]
        lib.nsli_solve.restype = ctypes.c_int
        lib.nsli_residual_max.argtypes = [H, ctypes.POINTER(d), ctypes.POINTER(d)]
        lib.nsli_residual_max.restype = ctypes.c_int
        lib.nsli_map_reduce.argtypes = [H, P, ctypes.POINTER(i64), P]
        lib.nsli_map_reduce.restype = ctypes.c_int
        lib.nsli_get_x.argtypes = [H, P]
        lib.nsli_get_x.restype = ctypes.c_int
        lib.nsli_set_x.argtypes = [H, P]
        lib.nsli_set_x.restype = ctypes.c_int
        lib.nsli_get_stored_rows.argtypes = [H, i64, i64, P]
        lib.nsli_get_stored_rows.restype = ctypes.c_int
        lib.nsli_test_inject_timeout.argtypes = [H, i32]
        lib.nsli_test_inject_timeout.restype = ctypes.c_int
        lib.nsli_get_norms2.argtypes = [H, P]
        lib.nsli_get_norms2.restype = ctypes.c_int
        lib.nsli_get_result.argtypes = [H, ctypes.POINTER(nsli_result)]
        lib.nsli_get_result.restype = ctypes.c_int
        lib.nsli_launch_count.argtypes = [H]
        lib.nsli_launch_count.restype = i64
        lib.nsli_sync.argtypes = [H]
        lib.nsli_sync.restype = ctypes.c_int
        lib.nsli_destroy.argtypes = [H]
        lib.nsli_destroy.restype = None
        lib.nsli_strerror.argtypes = [ctypes.c_int]
        lib.nsli_strerror.restype = ctypes.c_char_p
        lib.nsli_last_error.argtypes = [H]
        lib.nsli_last_error.restype = ctypes.c_char_p
        lib.nsli_map_reduce_noalloc.argtypes = [i64, i64, P, i64, P, P, P, P, P, P, P]
        lib.nsli_map_reduce_noalloc.restype = ctypes.c_int
        lib.nsli_shard_begin.argtypes = [H, ctypes.POINTER(nsli_params)]
        lib.nsli_shard_begin.restype = ctypes.c_int
        lib.nsli_shard_map.argtypes = [H, P]
        lib.nsli_shard_map.restype = ctypes.c_int
        lib.nsli_shard_step.argtypes = [H, P, i32, i32]
        lib.nsli_shard_step.restype = ctypes.c_int
        lib.nsli_batch_create.argtypes = [ctypes.POINTER(H), i64, i64, i32, P, i64, P, P, P, P, P]
        lib.nsli_batch_create.restype = ctypes.c_int
        lib.nsli_batch_iterate.argtypes = [H, ctypes.POINTER(nsli_params), i64]
        lib.nsli_batch_iterate.restype = ctypes.c_int
        lib.nsli_batch_map_reduce.argtypes = [H, d, P, P, P]
        lib.nsli_batch_map_reduce.restype = ctypes.c_int
        lib.nsli_batch_get_x.argtypes = [H, P]
        lib.nsli_batch_get_x.restype = ctypes.c_int
        lib.nsli_batch_residual_max.argtypes = [H, P]
        lib.nsli_batch_residual_max.restype = ctypes.c_int
        lib.nsli_batch_launch_count.argtypes = [H]
        lib.nsli_batch_launch_count.restype = i64
        lib.nsli_batch_sync.argtypes = [H]
        lib.nsli_batch_sync.restype = ctypes.c_int
        lib.nsli_batch_destroy.argtypes = [H]
        lib.nsli_batch_destroy.restype = None
        lib.nsli_batch_last_error.argtypes = [H]
        lib.nsli_batch_last_error.restype = ctypes.c_char_p
        lib.nsli_pool_create.argtypes = [ctypes.POINTER(H), i32, i64, P]
        lib.nsli_pool_create.restype = ctypes.c_int
        lib.nsli_pool_add.argtypes = [H, i64, i64, P, i64, P, P, P, ctypes.POINTER(nsli_params),
                                      ctypes.POINTER(i64)]
        lib.nsli_pool_add.restype = ctypes.c_int
        lib.nsli_pool_step.argtypes = [H, i32]
        lib.nsli_pool_step.restype = ctypes.c_int
        lib.nsli_pool_set_ticks.argtypes = [H, P, P, i64]
        lib.nsli_pool_set_ticks.restype = ctypes.c_int
        lib.nsli_pool_poll.argtypes = [H, P, P, P, i64, ctypes.POINTER(i64)]
        lib.nsli_pool_poll.restype = ctypes.c_int
        lib.nsli_pool_get_x.argtypes = [H, i64, P]
        lib.nsli_pool_get_x.restype = ctypes.c_int
        lib.nsli_pool_residual_max.argtypes = [H, i64, ctypes.POINTER(d), ctypes.POINTER(d)]
        lib.nsli_pool_residual_max.restype = ctypes.c_int
        lib.nsli_pool_remove.argtypes = [H, i64]
        lib.nsli_pool_remove.restype = ctypes.c_int
        for nm in ("nsli_pool_live", "nsli_pool_bytes_used", "nsli_pool_launch_count"):
            getattr(lib, nm).argtypes = [H]
            getattr(lib, nm).restype = i64
        lib.nsli_pool_sync.argtypes = [H]
        lib.nsli_pool_sync.restype = ctypes.c_int
        lib.nsli_pool_destroy.argtypes = [H]
        lib.nsli_pool_destroy.restype = None
        lib.nsli_pool_last_error.argtypes = [H]
        lib.nsli_pool_last_error.restype = ctypes.c_char_p
        lib.nsli_pool_launch.argtypes = [H, i64, d, d]
        lib.nsli_pool_launch.restype = ctypes.c_int
        lib.nsli_pool_yield.argtypes = [H]
        lib.nsli_pool_yield.restype = ctypes.c_int
        lib.nsli_pool_stopped.argtypes = [H]
        lib.nsli_pool_stopped.restype = i64
        lib.nsli_pool_wait.argtypes = [H, ctypes.POINTER(i64)]
        lib.nsli_pool_wait.restype = ctypes.c_int
        if path is None:
            _lib = lib
        return lib


def strerror(code: int) -> str:
    try:
        return load().nsli_strerror(int(code)).decode()
    except Exception:
        return "status %d" % code


def _ptr(a):
    """Address of a numpy array (host) or a CUDA tensor (device); None -> NULL."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    raise TypeError("expected a numpy array or a torch tensor, got %r" % type(a))


def _f64(a, n=None):
    if a is None:
        return None
    if isinstance(a, np.ndarray) or not hasattr(a, "data_ptr"):
        a = np.ascontiguousarray(a, dtype=np.float64)
    else:
        import torch
        a = a.to(torch.float64).contiguous()
    if n is not None and a.shape[0] != n:
        raise ValueError("expected %d elements, got %d" % (n, a.shape[0]))
    return a


def _check(code: int, where: str, h=None) -> int:
    if code < 0:
        detail = ""
        if h is not None:
            detail = load().nsli_last_error(h).decode()
        raise NsliError(code, where, detail)
    return code


def _sync_torch_inputs(*arrays):
    for a in arrays:
        if a is not None and hasattr(a, "is_cuda") and a.is_cuda:
            import torch
            torch.cuda.current_stream(a.device).synchronize()
            return


SHARD_HEADER = 4


def _check_record(t, n, rows):
    """A record array for the shard calls: a contiguous CUDA float64 tensor
    of rows x (SHARD_HEADER + n) elements (rows None: any whole number);
    returns the number of records."""
    if not (hasattr(t, "is_cuda") and t.is_cuda) or t.dtype.itemsize != 8 or not t.is_floating_point():
        raise ValueError("records must be a CUDA float64 tensor")
    if not t.is_contiguous():
        raise ValueError("records must be contiguous")
    per = SHARD_HEADER + n
    if t.numel() % per != 0 or t.numel() == 0 or (rows is not None and t.numel() != rows * per):
        raise ValueError("records must hold whole records of %d doubles" % per)
    return t.numel() // per


def map_reduce_noalloc(A, b, norms2, x, y, violated, max_viol, stream=None):
    """Allocation-free Map + Reduce on caller-held CUDA tensors of one device:
    A float32 (m, n) with unit column stride (row pitch A.stride(0) >= n),
    b and norms2 float32[m], x float32[n]; outputs y float64[n], violated
    int64[1], max_viol float64[1].  For callers that cannot allocate device
    memory (see nsli_map_reduce_noalloc in include/nsli.h).  The work is
    issued on ``stream`` (a cudaStream_t value), by default on torch's
    current stream of A's device, and is not synchronised."""
    import torch

    if A.dim() != 2 or A.stride(1) != 1 or A.stride(0) < A.shape[1]:
        raise ValueError("A must be a 2-D tensor with rows of unit stride")
    m, n = int(A.shape[0]), int(A.shape[1])
    want = [("A", A, torch.float32, None), ("b", b, torch.float32, m),
            ("norms2", norms2, torch.float32, m), ("x", x, torch.float32, n),
            ("y", y, torch.float64, n), ("violated", violated, torch.int64, 1),
            ("max_viol", max_viol, torch.float64, 1)]
    for name, t, dt, numel in want:
        if not (hasattr(t, "is_cuda") and t.is_cuda):
            raise ValueError("%s must be a CUDA tensor" % name)
        if t.device != A.device:
            raise ValueError("%s is on %s, A on %s" % (name, t.device, A.device))
        if t.dtype != dt:
            raise ValueError("%s must be %s, got %s" % (name, dt, t.dtype))
        if numel is not None and (t.numel() != numel or not t.is_contiguous()):
            raise ValueError("%s must be contiguous with %d elements" % (name, numel))
    with torch.cuda.device(A.device):
        if stream is None:
            stream = torch.cuda.current_stream(A.device).cuda_stream
        rc = load().nsli_map_reduce_noalloc(m, n, ctypes.c_void_p(A.data_ptr()), int(A.stride(0)),
                                            _ptr(b), _ptr(norms2), _ptr(x), _ptr(y), _ptr(violated),
                                            _ptr(max_viol), ctypes.c_void_p(stream) if stream else None)
    _check(rc, "nsli_map_reduce_noalloc")


def make_params(lam=1.0, rule="relaxed", stop="none", eps=0.0, max_iter=0,
                block_iters=0, rho=0.0) -> nsli_params:
    p = nsli_params()
    p.lambda_ = float(lam)
    p.rule = RULES[rule] if isinstance(rule, str) else int(rule)
    p.stop = STOPS[stop] if isinstance(stop, str) else int(stop)
    p.eps = float(eps)
    p.max_iter = int(max_iter)
    p.block_iters = int(block_iters)
    p.reserved = 0
    p.rho = float(rho)
    return p


class Solver:
    """One problem resident on the current CUDA device.

    A: (m, n) float32 or float64 array/tensor (row-major); b0, Av, norms2:
    length-m float64; x0: length-n float64.  ``storage`` is "f64", "f32",
    "bf16" or "fp8"."""

    def __init__(self, A, b0, x0, Av=None, norms2=None, storage="f32", stream=None):
        lib = load()
        m, n = int(A.shape[0]), int(A.shape[1])
        if isinstance(A, np.ndarray):
            if A.dtype not in (np.float32, np.float64):
                A = A.astype(np.float32)
            A = np.ascontiguousarray(A)
            a_dtype = F64 if A.dtype == np.float64 else F32
        else:
            import torch
            if A.dtype not in (torch.float32, torch.float64):
                A = A.to(torch.float32)
            A = A.contiguous()
            a_dtype = F64 if A.dtype == torch.float64 else F32
        self.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        b0, x0, Av, norms2 = _f64(b0, m), _f64(x0, n), _f64(Av, m), _f64(norms2, m)
        _sync_torch_inputs(A, b0, x0, Av, norms2)
        h = ctypes.c_void_p()
        s = None if stream is None else ctypes.c_void_p(stream)
        rc = lib.nsli_create(ctypes.byref(h), m, n, self.storage, a_dtype, _ptr(A), n,
                             _ptr(b0), _ptr(norms2), _ptr(Av), _ptr(x0), s)
        if rc != OK:
            raise NsliError(rc, "nsli_create")
        self._h = h
        self.m, self.n = m, n

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            load().nsli_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    # -- calls
    def update_b(self, b0=None, tick=-1):
        b0 = _f64(b0, self.m)
        _sync_torch_inputs(b0)
        _check(load().nsli_update_b(self._h, _ptr(b0), int(tick)), "nsli_update_b", self._h)

    def update_rows(self, row0, A_rows, b0=None):
        """Replace rows row0 .. row0 + len(A_rows) - 1 (and their b0)."""
        if isinstance(A_rows, np.ndarray):
            if A_rows.dtype not in (np.float32, np.float64):
                A_rows = A_rows.astype(np.float32)
            A_rows = np.ascontiguousarray(A_rows)
            a_dtype = F64 if A_rows.dtype == np.float64 else F32
        else:
            import torch
            if A_rows.dtype not in (torch.float32, torch.float64):
                A_rows = A_rows.to(torch.float32)
            A_rows = A_rows.contiguous()
            a_dtype = F64 if A_rows.dtype == torch.float64 else F32
        rows, lda = int(A_rows.shape[0]), int(A_rows.shape[1])
        b0 = _f64(b0, rows)
        _sync_torch_inputs(A_rows, b0)
        _check(load().nsli_update_rows(self._h, int(row0), rows, a_dtype, _ptr(A_rows), lda, _ptr(b0)),
               "nsli_update_rows", self._h)

    def iterate(self, n_iter, lam=1.0, rule="relaxed", rho=0.0, block_iters=0):
        p = make_params(lam=lam, rule=rule, rho=rho, block_iters=block_iters)
        _check(load().nsli_iterate(self._h, ctypes.byref(p), int(n_iter)), "nsli_iterate", self._h)

    def iterate_timed(self, n_iter, lam=1.0, rule="relaxed", rho=0.0):
        """Run n_iter iterations kernel by kernel; return summed device ms of
        (Map kernels, Reduce-and-step kernels)."""
        p = make_params(lam=lam, rule=rule, rho=rho)
        ms = np.zeros(2, np.float64)
        _check(load().nsli_iterate_timed(self._h, ctypes.byref(p), int(n_iter), _ptr(ms)),
               "nsli_iterate_timed", self._h)
        return float(ms[0]), float(ms[1])

    def solve(self, lam=1.0, rule="relaxed", stop="step", eps=1e-8, max_iter=100000,
              rho=0.0, block_iters=0) -> dict:
        p = make_params(lam=lam, rule=rule, stop=stop, eps=eps, max_iter=max_iter,
                        rho=rho, block_iters=block_iters)
        r = nsli_result()
        _check(load().nsli_solve(self._h, ctypes.byref(p), ctypes.byref(r)), "nsli_solve", self._h)
        return r.as_dict()

    def residual_max(self) -> tuple[float, float]:
        a, b = ctypes.c_double(), ctypes.c_double()
        _check(load().nsli_residual_max(self._h, ctypes.byref(a), ctypes.byref(b)),
               "nsli_residual_max", self._h)
        return a.value, b.value

    # -- row shards (ModAPL): see nsli_shard_* in include/nsli.h
    def shard_begin(self, lam=1.0, rule="relaxed", stop="none", eps=0.0, max_iter=0, rho=0.0):
        p = make_params(lam=lam, rule=rule, stop=stop, eps=eps, max_iter=max_iter, rho=rho)
        _check(load().nsli_shard_begin(self._h, ctypes.byref(p)), "nsli_shard_begin", self._h)

    def shard_map(self, record):
        """Map + local Reduce into `record` (a CUDA float64 tensor of
        SHARD_HEADER + n elements on the handle's device)."""
        _check_record(record, self.n, 1)
        _check(load().nsli_shard_map(self._h, _ptr(record)), "nsli_shard_map", self._h)

    def shard_step(self, records, force_step=False):
        """Global Reduce of `records` (CUDA float64, nranks x (SHARD_HEADER +
        n), worker order), the stop decision and the step."""
        R = _check_record(records, self.n, None)
        _check(load().nsli_shard_step(self._h, _ptr(records), R, int(bool(force_step))),
               "nsli_shard_step", self._h)

    def check(self):
        """Binary64 check at the current x and tick: (max r_i, max r_i /
        ||a_i||, max |b_i|, h)."""
        mv, mn = self.residual_max()
        r = self.result()
        return mv, mn, r["max_abs_b"], r["h"]

    def map_reduce(self):
        y = np.empty(self.n, np.float64)
        hv = ctypes.c_int64()
        stats = np.empty(3, np.float64)
        _check(load().nsli_map_reduce(self._h, _ptr(y), ctypes.byref(hv), _ptr(stats)),
               "nsli_map_reduce", self._h)
        return y, int(hv.value), {"maxviol": stats[0], "maxnorm": stats[1], "maxb": stats[2]}

    def get_x(self, out=None):
        x = np.empty(self.n, np.float64) if out is None else out
        _check(load().nsli_get_x(self._h, _ptr(x)), "nsli_get_x", self._h)
        return x

    def set_x(self, x):
        x = _f64(x, self.n)
        _sync_torch_inputs(x)
        _check(load().nsli_set_x(self._h, _ptr(x)), "nsli_set_x", self._h)

    def stored_rows(self, row0=0, rows=None):
        rows = self.m - row0 if rows is None else rows
        out = np.empty((rows, self.n), np.float64)
        _check(load().nsli_get_stored_rows(self._h, int(row0), int(rows), _ptr(out)),
               "nsli_get_stored_rows", self._h)
        return out

    def inject_timeout(self, slot=1):
        """Failure-detection test: returns the status of a Map launch whose
        first CTA waits on a bulk copy that is never issued."""
        return int(load().nsli_test_inject_timeout(self._h, int(slot)))

    def norms2(self):
        out = np.empty(self.m, np.float64)
        _check(load().nsli_get_norms2(self._h, _ptr(out)), "nsli_get_norms2", self._h)
        return out

    def result(self) -> dict:
        r = nsli_result()
        _check(load().nsli_get_result(self._h, ctypes.byref(r)), "nsli_get_result", self._h)
        return r.as_dict()

    def launch_count(self) -> int:
        return int(load().nsli_launch_count(self._h))

    def sync(self):
        _check(load().nsli_sync(self._h), "nsli_sync", self._h)


class SparseSolver(Solver):
    """One problem with a sparse A in compressed-row form (row_ptr int64,
    col_idx int32 strictly increasing within a row, val float64), resident
    on the current CUDA device.  ``storage`` is "f64" or "f32".  Every
    Solver method applies (inject_timeout reports ERR_UNSUPPORTED)."""

    def __init__(self, m, n, row_ptr, col_idx, val, b0, x0, Av=None, norms2=None, storage="f32",
                 stream=None):
        lib = load()
        m, n = int(m), int(n)
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
        val = np.ascontiguousarray(val, dtype=np.float64)
        if row_ptr.shape != (m + 1,) or col_idx.shape != val.shape or col_idx.ndim != 1:
            raise ValueError("row_ptr must have m + 1 entries and col_idx / val nnz entries")
        self.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        b0, x0, Av, norms2 = _f64(b0, m), _f64(x0, n), _f64(Av, m), _f64(norms2, m)
        _sync_torch_inputs(b0, x0, Av, norms2)
        h = ctypes.c_void_p()
        s = None if stream is None else ctypes.c_void_p(stream)
        rc = lib.nsli_create_csr(ctypes.byref(h), m, n, self.storage, int(col_idx.size), _ptr(row_ptr),
                                 _ptr(col_idx), _ptr(val), _ptr(b0), _ptr(norms2), _ptr(Av), _ptr(x0), s)
        if rc != OK:
            raise NsliError(rc, "nsli_create_csr")
        self._h = h
        self.m, self.n = m, n
        self.nnz = int(col_idx.size)


class BatchSolver:
    """P <= 64 problems sharing one matrix, iterated together on the tensor
    cores (nsli_batch_*).  A: (m, n) float32; b0, Av: length m; X0: (P, n);
    tick_offsets: length-P integers s_p (problem p sees b0 + (s_p + k) rho Av)."""

    def __init__(self, A, b0, X0, Av=None, tick_offsets=None, stream=None):
        lib = load()
        A = np.ascontiguousarray(A, dtype=np.float32) if isinstance(A, np.ndarray) else A.contiguous()
        m, n = int(A.shape[0]), int(A.shape[1])
        X0 = np.ascontiguousarray(X0, dtype=np.float64) if isinstance(X0, np.ndarray) else \
            X0.to(__import__("torch").float64).contiguous()
        P = int(X0.shape[0])
        b0, Av = _f64(b0, m), _f64(Av, m)
        offs = None if tick_offsets is None else np.ascontiguousarray(tick_offsets, dtype=np.int64)
        _sync_torch_inputs(A, b0, X0, Av)
        h = ctypes.c_void_p()
        rc = lib.nsli_batch_create(ctypes.byref(h), m, n, P, _ptr(A), n, _ptr(b0), _ptr(Av),
                                   _ptr(offs), _ptr(X0), None if stream is None else ctypes.c_void_p(stream))
        if rc != OK:
            raise NsliError(rc, "nsli_batch_create")
        self._h, self.m, self.n, self.P = h, m, n, P

    def close(self):
        if getattr(self, "_h", None):
            load().nsli_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, rc, where):
        if rc < 0:
            raise NsliError(rc, where, load().nsli_batch_last_error(self._h).decode())

    def iterate(self, n_iter, lam=1.0, rho=0.0, block_iters=0):
        p = make_params(lam=lam, rho=rho, block_iters=block_iters)
        self._check(load().nsli_batch_iterate(self._h, ctypes.byref(p), int(n_iter)), "nsli_batch_iterate")

    def map_reduce(self, rho=0.0):
        Y = np.empty((self.P, self.n), np.float64)
        hv = np.empty(self.P, np.int64)
        mv = np.empty(self.P, np.float64)
        self._check(load().nsli_batch_map_reduce(self._h, float(rho), _ptr(Y), _ptr(hv), _ptr(mv)),
                    "nsli_batch_map_reduce")
        return Y, hv, mv

    def get_x(self):
        X = np.empty((self.P, self.n), np.float64)
        self._check(load().nsli_batch_get_x(self._h, _ptr(X)), "nsli_batch_get_x")
        return X

    def residual_max(self):
        mv = np.empty(self.P, np.float64)
        self._check(load().nsli_batch_residual_max(self._h, _ptr(mv)), "nsli_batch_residual_max")
        return mv

    def launch_count(self) -> int:
        return int(load().nsli_batch_launch_count(self._h))

    def sync(self):
        self._check(load().nsli_batch_sync(self._h), "nsli_batch_sync")


class Pool:
    """Device-resident problems advanced together (continuous batching).
    See nsli_pool_* in include/nsli.h."""

    def __init__(self, storage="bf16", max_bytes=0, stream=None):
        h = ctypes.c_void_p()
        rc = load().nsli_pool_create(ctypes.byref(h), STORAGE[storage], int(max_bytes),
                                     None if stream is None else ctypes.c_void_p(stream))
        if rc != OK:
            raise NsliError(rc, "nsli_pool_create")
        self._h = h

    def _check(self, rc, where):
        if rc < 0:
            raise NsliError(rc, where, load().nsli_pool_last_error(self._h).decode())
        return rc

    def close(self):
        if getattr(self, "_h", None):
            load().nsli_pool_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def add(self, A, b0, x0, Av=None, **params):
        """Admit a problem; returns its slot, or None when it does not fit."""
        m, n = int(A.shape[0]), int(A.shape[1])
        if isinstance(A, np.ndarray):
            A = np.ascontiguousarray(A, dtype=np.float32)
        b0, x0, Av = _f64(b0, m), _f64(x0, n), _f64(Av, m)
        _sync_torch_inputs(A, b0, x0, Av)
        p = make_params(**params)
        slot = ctypes.c_int64(-1)
        rc = load().nsli_pool_add(self._h, m, n, _ptr(A), n, _ptr(b0), _ptr(Av), _ptr(x0),
                                  ctypes.byref(p), ctypes.byref(slot))
        if rc == ERR_OOM:
            return None
        self._check(rc, "nsli_pool_add")
        return int(slot.value)

    def step(self, rounds=1):
        self._check(load().nsli_pool_step(self._h, int(rounds)), "nsli_pool_step")

    def set_ticks(self, slots, ticks):
        sl = np.ascontiguousarray(slots, dtype=np.int64)
        tk = np.ascontiguousarray(ticks, dtype=np.int64)
        self._check(load().nsli_pool_set_ticks(self._h, _ptr(sl), _ptr(tk), int(sl.size)),
                    "nsli_pool_set_ticks")

    def poll(self, cap=4096):
        sl = np.empty(cap, np.int64)
        st = np.empty(cap, np.int32)
        it = np.empty(cap, np.int64)
        cnt = ctypes.c_int64()
        self._check(load().nsli_pool_poll(self._h, _ptr(sl), _ptr(st), _ptr(it), cap, ctypes.byref(cnt)),
                    "nsli_pool_poll")
        k = min(int(cnt.value), cap)
        return [(int(sl[i]), int(st[i]), int(it[i])) for i in range(k)]

    def launch(self, max_rounds=1 << 40, max_seconds=1.0, tick_s=0.0):
        """One persistent launch over every live problem (asynchronous)."""
        self._check(load().nsli_pool_launch(self._h, int(max_rounds), float(max_seconds), float(tick_s)),
                    "nsli_pool_launch")

    def yield_(self):
        self._check(load().nsli_pool_yield(self._h), "nsli_pool_yield")

    def stopped(self):
        return int(load().nsli_pool_stopped(self._h))

    def wait(self):
        r = ctypes.c_int64()
        self._check(load().nsli_pool_wait(self._h, ctypes.byref(r)), "nsli_pool_wait")
        return int(r.value)

    def get_x(self, slot, n):
        x = np.empty(n, np.float64)
        self._check(load().nsli_pool_get_x(self._h, int(slot), _ptr(x)), "nsli_pool_get_x")
        return x

    def residual_max(self, slot):
        a, b = ctypes.c_double(), ctypes.c_double()
        self._check(load().nsli_pool_residual_max(self._h, int(slot), ctypes.byref(a), ctypes.byref(b)),
                    "nsli_pool_residual_max")
        return a.value, b.value

    def remove(self, slot):
        self._check(load().nsli_pool_remove(self._h, int(slot)), "nsli_pool_remove")

    def live(self):
        return int(load().nsli_pool_live(self._h))

    def bytes_used(self):
        return int(load().nsli_pool_bytes_used(self._h))

    def launch_count(self):
        return int(load().nsli_pool_launch_count(self._h))

    def sync(self):
        self._check(load().nsli_pool_sync(self._h), "nsli_pool_sync")
