"""The allocation-free Map + Reduce entry point.

Callers that cannot allocate device memory (code under a fixed
device-memory budget, or inside a host framework that owns all device
memory through its own allocator) use nsli_map_reduce_noalloc, whose
scratch is a fixed array inside the library.  Its results must agree with
the existing, allocating entry point nsli_map_reduce on the same system,
on two calls in a row (the second one with another x, so stale scratch
from the first call would show), and with the FP64 oracle element by
element.  This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import parity
from paper_2003_09956_gb300 import _build, nsli, workloads

pytestmark = pytest.mark.gpu

M, N = 3001, 1000


def _handle_reference(p, x):
    """y, h and max r from the existing entry point (handle, binary32 storage)."""
    with nsli.Solver(p["A"], p["b0"], x, storage="f32") as s:
        y, h, st = s.map_reduce()
        n2 = s.norms2()
    return y, h, st["maxviol"], n2


def _inputs():
    p = workloads.dense_system(M, N, seed=606)
    rng = np.random.default_rng(7)
    xs = [p["x0"], rng.normal(0, 2, N).astype(np.float32).astype(np.float64)]
    return p, xs


def _check_against_oracle(p, b32, n2_32, x, y, h, mv, y_existing):
    """Element by element against the oracle on the binary32 values the call
    was given (b and ||a_i||^2 rounded to binary32), and against the
    existing entry point's y within the sum of the two rounding bounds."""
    b = b32.astype(np.float64)
    n2 = n2_32.astype(np.float64)
    ref = parity.MapRef(p["A"], b, x, "f32", depth=M + 8, n2=n2, levels=N // 256 + 32)
    ref.check_h(h)
    ref.check_y(y, parity.TOL["f32"])
    ref.check_maxima(mv)
    lim = 2 * (parity.TOL["f32"] * np.abs(ref.y) + ref.B)
    assert np.all(np.abs(y - y_existing) <= lim)


def test_noalloc_matches_existing_entry_point_on_two_calls():
    import torch

    _build.build()
    nsli.load()
    p, xs = _inputs()
    dev = torch.device("cuda", torch.cuda.current_device())
    A = torch.from_numpy(p["A"]).to(dev)
    b32 = p["b0"].astype(np.float32)
    b = torch.from_numpy(b32).to(dev)
    for x in xs:
        y_ref, h_ref, mv_ref, n2 = _handle_reference(p, x)
        n2_32 = n2.astype(np.float32)
        norms2 = torch.from_numpy(n2_32).to(dev)
        xt = torch.from_numpy(x.astype(np.float32)).to(dev)
        y = torch.full((N,), float("nan"), dtype=torch.float64, device=dev)
        hv = torch.zeros(1, dtype=torch.int64, device=dev)
        mv = torch.zeros(1, dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream(dev)
        nsli.map_reduce_noalloc(A, b, norms2, xt, y, hv, mv, stream=stream.cuda_stream)
        stream.synchronize()
        yc = y.cpu().numpy()
        # the existing entry point, within the tests' tolerance
        assert np.all(np.isfinite(yc))
        assert int(hv.item()) == h_ref
        assert np.linalg.norm(yc - y_ref) <= 1e-5 * np.linalg.norm(y_ref)
        assert abs(float(mv.item()) - mv_ref) <= 1e-5 * max(1.0, abs(mv_ref))
        # and the oracle, element by element
        _check_against_oracle(p, b32, n2_32, x, yc, int(hv.item()), float(mv.item()), y_ref)


def test_noalloc_padded_rows_through_the_c_abi():
    """A held with a row pitch lda = n + 3 (the C ABI's lda > n), called
    twice through ctypes with raw device pointers."""
    import torch

    _build.build()
    lib = nsli.load()
    p, xs = _inputs()
    dev = torch.device("cuda", torch.cuda.current_device())
    lda = N + 3
    Ap = torch.full((M, lda), float("nan"), dtype=torch.float32, device=dev)
    Ap[:, :N] = torch.from_numpy(p["A"]).to(dev)
    b32 = p["b0"].astype(np.float32)
    b = torch.from_numpy(b32).to(dev)
    P = ctypes.c_void_p
    for x in xs:
        y_ref, h_ref, mv_ref, n2 = _handle_reference(p, x)
        n2_32 = n2.astype(np.float32)
        norms2 = torch.from_numpy(n2_32).to(dev)
        xt = torch.from_numpy(x.astype(np.float32)).to(dev)
        y = torch.full((N,), float("nan"), dtype=torch.float64, device=dev)
        hv = torch.zeros(1, dtype=torch.int64, device=dev)
        mv = torch.zeros(1, dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream(dev)
        rc = lib.nsli_map_reduce_noalloc(M, N, P(Ap.data_ptr()), lda, P(b.data_ptr()), P(norms2.data_ptr()),
                                         P(xt.data_ptr()), P(y.data_ptr()), P(hv.data_ptr()),
                                         P(mv.data_ptr()), P(stream.cuda_stream))
        assert rc == nsli.OK
        stream.synchronize()
        yc = y.cpu().numpy()
        assert int(hv.item()) == h_ref
        assert np.linalg.norm(yc - y_ref) <= 1e-5 * np.linalg.norm(y_ref)
        _check_against_oracle(p, b32, n2_32, x, yc, int(hv.item()), float(mv.item()), y_ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch

    _build.build()
    lib = nsli.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    t = torch.zeros(4, dtype=torch.float32, device=dev)
    d = torch.zeros(4, dtype=torch.float64, device=dev)
    k = torch.zeros(1, dtype=torch.int64, device=dev)
    P = ctypes.c_void_p
    n = (1 << 20) + 1
    rc = lib.nsli_map_reduce_noalloc(1, n, P(t.data_ptr()), n, P(t.data_ptr()), P(t.data_ptr()),
                                     P(t.data_ptr()), P(d.data_ptr()), P(k.data_ptr()),
                                     P(d.data_ptr()), None)
    assert rc == nsli.ERR_UNSUPPORTED
    rc = lib.nsli_map_reduce_noalloc(0, 4, P(t.data_ptr()), 4, P(t.data_ptr()), P(t.data_ptr()),
                                     P(t.data_ptr()), P(d.data_ptr()), P(k.data_ptr()),
                                     P(d.data_ptr()), None)
    assert rc == nsli.ERR_ARG


def test_noalloc_wrapper_rejects_mistyped_tensors():
    """The binding checks dtypes, sizes and devices before calling the
    library, so a short or mistyped tensor never reaches a kernel."""
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    A = torch.zeros((8, 4), dtype=torch.float32, device=dev)
    f = lambda k: torch.zeros(k, dtype=torch.float32, device=dev)  # noqa: E731
    d = lambda k: torch.zeros(k, dtype=torch.float64, device=dev)  # noqa: E731
    i = torch.zeros(1, dtype=torch.int64, device=dev)
    good = [A, f(8), f(8), f(4), d(4), i, d(1)]
    for pos, bad in [(1, f(7)), (2, d(8)), (3, f(5)), (4, f(4)), (5, i.to(torch.int32)), (6, f(1)),
                     (0, A.to(torch.float64)), (3, torch.zeros(4))]:
        args = list(good)
        args[pos] = bad
        with pytest.raises(ValueError):
            nsli.map_reduce_noalloc(*args)
