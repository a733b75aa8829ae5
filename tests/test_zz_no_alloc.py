"""The allocation-free Map + Reduce entry point.

Callers that cannot allocate device memory (code running while a stream is
captured into a CUDA graph, or under a fixed memory budget / a host
framework's own allocator) use nsli_map_reduce_noalloc, whose scratch is a
fixed array inside the library.  Its results must agree with the existing,
allocating entry point nsli_map_reduce on the same system, on two calls in a
row (the second one with another x, so stale scratch from the first call
would show).  This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_2003_09956_gb300 import _build, nsli, workloads

pytestmark = pytest.mark.gpu


def _handle_reference(p, x):
    """y, h and max r from the existing entry point (handle, binary32 storage)."""
    with nsli.Solver(p["A"], p["b0"], x, storage="f32") as s:
        y, h, st = s.map_reduce()
        n2 = s.norms2()
    return y, h, st["maxviol"], n2


def test_noalloc_matches_existing_entry_point_on_two_calls():
    import torch

    _build.build()
    nsli.load()
    m, n = 3001, 1000
    p = workloads.dense_system(m, n, seed=606)
    rng = np.random.default_rng(7)
    xs = [p["x0"], rng.normal(0, 2, n).astype(np.float32).astype(np.float64)]
    A64 = p["A"].astype(np.float64)
    dev = torch.device("cuda", torch.cuda.current_device())
    A = torch.from_numpy(p["A"]).to(dev)
    b = torch.from_numpy(p["b0"].astype(np.float32)).to(dev)
    for x in xs:
        # both classifications must be unambiguous for an exact count check
        r = A64 @ x - p["b0"]
        assert np.min(np.abs(r)) > 1e-4 * np.max(np.abs(r))
    for x in xs:
        y_ref, h_ref, mv_ref, n2 = _handle_reference(p, x)
        norms2 = torch.from_numpy(n2.astype(np.float32)).to(dev)
        xt = torch.from_numpy(x.astype(np.float32)).to(dev)
        y = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
        hv = torch.zeros(1, dtype=torch.int64, device=dev)
        mv = torch.zeros(1, dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream(dev)
        nsli.map_reduce_noalloc(A, b, norms2, xt, y, hv, mv, stream=stream.cuda_stream)
        stream.synchronize()
        yc = y.cpu().numpy()
        assert np.all(np.isfinite(yc))
        assert int(hv.item()) == h_ref
        rel = np.linalg.norm(yc - y_ref) / np.linalg.norm(y_ref)
        assert rel <= 1e-5, rel
        assert abs(float(mv.item()) - mv_ref) <= 1e-5 * max(1.0, abs(mv_ref))


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
