"""Row shards (ModAPL, Section 3) on one GPU, through the C ABI.

One system is split into contiguous row blocks held by separate handles on
the same device and stream (one per worker); each worker's nsli_shard_map
writes its record straight into its row of the records array (what the
allgather of a multi-GPU run delivers), then nsli_shard_step runs on every
worker.  Every worker must hold the same iterate bit for bit; each step must
equal the oracle's step from the same x_k element by element; and the run
must match one handle over all rows within the parity tolerance."""
import numpy as np
import pytest

import oracle
import parity
from paper_2003_09956_gb300 import nsli, shard, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session", autouse=True)
def built_library():
    from paper_2003_09956_gb300 import _build
    _build.build()
    nsli.load()


def _workers(p, R, storage, stream):
    m = p["A"].shape[0]
    out = []
    for w in range(R):
        r0, r1 = shard.row_range(m, R, w)
        src = p["A"][r0:r1] if storage != "f64" else p["A"][r0:r1].astype(np.float64)
        out.append(nsli.Solver(np.ascontiguousarray(src), p["b0"][r0:r1], p["x0"], Av=p["Av"][r0:r1],
                               storage=storage, stream=stream.cuda_stream))
    return out


def _stored(A32, storage):
    if storage == "bf16":
        return oracle.quantize_bf16(A32)
    if storage == "fp8":
        return np.concatenate([oracle.quantize_e4m3_rows(A32[i:i + 1])[0] for i in range(A32.shape[0])])
    return A32


@pytest.mark.parametrize("R", [2, 3])
@pytest.mark.parametrize("storage,rule", [("f32", "relaxed"), ("bf16", "modap"), ("f64", "relaxed"),
                                          ("fp8", "relaxed")])
def test_sharded_steps_match_oracle_and_single_handle(R, storage, rule):
    import torch
    m, n, K = 1201, 300, 12
    rho, lam = 1e-3, (1.0 if rule == "relaxed" else 0.5)
    p = workloads.dense_system(m, n, seed=700 + R)
    A_eff = _stored(p["A"], storage)
    stream = torch.cuda.Stream()
    ws = _workers(p, R, storage, stream)
    recs = torch.zeros((R, shard.HEADER + n), dtype=torch.float64, device="cuda")
    try:
        for s in ws:
            s.shard_begin(lam=lam, rule=rule, stop="none", max_iter=1 << 40, rho=rho)
        n2, _ = oracle.norms2(A_eff)
        G = parity.num_sms()
        depth = parity.dense_y_depth(m // R + 1, G) + R + 2
        for k in range(K):
            xk = ws[0].get_x()
            for w, s in enumerate(ws):
                s.shard_map(recs[w])
            for s in ws:
                s.shard_step(recs)
            xs = [s.get_x() for s in ws]
            for x in xs[1:]:
                np.testing.assert_array_equal(x, xs[0])
            res = ws[0].result()
            assert res["tick"] == k + 1 and res["iters"] == k + 1
            parity.check_step(xk, xs[0], int(recs[:, 0].sum().item()), A_eff, oracle.tick_b(p["b0"], p["Av"], rho, k), storage,
                              depth=depth, lam=lam, rule=rule, n2=n2, levels=parity.dot_levels(n))
        src = p["A"] if storage != "f64" else p["A"].astype(np.float64)
        with nsli.Solver(src, p["b0"], p["x0"], Av=p["Av"], storage=storage) as one:
            one.iterate(K, lam=lam, rule=rule, rho=rho)
            x1 = one.get_x()
        assert np.linalg.norm(xs[0] - x1) <= parity.TOL[storage] * np.linalg.norm(x1 - p["x0"]) * 10 + \
            1e-12 * np.linalg.norm(x1)
    finally:
        for s in ws:
            s.close()


def test_sharded_sparse_workers():
    """Compressed-row workers: the same exchange, same bits on every worker."""
    import torch
    p = workloads.sparse_system(2000, 500, 9, seed=711)
    A = workloads.csr_to_dense(p["rp"], p["ci"], p["val"], p["n"])
    n2, _ = oracle.norms2(A)
    R, rho, K = 2, 1e-3, 8
    stream = torch.cuda.Stream()
    ws = []
    for w in range(R):
        r0, r1 = shard.row_range(p["m"], R, w)
        a, b = p["rp"][r0], p["rp"][r1]
        ws.append(nsli.SparseSolver(r1 - r0, p["n"], p["rp"][r0:r1 + 1] - a, p["ci"][a:b], p["val"][a:b],
                                    p["b0"][r0:r1], p["x0"], Av=p["Av"][r0:r1], storage="f64",
                                    stream=stream.cuda_stream))
    recs = torch.zeros((R, shard.HEADER + p["n"]), dtype=torch.float64, device="cuda")
    try:
        for s in ws:
            s.shard_begin(stop="none", max_iter=1 << 40, rho=rho)
        for k in range(K):
            xk = ws[0].get_x()
            for w, s in enumerate(ws):
                s.shard_map(recs[w])
            for s in ws:
                s.shard_step(recs)
            xs = [s.get_x() for s in ws]
            np.testing.assert_array_equal(xs[1], xs[0])
            parity.check_step(xk, xs[0], int(recs[:, 0].sum().item()), A, oracle.tick_b(p["b0"], p["Av"], rho, k), "f64",
                              depth=2000, n2=n2, levels=64)
    finally:
        for s in ws:
            s.close()


class LocalExchange:
    """The exchange of a one-worker group (no other process)."""
    world, rank = 1, 0

    def allgather(self, rec, recs):
        recs.copy_(rec)

    def allreduce_max(self, values):
        return list(values)


@pytest.mark.parametrize("stop,eps", [("maxviol_rel", 1e-6), ("step", 1e-8)])
def test_sharded_run_solve_on_device(stop, eps):
    """The product's control flow (shard.ShardedRun with DeviceOps) on one
    worker: a solve to the oracle's iteration count (within 1%)."""
    if stop == "step":
        p = workloads.model_system(256, seed=0)
        storage = "f64"
        A_eff = p["A"]
    else:
        p = workloads.dense_system(256, 48, seed=21, x0_std=1.0)
        storage = "f32"
        A_eff = p["A"]
    ref = oracle.solve(A_eff, p["b0"], p["x0"], stop={"step": oracle.STOP_STEP,
                                                       "maxviol_rel": oracle.STOP_MAXVIOL_REL}[stop],
                       eps=eps, max_iter=400000)
    assert ref["status"] == oracle.OK
    import torch
    stream = torch.cuda.Stream()
    with nsli.Solver(p["A"], p["b0"], p["x0"], storage=storage, stream=stream.cuda_stream) as s:
        run = shard.ShardedRun(shard.DeviceOps(s, stream), LocalExchange())
        res = run.solve(stop=stop, eps=eps, max_iter=400000, block_iters=64)
    assert res["status"] == nsli.OK
    assert abs(res["iters"] - ref["iters"]) <= max(2, 0.01 * ref["iters"]), (res["iters"], ref["iters"])
    if stop == "maxviol_rel":
        assert res["max_viol"] <= eps * res["max_abs_b"]


def test_shard_argument_errors():
    import torch
    p = workloads.dense_system(100, 20, seed=3)
    with nsli.Solver(p["A"], p["b0"], p["x0"]) as s:
        recs = torch.zeros((2, shard.HEADER + 20), dtype=torch.float64, device="cuda")
        with pytest.raises(nsli.NsliError) as e:
            s.shard_step(recs)                      # before nsli_shard_begin
        assert e.value.code == nsli.ERR_ARG
        with pytest.raises(ValueError):
            s.shard_map(torch.zeros(shard.HEADER + 19, dtype=torch.float64, device="cuda"))
        with pytest.raises(ValueError):
            s.shard_step(torch.zeros((2, shard.HEADER + 20), dtype=torch.float32, device="cuda"))
