"""Row-sharded runs (ModAPL, Section 3) with two and three gloo ranks on CPU.

Every rank runs the product's control flow (shard.ShardedRun: Map, allgather
of the records in rank order, global Reduce + step, binary64 check of stop
candidates with a MAX all-reduce) on its own contiguous rows, with the local
steps done by the FP64 oracle (OracleOps below: oracle.map_reduce on the
rank's rows, oracle.combine_step on the gathered records).  The trajectory
must equal the single-process oracle on the whole system to rounding, and
every rank must hold the same iterate bit for bit."""
import contextlib
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from paper_2003_09956_gb300 import nsli, shard, workloads

STOPS = {"none": oracle.STOP_NONE, "step": oracle.STOP_STEP, "epsmem": oracle.STOP_EPSMEM,
         "maxviol_rel": oracle.STOP_MAXVIOL_REL}
RULES = {"relaxed": oracle.RULE_RELAXED, "modap": oracle.RULE_MODAP}


class OracleOps:
    """A worker's local steps on the CPU with the FP64 oracle, with the
    device state machine of nsli_shard_step (candidate, step rule, cap)."""

    def __init__(self, A, b0, Av, x0):
        self.A, self.b0, self.Av = A, b0, Av
        self.n2, _ = oracle.norms2(A)
        self.x = np.array(x0, dtype=np.float64)
        self.n = self.x.shape[0]
        self.tick = 0
        self.it = 0
        self.status = nsli.RUNNING
        self.h = 0

    def new_records(self, rows):
        return torch.zeros((rows, shard.HEADER + self.n), dtype=torch.float64)

    def stream_context(self):
        return contextlib.nullcontext()

    def begin(self, params):
        self.p = dict(params)
        self.it = 0
        self.status = nsli.RUNNING

    def _b(self):
        return oracle.tick_b(self.b0, self.Av, self.p["rho"], self.tick)

    def map(self, rec):
        mr = oracle.map_reduce(self.A, self._b(), self.n2, self.x) if self.A.shape[0] else \
            {"y": np.zeros(self.n), "h": 0, "maxviol": -np.inf, "maxnorm": -np.inf, "maxb": 0.0}
        rec.view(-1)[:shard.HEADER] = torch.tensor([mr["h"], mr["maxviol"], mr["maxnorm"], mr["maxb"]])
        rec.view(-1)[shard.HEADER:] = torch.from_numpy(mr["y"])

    def step(self, recs, force_step=False):
        if self.status != nsli.RUNNING and not force_step:
            return
        r = recs.numpy()
        records = [{"h": int(q[0]), "maxviol": q[1], "maxnorm": q[2], "maxb": q[3], "y": q[shard.HEADER:]}
                   for q in r]
        stop, eps = STOPS[self.p["stop"]], self.p["eps"]
        code, x1, st, _ = oracle.combine_step(records, self.x, lam=self.p["lam"], rule=RULES[self.p["rule"]],
                                              stop=stop, eps=eps, force_step=force_step)
        self.h = st["h"]
        if code == oracle.IT_CONVERGED:
            self.status = nsli.CANDIDATE
            return
        if self.it >= self.p["max_iter"]:
            self.status = nsli.NOT_CONVERGED
            return
        self.status = nsli.RUNNING
        self.x = x1
        self.it += 1
        self.tick += 1
        if code == oracle.IT_STEP_STOP:
            self.status = nsli.OK

    def progress(self):
        return {"status": self.status, "iters": self.it, "tick": self.tick, "h": self.h}

    def check(self):
        if not self.A.shape[0]:
            return -np.inf, -np.inf, 0.0
        mr = oracle.map_reduce(self.A, self._b(), self.n2, self.x)
        return mr["maxviol"], mr["maxnorm"], mr["maxb"]

    def get_x(self):
        return self.x.copy()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _system(kind):
    if kind == "model":
        p = workloads.model_system(48, seed=5)
        return p["A"], p["b0"], np.zeros(p["m"]), p["x0"]
    p = workloads.dense_system(301, 23, seed=8, x0_std=1.0)
    return p["A"].astype(np.float64), p["b0"], p["Av"], p["x0"]


def _worker(rank, world, port, kind, args, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        A, b0, Av, x0 = _system(kind)
        r0, r1 = shard.row_range(A.shape[0], world, rank)
        ops = OracleOps(np.ascontiguousarray(A[r0:r1]), b0[r0:r1], Av[r0:r1], x0)
        run = shard.ShardedRun(ops, shard.TorchExchange())
        if args["mode"] == "iterate":
            run.iterate(args["K"], lam=args["lam"], rule=args["rule"], rho=args["rho"])
            res = ops.progress()
        else:
            res = run.solve(lam=args["lam"], rule=args["rule"], stop=args["stop"], eps=args["eps"],
                            max_iter=args["max_iter"], block_iters=args["block"])
        out.put((rank, res, ops.get_x()))
    finally:
        dist.destroy_process_group()


def _run(world, kind, args):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, kind, args, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("rule", ["relaxed", "modap"])
def test_sharded_trajectory_equals_single_process_oracle(world, rule):
    lam, rho, K = (1.0 if rule == "relaxed" else 0.3), 1e-2, 25
    res = _run(world, "dense", dict(mode="iterate", K=K, lam=lam, rule=rule, rho=rho))
    A, b0, Av, x0 = _system("dense")
    ref = oracle.solve(A, b0, x0, Av=Av, rho=rho, lam=lam, rule=RULES[rule], stop=oracle.STOP_NONE,
                       max_iter=K)
    for rank, r, x in res:
        assert r["iters"] == K and r["tick"] == K
        np.testing.assert_array_equal(x, res[0][2])          # every worker: the same bits
    np.testing.assert_allclose(res[0][2], ref["x"], rtol=1e-12, atol=1e-12 * np.abs(ref["x"]).max())


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("stop,eps", [("step", 1e-8), ("maxviol_rel", 1e-6), ("epsmem", 1e-6)])
def test_sharded_solve_matches_oracle_solve(world, stop, eps):
    """The model system (n = 48) solved to each stop rule: the sharded run
    stops after the oracle's iteration count (within 1%), with a binary64
    confirmed result."""
    res = _run(world, "model", dict(mode="solve", lam=1.0, rule="relaxed", stop=stop, eps=eps,
                                    max_iter=200000, block=16))
    A, b0, Av, x0 = _system("model")
    ref = oracle.solve(A, b0, x0, stop=STOPS[stop], eps=eps, max_iter=200000)
    assert ref["status"] == oracle.OK
    for rank, r, x in res:
        assert r["status"] == nsli.OK
        assert abs(r["iters"] - ref["iters"]) <= max(1, 0.01 * ref["iters"])
        np.testing.assert_array_equal(x, res[0][2])
    mb = np.abs(b0).max()
    np.testing.assert_allclose(res[0][2], ref["x"], rtol=0, atol=1e-6 * mb)
    if stop == "maxviol_rel":
        assert res[0][1]["max_viol"] <= eps * res[0][1]["max_abs_b"]


def test_sharded_solve_hits_the_cap():
    res = _run(2, "model", dict(mode="solve", lam=1.0, rule="relaxed", stop="step", eps=1e-14,
                                max_iter=40, block=16))
    for rank, r, x in res:
        assert r["status"] == nsli.NOT_CONVERGED and r["iters"] == 40


def test_row_ranges_cover_the_rows_once():
    for m in (1, 2, 7, 100, 131072):
        for world in (1, 2, 3, 8):
            rs = [shard.row_range(m, world, w) for w in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == m
            assert all(rs[w][1] == rs[w + 1][0] for w in range(world - 1))
            sizes = [b - a for a, b in rs]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.row_range(10, 2, 2)
