"""Row-sharded runs of one system over a process group: ModAPL (Section 3).

Section 3 splits the list of inequalities into sublists, one per worker;
every worker maps and reduces its sublist, the partial results are added,
and the step is taken with the sums.  Here worker w (rank w of a
torch.distributed process group, normally one GPU each) holds the rows
``row_range(m, R, w)`` of the system, with the same x0 everywhere.  One
iteration is

    ops.map(rec)                    Map + local Reduce of the worker's rows
    exchange(rec, recs)             allgather of the R records, worker order
    ops.step(recs)                  global Reduce (fixed worker order), stop
                                    decision and step, on every worker alike

and the iterates of all workers stay bit-identical without a broadcast of
x (every worker adds the same records in the same order).  The only other
exchange is the binary64 check of a stop candidate: every worker checks its
own rows and the maxima are combined with an all-reduce (MAX).

``ShardedRun`` holds that control flow and nothing of the method's
arithmetic; the local operations come from ``ops``: ``DeviceOps`` calls
the C ABI (nsli_shard_begin / nsli_shard_map / nsli_shard_step on one
handle per worker).  The exchange is a plain allgather of
``SHARD_HEADER + n`` doubles per worker (NCCL on GPUs, gloo on CPUs); no
peer memory is read by a kernel.
"""
from __future__ import annotations

from . import nsli

HEADER = nsli.SHARD_HEADER
STATUS_RUNNING, STATUS_CANDIDATE = nsli.RUNNING, nsli.CANDIDATE


def row_range(m: int, world: int, rank: int) -> tuple[int, int]:
    """Rows [r0, r1) of worker `rank` among `world`: contiguous, balanced
    (sizes differ by at most one), in rank order."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    return m * rank // world, m * (rank + 1) // world


class DeviceOps:
    """A worker's local steps through the C ABI, on one nsli handle (a
    ``nsli.Solver`` or ``nsli.SparseSolver`` over the worker's rows) that
    was created on the torch CUDA stream ``stream``.  The exchange runs on
    that stream too (``stream_context``), so the allgather is ordered after
    the Map that wrote the record and before the step that reads the
    gathered records, without a host synchronisation."""

    def __init__(self, solver, stream):
        self.solver = solver
        self.stream = stream
        self.n = solver.n

    def stream_context(self):
        import torch
        return torch.cuda.stream(self.stream)

    def new_records(self, rows):
        import torch
        return torch.zeros((rows, HEADER + self.n), dtype=torch.float64,
                           device=torch.device("cuda", torch.cuda.current_device()))

    def begin(self, params: dict):
        self.solver.shard_begin(**params)

    def map(self, rec):
        self.solver.shard_map(rec)

    def step(self, recs, force_step=False):
        self.solver.shard_step(recs, force_step=force_step)

    def progress(self) -> dict:
        return self.solver.result()

    def check(self):
        mv, mn, mb, _ = self.solver.check()
        return mv, mn, mb

    def get_x(self):
        return self.solver.get_x()


class TorchExchange:
    """Allgather and MAX all-reduce over a torch.distributed process group."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)

    def allgather(self, rec, recs):
        self.dist.all_gather_into_tensor(recs.view(-1), rec.view(-1), group=self.group)

    def allreduce_max(self, values):
        import torch
        t = torch.tensor(values, dtype=torch.float64)
        if self.dist.get_backend(self.group) == "nccl":
            t = t.cuda()
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        return [float(v) for v in t.cpu()]


class ShardedRun:
    """The control flow of a row-sharded run on one worker."""

    def __init__(self, ops, exchange):
        self.ops = ops
        self.ex = exchange
        self.rec = ops.new_records(1)
        self.recs = ops.new_records(exchange.world)
        self.force = False

    def _iteration(self):
        self.ops.map(self.rec)
        with self.ops.stream_context():
            self.ex.allgather(self.rec, self.recs)
        self.ops.step(self.recs, force_step=self.force)
        self.force = False

    def iterate(self, n_iter, lam=1.0, rule="relaxed", rho=0.0):
        """n_iter iterations, no stop test (the timed form)."""
        self.ops.begin(dict(lam=lam, rule=rule, stop="none", eps=0.0, max_iter=1 << 62, rho=rho))
        for _ in range(int(n_iter)):
            self._iteration()

    def solve(self, lam=1.0, rule="relaxed", stop="maxviol_rel", eps=1e-6, max_iter=100000, rho=0.0,
              block_iters=32) -> dict:
        """Until the stop rule holds (a candidate confirmed by the binary64
        check over all workers' rows), the step rule, or max_iter updates."""
        self.ops.begin(dict(lam=lam, rule=rule, stop=stop, eps=eps, max_iter=max_iter, rho=rho))
        self.force = False
        rejected = 0
        status = nsli.NOT_CONVERGED
        # every block makes block_iters updates or ends the run; a rejected
        # candidate forces one update, so this bound is never reached
        for _ in range(max_iter // max(1, block_iters) + max_iter + 4):
            for _ in range(block_iters):
                self._iteration()
            st = self.ops.progress()["status"]
            if st == STATUS_RUNNING:
                continue
            if st == STATUS_CANDIDATE:
                mv, mn, mb = self.ex.allreduce_max(list(self.ops.check()))
                if stop == "epsmem":
                    accept = mn < eps
                elif stop == "maxviol_rel":
                    accept = mv <= eps * mb
                else:
                    accept = mv <= 0.0          # h = 0: no row with r_i > 0
                if accept:
                    status = nsli.OK
                    break
                rejected += 1
                self.force = True
                continue
            status = st
            break
        res = dict(self.ops.progress())
        mv, mn, mb = self.ex.allreduce_max(list(self.ops.check()))
        res.update(status=status, rejected=rejected, max_viol=mv, max_viol_norm=mn, max_abs_b=mb)
        return res
