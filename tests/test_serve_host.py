"""The serving loop's host logic (serve.Server) on the CPU, with a fake pool
in place of nsli.Pool: admission in arrival order while memory allows, the
persistent launch loop (yield when a problem stopped or new work arrived),
per-request iteration counts, and retirement that frees memory for queued
requests."""
import numpy as np

from paper_2003_09956_gb300 import nsli, serve


class FakePool:
    """Problems of a given size finish after `need` rounds; the memory
    budget admits `cap` problems at a time; a launch runs until a problem
    stops (the fake has no wall clock)."""

    def __init__(self, cap, need):
        self.cap, self.need = cap, need
        self.live = {}           # slot -> [rounds done, need]
        self.next_slot = 0
        self.running = False
        self.stopped_count = 0
        self.launches = 0
        self.yields = 0
        self.removed = []

    def add(self, A, b0, x0, Av=None, **params):
        if len(self.live) >= self.cap:
            return None
        s = self.next_slot
        self.next_slot += 1
        self.live[s] = [0, self.need[int(A.shape[1])], params.get("max_iter", 1 << 40)]
        return s

    def set_ticks(self, slots, ticks):
        assert all(s in self.live for s in slots)

    def launch(self, max_rounds=1 << 40, max_seconds=1.0, tick_s=0.0):
        assert not self.running
        self.running = True
        self.launches += 1
        self.rounds = 0
        # run rounds until some running problem stops
        while True:
            running = [v for v in self.live.values() if v[0] < min(v[1], v[2])]
            if not running:
                break
            for v in running:
                v[0] += 1
            self.rounds += 1
            if any(v[0] >= min(v[1], v[2]) for v in running):
                break
        self.stopped_count = sum(1 for v in self.live.values() if v[0] >= min(v[1], v[2]))

    def stopped(self):
        return self.stopped_count if self.running else 0

    def yield_(self):
        self.yields += 1

    def wait(self):
        self.running = False
        return self.rounds

    def poll(self):
        out = []
        for s, v in self.live.items():
            if v[0] >= min(v[1], v[2]):
                out.append((s, nsli.OK if v[0] >= v[1] else nsli.NOT_CONVERGED, v[0]))
        return out

    def get_x(self, slot, n):
        return np.full(n, float(slot))

    def residual_max(self, slot):
        return 0.0, 0.0

    def remove(self, slot):
        del self.live[slot]
        self.removed.append(slot)

    def launch_count(self):
        return self.launches

    def close(self):
        pass


def make_server(pool):
    srv = serve.Server.__new__(serve.Server)
    srv.pool = pool
    srv.tick_s = 0.01
    srv.rounds = 4
    srv.persistent = True
    srv.epoch_s = 10.0
    srv.launches = 0
    srv.clock = iter(range(10 ** 6)).__next__
    srv.queue, srv.live, srv.done = [], {}, []
    srv.rounds_run = srv.problem_iterations = srv.bytes_streamed = 0
    srv.busy_s = 0.0
    return srv


def request(rid, n, budget=10 ** 6):
    A = np.zeros((2 * n, n), np.float32)
    return serve.Request(rid, A, np.zeros(2 * n), np.zeros(n), params={"max_iter": budget}, arrival=0.0)


def test_admission_order_retirement_and_iteration_counts():
    need = {10: 3, 20: 7, 30: 5}
    pool = FakePool(cap=2, need=need)
    srv = make_server(pool)
    for rid, n in enumerate([10, 20, 30, 10]):
        srv.submit(request(rid, n))
    guard = 0
    while (srv.queue or srv.live) and guard < 50:
        srv.pump()
        guard += 1
    assert not srv.queue and not srv.live
    done = {r.rid: r for r in srv.done}
    assert sorted(done) == [0, 1, 2, 3]
    for rid, n in enumerate([10, 20, 30, 10]):
        assert done[rid].status == nsli.OK and done[rid].iters == need[n]
    # arrival order: request 2 was admitted only after request 0 retired
    assert done[2].admitted > done[0].finished - 1
    assert pool.removed.index(0) < pool.removed.index(3)
    # every iteration was counted once
    assert srv.problem_iterations == sum(need[n] for n in [10, 20, 30, 10])
    # a launch ends when a problem stops: the loop yielded each time
    assert pool.yields == pool.launches


def test_budget_ends_a_request_not_converged():
    pool = FakePool(cap=4, need={10: 50})
    srv = make_server(pool)
    srv.submit(request(0, 10, budget=12))
    while srv.queue or srv.live:
        srv.pump()
    r = srv.done[0]
    assert r.status == nsli.NOT_CONVERGED and r.iters == 12


def test_wake_ends_a_launch_for_new_work():
    """The caller's wake test (a request arrived) makes the loop yield even
    when no problem stopped."""
    class SlowPool(FakePool):
        def launch(self, **kw):
            self.running = True
            self.launches += 1
            self.rounds = 1
            for v in self.live.values():
                v[0] += 1
            self.stopped_count = 0

    pool = SlowPool(cap=4, need={10: 100})
    srv = make_server(pool)
    srv.submit(request(0, 10))
    srv.pump(wake=lambda: True)
    assert pool.yields == 1 and srv.live and srv.problem_iterations == 1
