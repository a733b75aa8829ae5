"""Serving loop with continuous batching over an nsli pool.

Requests (feasibility problems of mixed sizes) are queued on arrival and
admitted in arrival order as soon as they fit the pool's memory; every
admitted problem stays on the device (A, x, b) and advances with all other
live problems.  In the persistent mode (the default) one launch iterates
every live problem round after round until a problem stops, the caller's
`wake` test reports new work, or `epoch_s` passes; otherwise each round is
one grouped Map launch and one grouped Reduce launch.  Finished problems
are retired (x and the binary64 check read back, memory released), which
makes room for queued ones.  With `tick_s` set, the right-hand side of each
problem moves with wall-clock time: tick k = floor((now - arrival) /
tick_s), advanced on the device during a persistent launch.

The scheduling is host logic; every arithmetic step runs in libnsli.so.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import nsli


@dataclass
class Request:
    rid: int
    A: object
    b0: object
    x0: object
    Av: object = None
    params: dict = field(default_factory=dict)
    arrival: float = 0.0
    admitted: float | None = None
    finished: float | None = None
    status: int | None = None
    iters: int = 0
    x: np.ndarray | None = None
    max_viol: float | None = None
    slot: int | None = None
    stored_bytes: int = 0

    def __post_init__(self):
        m, n = int(self.A.shape[0]), int(self.A.shape[1])
        self.stored_bytes = m * n * 2   # bf16 rows streamed per iteration

    @property
    def latency(self):
        return None if self.finished is None else self.finished - self.arrival


class Server:
    def __init__(self, storage="bf16", max_bytes=0, tick_s=None, rounds_per_poll=4, stream=None,
                 clock=time.perf_counter, persistent=True, epoch_s=0.05):
        self.pool = nsli.Pool(storage=storage, max_bytes=max_bytes, stream=stream)
        self.tick_s = tick_s
        self.rounds = rounds_per_poll
        self.persistent = persistent
        self.epoch_s = epoch_s
        self.launches = 0
        self.clock = clock
        self.queue: list[Request] = []
        self.live: dict[int, Request] = {}
        self.done: list[Request] = []
        self.rounds_run = 0
        self.problem_iterations = 0   # iterations of every problem, running or finished
        self.bytes_streamed = 0       # bytes of A read by the grouped Map launches
        self.busy_s = 0.0             # wall time inside rounds + polls

    def submit(self, req: Request):
        if req.arrival == 0.0:
            req.arrival = self.clock()
        self.queue.append(req)
        return req

    def _admit(self):
        while self.queue:
            r = self.queue[0]
            slot = self.pool.add(r.A, r.b0, r.x0, Av=r.Av, **r.params)
            if slot is None:        # does not fit now: wait for memory to free up
                break
            self.queue.pop(0)
            r.slot = slot
            r.admitted = self.clock()
            self.live[slot] = r

    def _ticks(self):
        if self.tick_s is None or not self.live:
            return
        now = self.clock()
        slots = list(self.live.keys())
        ticks = [int((now - self.live[s].arrival) / self.tick_s) for s in slots]
        self.pool.set_ticks(slots, ticks)

    def _run_rounds(self, wake):
        """Advance every live problem; returns the rounds run."""
        if not self.persistent:
            self.pool.step(self.rounds)
            return self.rounds
        t0 = self.clock()
        self.pool.launch(max_seconds=self.epoch_s, tick_s=self.tick_s or 0.0)
        self.launches += 1
        while True:
            if self.pool.stopped() > 0 or (wake is not None and wake()):
                self.pool.yield_()
                break
            if self.clock() - t0 > self.epoch_s:
                break
            time.sleep(0.0001)
        return self.pool.wait()

    def pump(self, wake=None):
        """Admit what fits, advance the live problems (until something
        stopped or `wake()` reports new work), retire what finished."""
        self._admit()
        if not self.live:
            return 0
        self._ticks()
        t0 = self.clock()
        running = [r for r in self.live.values() if r.status is None]
        rounds = self._run_rounds(wake)
        self.rounds_run += rounds
        finished = self.pool.poll()
        now = self.clock()
        self.busy_s += now - t0
        fin_slots = {f[0]: f[2] for f in finished}
        for r in running:
            # a running problem advances one iteration per round until it stops
            done_iters = fin_slots.get(r.slot)
            step = rounds if done_iters is None else max(0, done_iters - r.iters)
            self.problem_iterations += step
            self.bytes_streamed += step * r.stored_bytes
            if done_iters is None:
                r.iters += rounds
        for slot, status, iters in finished:
            r = self.live.pop(slot)
            r.status, r.iters = status, iters
            r.x = self.pool.get_x(slot, int(r.x0.shape[0]))
            r.max_viol = self.pool.residual_max(slot)[0]
            r.finished = now
            self.pool.remove(slot)
            self.done.append(r)
        return len(finished)

    def drain(self, timeout_s=None):
        t0 = self.clock()
        while self.queue or self.live:
            self.pump()
            if timeout_s is not None and self.clock() - t0 > timeout_s:
                break
        return self.done

    def close(self):
        self.pool.close()
