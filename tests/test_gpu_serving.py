"""Continuous batching (pool / server) through the C ABI.

The key property: a problem's iterates do not depend on which other
problems share the grouped launches, when they were admitted, or how many
are live (iteration-indexed ticks or rho = 0 make the result timing-free)."""
import numpy as np
import pytest

import oracle
import parity
from paper_2003_09956_gb300 import nsli, serve, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session", autouse=True)
def built_library():
    from paper_2003_09956_gb300 import _build
    _build.build()
    nsli.load()


SIZES = [(130, 64, 2), (400, 100, 4), (2056, 257, 8), (1000, 500, 2), (4100, 1024, 4), (3000, 1500, 2)]


def problems(seed=0):
    out = []
    for q, (m, n, c) in enumerate(SIZES):
        p = workloads.dense_system(m, n, seed=seed + 31 * q)
        out.append(p)
    return out


def run_alone(p, K, storage, rho):
    with nsli.Pool(storage=storage) as pool:
        s = pool.add(p["A"], p["b0"], p["x0"], Av=p["Av"], stop="none", max_iter=K, rho=rho)
        for _ in range(K + 10):
            pool.step(3)
            fin = pool.poll()
            if fin:
                assert fin[0][1] == nsli.NOT_CONVERGED and fin[0][2] == K
                return pool.get_x(s, p["n"])
        raise AssertionError("problem did not finish after its max_iter rounds")


@pytest.mark.parametrize("storage", ["bf16", "f32"])
def test_pool_results_identical_alone_and_in_the_mix(storage):
    K, rho = 12, 1e-3
    probs = problems()
    alone = [run_alone(p, K, storage, rho) for p in probs]
    with nsli.Pool(storage=storage) as pool:
        slots = {}
        # staggered admission: half now, half after a few rounds
        for q in range(0, len(probs), 2):
            p = probs[q]
            slots[q] = pool.add(p["A"], p["b0"], p["x0"], Av=p["Av"], stop="none", max_iter=K, rho=rho)
        pool.step(4)
        for q in range(1, len(probs), 2):
            p = probs[q]
            slots[q] = pool.add(p["A"], p["b0"], p["x0"], Av=p["Av"], stop="none", max_iter=K, rho=rho)
        finished = {}
        for _ in range(40):
            pool.step(2)
            for slot, status, iters in pool.poll():
                finished[slot] = (status, iters)
            if len(finished) == len(probs):
                break
        assert len(finished) == len(probs)
        for q, p in enumerate(probs):
            assert finished[slots[q]] == (nsli.NOT_CONVERGED, K)
            np.testing.assert_array_equal(pool.get_x(slots[q], p["n"]), alone[q])


def test_pool_matches_single_problem_solver_and_oracle():
    K, rho = 6, 1e-3
    p = workloads.dense_system(3000, 700, seed=404)
    xa = run_alone(p, K, "bf16", rho)
    with nsli.Solver(p["A"], p["b0"], p["x0"], Av=p["Av"], storage="bf16") as s:
        s.iterate(K, rho=rho)
        xs = s.get_x()
    assert np.linalg.norm(xa - xs) <= 1e-5 * np.linalg.norm(xs)
    A_eff = oracle.quantize_bf16(p["A"])
    ref = oracle.solve(A_eff, p["b0"], p["x0"], Av=p["Av"], rho=rho, stop=oracle.STOP_NONE, max_iter=K)
    assert np.linalg.norm(xa - ref["x"]) <= 1e-5 * np.linalg.norm(ref["x"])


def test_pool_admission_by_memory_budget():
    p1 = workloads.dense_system(2000, 512, seed=1)
    p2 = workloads.dense_system(2000, 512, seed=2)
    with nsli.Pool(storage="bf16") as probe:
        s = probe.add(p1["A"], p1["b0"], p1["x0"], stop="none", max_iter=1)
        one = probe.bytes_used()
        assert s is not None and one > 0
    with nsli.Pool(storage="bf16", max_bytes=int(one * 1.5)) as pool:
        s1 = pool.add(p1["A"], p1["b0"], p1["x0"], stop="none", max_iter=3)
        assert s1 is not None
        assert pool.add(p2["A"], p2["b0"], p2["x0"], stop="none", max_iter=3) is None
        assert pool.live() == 1 and pool.bytes_used() == one
        pool.remove(s1)
        assert pool.live() == 0 and pool.bytes_used() == 0
        s2 = pool.add(p2["A"], p2["b0"], p2["x0"], stop="none", max_iter=3)
        assert s2 is not None


@pytest.mark.parametrize("persistent", [True, False])
def test_server_continuous_batching_to_feasibility(persistent):
    """Requests arrive while others run; each is admitted when memory frees
    up; every result equals the same request solved alone, and converged
    ones pass the binary64 check (persistent launches and grouped launches)."""
    reqs_spec = []
    for q in range(8):
        n = [32, 48, 64, 40, 56, 72, 36, 60][q]
        p = workloads.dense_system(4 * n, n, seed=900 + q, x0_std=0.5)
        reqs_spec.append(p)
    params = dict(stop="maxviol_rel", eps=1e-6, max_iter=50000, rho=0.0)
    # alone
    alone = []
    for p in reqs_spec:
        srv = serve.Server(storage="f32", rounds_per_poll=16, persistent=persistent)
        r = srv.submit(serve.Request(0, p["A"], p["b0"], p["x0"], params=params))
        srv.drain(timeout_s=120)
        alone.append(r)
        srv.close()
    one = nsli.Pool(storage="f32")
    s = one.add(reqs_spec[0]["A"], reqs_spec[0]["b0"], reqs_spec[0]["x0"], stop="none", max_iter=1)
    budget = int(one.bytes_used() * 3.5)   # about three small problems at a time
    one.close()
    srv = serve.Server(storage="f32", max_bytes=budget, rounds_per_poll=16, persistent=persistent)
    reqs = []
    for q, p in enumerate(reqs_spec):
        reqs.append(srv.submit(serve.Request(q, p["A"], p["b0"], p["x0"], params=params)))
        srv.pump()
    srv.drain(timeout_s=300)
    srv.close()
    for q, r in enumerate(reqs):
        a = alone[q]
        assert r.status == a.status == nsli.OK
        assert r.iters == a.iters
        np.testing.assert_array_equal(r.x, a.x)
        maxb = np.abs(reqs_spec[q]["b0"]).max()
        assert r.max_viol <= 1e-6 * maxb


# ------------------------------------------------------------ persistent launches

def run_alone_persistent(p, K, storage, rho):
    with nsli.Pool(storage=storage) as pool:
        s = pool.add(p["A"], p["b0"], p["x0"], Av=p["Av"], stop="none", max_iter=K, rho=rho)
        pool.launch(max_seconds=30.0)
        rounds = pool.wait()
        fin = pool.poll()
        assert rounds == K + 1 or rounds == K, rounds   # the launch ends once nothing runs
        assert fin == [(s, nsli.NOT_CONVERGED, K)]
        return pool.get_x(s, p["n"])


@pytest.mark.parametrize("storage", ["bf16", "f32"])
def test_persistent_results_identical_alone_and_in_the_mix(storage):
    """One persistent launch over problems of mixed sizes, admitted at two
    different times (two launches): every problem's iterate equals, bit for
    bit, the same problem run alone."""
    K, rho = 12, 1e-3
    probs = problems()
    alone = [run_alone_persistent(p, K, storage, rho) for p in probs]
    with nsli.Pool(storage=storage) as pool:
        slots = {}
        for q in range(0, len(probs), 2):
            p = probs[q]
            slots[q] = pool.add(p["A"], p["b0"], p["x0"], Av=p["Av"], stop="none", max_iter=K, rho=rho)
        pool.launch(max_rounds=4, max_seconds=30.0)
        assert pool.wait() == 4
        assert pool.poll() == []
        for q in range(1, len(probs), 2):
            p = probs[q]
            slots[q] = pool.add(p["A"], p["b0"], p["x0"], Av=p["Av"], stop="none", max_iter=K, rho=rho)
        finished = {}
        for _ in range(10):
            pool.launch(max_seconds=30.0)
            pool.wait()
            for slot, status, iters in pool.poll():
                finished[slot] = (status, iters)
            if len(finished) == len(probs):
                break
        assert len(finished) == len(probs)
        for q, p in enumerate(probs):
            assert finished[slots[q]] == (nsli.NOT_CONVERGED, K)
            np.testing.assert_array_equal(pool.get_x(slots[q], p["n"]), alone[q])


@pytest.mark.parametrize("storage", ["bf16", "f32"])
def test_persistent_steps_match_oracle(storage):
    """Each round of a persistent launch is one iteration of the method:
    launches of one round each, every step against the oracle's step from
    the same x_k, element by element."""
    p = workloads.dense_system(2056, 257, seed=431)
    A_eff = oracle.quantize_bf16(p["A"]) if storage == "bf16" else p["A"]
    n2, _ = oracle.norms2(A_eff)
    rho = 1e-3
    with nsli.Pool(storage=storage) as pool:
        s = pool.add(p["A"], p["b0"], p["x0"], Av=p["Av"], stop="none", max_iter=100, rho=rho)
        for k in range(6):
            xk = pool.get_x(s, p["n"])
            pool.launch(max_rounds=1, max_seconds=30.0)
            assert pool.wait() == 1
            x1 = pool.get_x(s, p["n"])
            ref = parity.MapRef(A_eff, oracle.tick_b(p["b0"], p["Av"], rho, k), parity.to_accumulation(xk, storage),
                                storage, depth=2056 + 64, n2=n2, levels=parity.dot_levels(257))
            # the kernel's h is the one that makes its step equal lambda y / h
            dx = xk - x1
            j = int(np.argmax(np.abs(ref.y)))
            h_g = int(round(ref.y[j] / dx[j]))
            parity.check_dx(ref, xk, x1, h_g, 1.0, "relaxed", parity.TOL[storage])


def test_persistent_yield_and_wall_clock_ticks():
    """A launch with no round bound runs until yielded; with tick_s the
    device advances the ticks: a problem's b moves with wall-clock time, so
    the same launch with a long tick gives a different iterate."""
    import time
    p = workloads.dense_system(3000, 300, seed=432)
    xs = []
    for tick_s in (1e-4, 100.0):
        with nsli.Pool(storage="bf16") as pool:
            s = pool.add(p["A"], p["b0"], p["x0"], Av=p["Av"], stop="none", max_iter=1 << 40, rho=0.05)
            pool.set_ticks([s], [0])
            pool.launch(max_seconds=30.0, tick_s=tick_s)
            time.sleep(0.2)
            assert pool.stopped() == 0
            pool.yield_()
            rounds = pool.wait()
            assert rounds > 10
            xs.append(pool.get_x(s, p["n"]))
            with pytest.raises(nsli.NsliError):
                pool.launch(max_seconds=-1.0)
    assert not np.array_equal(xs[0], xs[1])


def test_persistent_pool_calls_refused_while_running():
    p = workloads.dense_system(500, 100, seed=433)
    with nsli.Pool(storage="f32") as pool:
        pool.add(p["A"], p["b0"], p["x0"], stop="none", max_iter=1 << 40)
        pool.launch(max_seconds=30.0)
        try:
            with pytest.raises(nsli.NsliError) as e:
                pool.add(p["A"], p["b0"], p["x0"], stop="none", max_iter=5)
            assert e.value.code == nsli.ERR_ARG
            with pytest.raises(nsli.NsliError):
                pool.step(1)
            with pytest.raises(nsli.NsliError):
                pool.launch(max_seconds=1.0)
        finally:
            pool.yield_()
            pool.wait()
        assert pool.live() == 1
