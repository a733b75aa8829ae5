"""Continuous batching (pool / server) through the C ABI.

The key property: a problem's iterates do not depend on which other
problems share the grouped launches, when they were admitted, or how many
are live (iteration-indexed ticks or rho = 0 make the result timing-free)."""
import numpy as np
import pytest

import oracle
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


def test_server_continuous_batching_to_feasibility():
    """Requests arrive while others run; each is admitted when memory frees
    up; every result equals the same request solved alone, and converged
    ones pass the binary64 check."""
    reqs_spec = []
    for q in range(8):
        n = [32, 48, 64, 40, 56, 72, 36, 60][q]
        p = workloads.dense_system(4 * n, n, seed=900 + q, x0_std=0.5)
        reqs_spec.append(p)
    params = dict(stop="maxviol_rel", eps=1e-6, max_iter=50000, rho=0.0)
    # alone
    alone = []
    for p in reqs_spec:
        srv = serve.Server(storage="f32", rounds_per_poll=16)
        r = srv.submit(serve.Request(0, p["A"], p["b0"], p["x0"], params=params))
        srv.drain(timeout_s=120)
        alone.append(r)
        srv.close()
    one = nsli.Pool(storage="f32")
    s = one.add(reqs_spec[0]["A"], reqs_spec[0]["b0"], reqs_spec[0]["x0"], stop="none", max_iter=1)
    budget = int(one.bytes_used() * 3.5)   # about three small problems at a time
    one.close()
    srv = serve.Server(storage="f32", max_bytes=budget, rounds_per_poll=16)
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
