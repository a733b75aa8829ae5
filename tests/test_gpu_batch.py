"""Batched form (many problems sharing one bf16 A, tcgen05 tensor cores)
against the FP64 oracle, problem by problem, through the C ABI."""
import numpy as np
import pytest

import oracle
import parity
from paper_2003_09956_gb300 import nsli, workloads

pytestmark = pytest.mark.gpu

# binary32 accumulation on the tensor cores, whose internal order and
# rounding of the partial sums are not specified: a rounding unit of 2^-23
# and at least 128 levels for the residuals (K = n), m / 16 + 64 for y
# (K = m in 16-deep MMA steps over two splits)
U32 = 2.0 ** -23


@pytest.fixture(scope="session", autouse=True)
def built_library():
    from paper_2003_09956_gb300 import _build
    _build.build()
    nsli.load()


def make_batch(m, n, P, seed, rho, x_std=5.0):
    p = workloads.dense_system(m, n, seed=seed)
    rng = np.random.default_rng(seed + 1)
    X0 = rng.normal(0.0, x_std, (P, n)).astype(np.float32).astype(np.float64)
    offs = np.arange(P, dtype=np.int64) * 3
    A_eff = oracle.quantize_bf16(p["A"])
    return p, X0, offs, A_eff


def problem_ref(A_eff, n2, b, x):
    m, n = A_eff.shape
    return parity.MapRef(A_eff, b, x, "f32", depth=m // 16 + 64, n2=n2, levels=max(128, n // 16 + 64), u=U32)


def check_problem(A_eff, n2, b, x, y_g, h_g, tol=1e-5):
    """One problem's y and h against the oracle, element by element."""
    ref = problem_ref(A_eff, n2, b, x)
    ref.check_h(h_g)
    ref.check_y(y_g, tol)


@pytest.mark.parametrize("m,n,P", [(1000, 500, 5), (777, 130, 16), (4096, 2048, 64), (300, 64, 1)])
def test_batch_map_reduce_matches_oracle(m, n, P):
    rho = 0.3
    p, X0, offs, A_eff = make_batch(m, n, P, seed=50 + m + P, rho=rho)
    n2, _ = oracle.norms2(A_eff)
    with nsli.BatchSolver(p["A"], p["b0"], X0, Av=p["Av"], tick_offsets=offs) as bs:
        Y, hv, mv = bs.map_reduce(rho=rho)
    for q in range(P):
        b = oracle.tick_b(p["b0"], p["Av"], rho, int(offs[q]))
        check_problem(A_eff, n2, b, X0[q], Y[q], int(hv[q]))


@pytest.mark.parametrize("rho", [0.0, 1e-3])
def test_batch_iterations_match_oracle(rho):
    """Every problem's step, from the batch's own x_k, against the oracle's
    step from that x_k element by element (K iterations); the independent
    trajectories also agree to 1e-5 relative until the first ambiguous row."""
    m, n, P, K = 800, 257, 6, 12
    p, X0, offs, A_eff = make_batch(m, n, P, seed=91, rho=rho)
    n2, _ = oracle.norms2(A_eff)
    with nsli.BatchSolver(p["A"], p["b0"], X0, Av=p["Av"], tick_offsets=offs) as bs:
        xs_g, hs_g = [X0.copy()], []
        for k in range(K):
            _, hv, _ = bs.map_reduce(rho=rho)     # the Map the next step takes
            hs_g.append(hv.copy())
            bs.iterate(1, rho=rho)
            xs_g.append(bs.get_x())
    for q in range(P):
        x = X0[q].copy()
        together = True
        for k in range(K):
            tick = int(offs[q]) + k
            b_k = oracle.tick_b(p["b0"], p["Av"], rho, tick)
            ref = problem_ref(A_eff, n2, b_k, xs_g[k][q])
            h_g = int(hs_g[k][q])
            ref.check_h(h_g)
            dx_ref, dB = ref.step(h_g, 1.0, "relaxed")
            dx_g = xs_g[k][q] - xs_g[k + 1][q]
            lim = 1e-5 * np.abs(dx_ref) + dB + 1e-15 * np.abs(xs_g[k][q])
            assert np.all(np.abs(dx_g - dx_ref) <= lim), (q, k)
            if together:
                drift = np.linalg.norm(xs_g[k][q] - x)
                mr = oracle.map_reduce(A_eff, b_k, n2, x)
                if np.any(np.abs(mr["r"]) <= parity.residual_bound(A_eff, x, b_k, U32, 128) / 2 +
                          np.sqrt(n2) * drift * 1.01):
                    together = False  # an ambiguous row: both continuations are correct
                else:
                    _, x, _, _, _ = oracle.iteration(A_eff, p["b0"], p["Av"], rho, tick, n2, x)
                    rel = np.linalg.norm(xs_g[k + 1][q] - x) / np.linalg.norm(x)
                    assert rel <= 1e-5, (q, k, rel)


def test_batch_equals_single_problem_solver():
    m, n, P, K = 2048, 512, 4, 6
    rho = 1e-3
    p, X0, offs, A_eff = make_batch(m, n, P, seed=17, rho=rho)
    with nsli.BatchSolver(p["A"], p["b0"], X0, Av=p["Av"], tick_offsets=offs) as bs:
        bs.iterate(K, rho=rho, block_iters=3)
        Xb = bs.get_x()
    for q in range(P):
        with nsli.Solver(p["A"], p["b0"], X0[q], Av=p["Av"], storage="bf16") as s:
            s.update_b(None, tick=int(offs[q]))
            s.iterate(K, rho=rho)
            xq = s.get_x()
        assert np.linalg.norm(Xb[q] - xq) <= 1e-5 * np.linalg.norm(xq)


def test_batch_binary64_check():
    m, n, P = 1500, 300, 3
    rho = 0.05
    p, X0, offs, A_eff = make_batch(m, n, P, seed=23, rho=rho)
    n2, _ = oracle.norms2(A_eff)
    with nsli.BatchSolver(p["A"], p["b0"], X0, Av=p["Av"], tick_offsets=offs) as bs:
        bs.iterate(0, rho=rho)
        mv = bs.residual_max()
    for q in range(P):
        b = oracle.tick_b(p["b0"], p["Av"], rho, int(offs[q]))
        ref = oracle.map_reduce(A_eff, b, n2, X0[q])["maxviol"]
        assert mv[q] == pytest.approx(ref, rel=1e-12, abs=1e-9)


def test_batch_full_size_65536x8192x64_sampled():
    """The batched benchmark shape: one Map/Reduce for all 64 problems,
    three of them checked against the oracle."""
    m, n, P = 65536, 8192, 64
    rho = 1e-4
    p = workloads.dense_system(m, n, seed=2007)
    rng = np.random.default_rng(2008)
    X0 = rng.normal(0.0, 5.0, (P, n)).astype(np.float32).astype(np.float64)
    offs = np.arange(P, dtype=np.int64)
    A_eff = oracle.quantize_bf16(p["A"])
    n2, _ = oracle.norms2(A_eff)
    with nsli.BatchSolver(p["A"], p["b0"], X0, Av=p["Av"], tick_offsets=offs) as bs:
        Y, hv, mv = bs.map_reduce(rho=rho)
    for q in (0, 31, 63):
        b = oracle.tick_b(p["b0"], p["Av"], rho, int(offs[q]))
        check_problem(A_eff, n2, b, X0[q], Y[q], int(hv[q]))
