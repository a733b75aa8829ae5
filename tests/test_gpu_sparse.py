"""Sparse A (compressed rows + compressed columns on the device) against the
FP64 oracle, through the C ABI, on seeded inputs.

The compressed-row oracle is pinned bit for bit to the dense oracle
(test_oracle_pins.py).  As for the dense path, rows whose oracle residual
lies within a rigorous rounding bound of 0 may be classified either way; the
bound here uses each row's own length: a sum of L products in any order has
error <= gamma_L (sum |a_ij x_j|), plus the rounding of x, b0 and the tick
term into the accumulation type.
"""
import numpy as np
import pytest

import oracle
import parity
from paper_2003_09956_gb300 import nsli, workloads

pytestmark = pytest.mark.gpu

U = {"f64": 2.0 ** -53, "f32": 2.0 ** -24}


@pytest.fixture(scope="session", autouse=True)
def built_library():
    from paper_2003_09956_gb300 import _build
    _build.build()
    nsli.load()


def solver(p, storage, x0=None):
    return nsli.SparseSolver(p["m"], p["n"], p["rp"], p["ci"], p["val"], p["b0"],
                             p["x0"] if x0 is None else x0, Av=p["Av"], storage=storage)


def row_bounds(p, x, b0, shift, u):
    """Rounding bound of each computed residual (4x slack)."""
    rp, ci, val = p["rp"], p["ci"], p["val"]
    L = np.diff(rp).astype(np.float64)
    absdot = np.add.reduceat(np.abs(val) * np.abs(x[ci]), rp[:-1])
    return 4.0 * (L + 16.0) * u * (absdot + np.abs(b0) + np.abs(shift) + 1e-300)


def check_one_step(s, p, storage, b0, shift, x, tol_rel=None):
    """y, h and maxima of one Map/Reduce against the oracle, element by
    element (tests/parity.py)."""
    y_g, h_g, st_g = s.map_reduce()
    n2, zero = oracle.norms2_csr(p["rp"], p["val"])
    assert zero == 0
    xa = parity.to_accumulation(x, storage)
    ref = parity.CsrMapRef(p["rp"], p["ci"], p["val"], p["n"], b0 + shift, xa, storage, n2=n2,
                           b_parts=(b0, shift))
    ref.check_h(h_g)
    ref.check_y(y_g, parity.TOL[storage] if tol_rel is None else tol_rel)
    ref.check_maxima(st_g["maxviol"], st_g["maxb"])
    return ref.mr, h_g


def check_sparse_step(s, p, storage, b_k, lam, rule, rho, n2, b_parts=None):
    """One iteration from the device's own x_k against the oracle's step
    from that x_k, element by element."""
    xk = s.get_x()
    s.iterate(1, lam=lam, rule=rule, rho=rho)
    x1 = s.get_x()
    ref = parity.CsrMapRef(p["rp"], p["ci"], p["val"], p["n"], b_k, parity.to_accumulation(xk, storage),
                           storage, n2=n2, b_parts=b_parts)
    parity.check_dx(ref, xk, x1, None, lam, rule, parity.TOL[storage])
    return x1


def case(name):
    """Seeded sparse systems covering every launch shape of the kernels."""
    g = np.random.default_rng(sum(map(ord, name)))
    if name == "one-by-one":
        return workloads.sparse_system(1, 1, 1, seed=1)
    if name == "ragged":            # mean 20 per row: 16 lanes per row
        return workloads.sparse_system(3000, 500, 0, seed=2, lengths=g.integers(1, 40, 3000))
    if name == "short-rows":        # 3 per row, 2 lanes per row, 1 per column
        return workloads.sparse_system(5000, 2000, 3, seed=3)
    if name == "heavy-rows":        # every 50th row cut into two pieces
        L = np.full(400, 5)
        L[::50] = 2500
        return workloads.sparse_system(400, 3000, 0, seed=4, lengths=L)
    if name == "heavy-cols":        # columns 0, 1 in every one of 5000 rows (3 pieces each)
        return workloads.sparse_system(5000, 1500, 0, seed=5, lengths=g.integers(3, 12, 5000),
                                       dense_cols=2)
    if name == "few-long-rows":     # m far below the SM count, long light rows
        return workloads.sparse_system(20, 50000, 2000, seed=6)
    if name == "wide":              # many columns, k = 32
        return workloads.sparse_system(40000, 100000, 32, seed=7)
    raise KeyError(name)


CASES = ["one-by-one", "ragged", "short-rows", "heavy-rows", "heavy-cols", "few-long-rows", "wide"]


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("name", CASES)
def test_sparse_map_reduce_one_step(storage, name):
    p = case(name)
    with solver(p, storage) as s:
        n2, _ = oracle.norms2_csr(p["rp"], p["val"])
        np.testing.assert_allclose(s.norms2(), n2, rtol=1e-13)
        check_one_step(s, p, storage, p["b0"], np.zeros(p["m"]), p["x0"])


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_sparse_map_reduce_after_tick_and_new_b(storage):
    p = case("ragged")
    rng = np.random.default_rng(3)
    b_new = p["b0"] + rng.uniform(-5, 5, p["m"])
    rho, tick = 0.25, 7
    with solver(p, storage) as s:
        s.iterate(0, rho=rho)
        s.update_b(b_new, tick=tick)
        b_k = oracle.tick_b(b_new, p["Av"], rho, tick)
        check_one_step(s, p, storage, b_new, b_k - b_new, p["x0"])


def test_sparse_stored_rows_and_model_system():
    p = workloads.model_system_csr(300, seed=1)
    A = workloads.csr_to_dense(p["rp"], p["ci"], p["val"], p["n"])
    with solver(p, "f64") as s:
        np.testing.assert_array_equal(s.stored_rows(), A)
        np.testing.assert_array_equal(s.stored_rows(598, 3), A[598:601])
        check_one_step(s, p, "f64", p["b0"], np.zeros(p["m"]), p["x0"])


@pytest.mark.parametrize("path", ["one-cta", "grid"])
@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("rule", ["relaxed", "modap"])
@pytest.mark.parametrize("rho", [0.0, 1e-3])
def test_sparse_trajectory_matches_oracle(monkeypatch, path, storage, rule, rho):
    """Every step, taken on the device from its own x_k, equals the oracle's
    step from that x_k element by element (30 iterations, one per call, so
    the one-CTA path also carries its state across launches); the two
    independent trajectories agree to 1e-5 relative (1e-12 for binary64)
    until the first Map with an ambiguous row (dense oracle on the
    densified matrix)."""
    monkeypatch.setenv("NSLI_SPARSE_RESIDENT", "1" if path == "one-cta" else "0")
    p = workloads.sparse_system(1500, 400, 12, seed=31 + int(rho * 1e4))
    A = workloads.csr_to_dense(p["rp"], p["ci"], p["val"], p["n"])
    n2, _ = oracle.norms2(A)
    n2c, _ = oracle.norms2_csr(p["rp"], p["val"])
    lam = 1.0 if rule == "relaxed" else 0.5
    orule = oracle.RULE_RELAXED if rule == "relaxed" else oracle.RULE_MODAP
    tol = parity.TOL[storage]
    K = 30
    x = p["x0"].copy()
    compared = 0
    together = True
    with solver(p, storage) as s:
        xg = s.get_x()
        for k in range(K):
            b0k = p["b0"]
            shift = oracle.tick_b(p["b0"], p["Av"], rho, k) - b0k
            if together:
                drift = np.linalg.norm(xg - x)
                code, x_next, st, y, r = oracle.iteration(A, p["b0"], p["Av"], rho, k, n2, x, lam=lam,
                                                          rule=orule)
                bound = row_bounds(p, x, b0k, shift, U[storage]) / 4 + np.sqrt(n2) * drift * 1.01
                together = not np.any(np.abs(r) <= bound)
            xg = check_sparse_step(s, p, storage, b0k + shift, lam, rule, rho, n2c, b_parts=(b0k, shift))
            if together:
                x = x_next
                rel = np.linalg.norm(xg - x) / np.linalg.norm(x)
                assert rel <= tol, (k, rel)
                compared += 1
        assert compared >= 3, "seeded case became ambiguous too early"
        assert s.result()["tick"] == K


@pytest.mark.parametrize("path", ["one-cta", "grid"])
@pytest.mark.parametrize("rule,lam", [("relaxed", 1.0), ("modap", 1.0)])
def test_sparse_model_system_solve_matches_dense(monkeypatch, path, rule, lam):
    """Model system n = 256 in compressed form: the same solve as the dense
    oracle (binary64, ||dx|| < 1e-8), iteration count within 1%, both on
    one CTA (where this small system runs by default) and on the grid
    kernels."""
    monkeypatch.setenv("NSLI_SPARSE_RESIDENT", "1" if path == "one-cta" else "0")
    p = workloads.model_system_csr(256, seed=0)
    A = workloads.csr_to_dense(p["rp"], p["ci"], p["val"], p["n"])
    orule = oracle.RULE_RELAXED if rule == "relaxed" else oracle.RULE_MODAP
    ref = oracle.solve(A, p["b0"], p["x0"], rule=orule, lam=lam, stop=oracle.STOP_STEP, eps=1e-8,
                       max_iter=200000)
    with solver(p, "f64") as s:
        res = s.solve(lam=lam, rule=rule, stop="step", eps=1e-8, max_iter=200000, block_iters=64)
        xg = s.get_x()
    assert res["status"] == ref["status"] == nsli.OK
    assert abs(res["iters"] - ref["iters"]) <= max(1, 0.01 * ref["iters"])
    maxb = np.abs(p["b0"]).max()
    assert res["max_viol"] <= 1e-6 * maxb
    np.testing.assert_allclose(xg, ref["x"], rtol=0, atol=1e-6 * maxb)


@pytest.mark.parametrize("path", ["one-cta", "grid"])
@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_sparse_solve_to_feasibility(monkeypatch, path, storage):
    monkeypatch.setenv("NSLI_SPARSE_RESIDENT", "1" if path == "one-cta" else "0")
    p = workloads.sparse_system(600, 150, 6, seed=41, x0_std=1.0)
    A = workloads.csr_to_dense(p["rp"], p["ci"], p["val"], p["n"])
    ref = oracle.solve(A, p["b0"], p["x0"], stop=oracle.STOP_MAXVIOL_REL, eps=1e-6, max_iter=400000)
    assert ref["status"] == oracle.OK
    with solver(p, storage) as s:
        res = s.solve(stop="maxviol_rel", eps=1e-6, max_iter=400000, block_iters=64)
    assert res["status"] == nsli.OK
    assert abs(res["iters"] - ref["iters"]) <= max(2, 0.01 * ref["iters"]), (res["iters"], ref["iters"])
    assert res["max_viol"] <= 1e-6 * res["max_abs_b"]


def test_sparse_graph_blocks_equal_single_launches_and_determinism(monkeypatch):
    monkeypatch.setenv("NSLI_SPARSE_RESIDENT", "0")
    p = case("ragged")
    xs = []
    for block in (8, 1, 8):
        with solver(p, "f32") as s:
            if block == 1:
                for _ in range(40):
                    s.iterate(1, rho=1e-3, rule="modap", lam=0.5)
            else:
                s.iterate(40, rho=1e-3, rule="modap", lam=0.5, block_iters=block)
            xs.append(s.get_x())
            assert s.result()["tick"] == 40
    np.testing.assert_array_equal(xs[0], xs[1])
    np.testing.assert_array_equal(xs[0], xs[2])


def test_sparse_launch_count(monkeypatch):
    monkeypatch.setenv("NSLI_SPARSE_RESIDENT", "0")
    p = case("short-rows")
    with solver(p, "f32") as s:
        c0 = s.launch_count()
        s.iterate(64, block_iters=32)
        s.sync()
        assert s.launch_count() - c0 == 1 + 2 * 64
        c1 = s.launch_count()
        s.iterate(64, block_iters=32, rule="modap")
        s.sync()
        assert s.launch_count() - c1 == 1 + 3 * 64


def test_sparse_binary64_check():
    p = case("heavy-cols")
    rho, tick = 0.05, 3
    with solver(p, "f32") as s:
        s.iterate(0, rho=rho)
        s.update_b(None, tick=tick)
        mv, mn = s.residual_max()
    n2, _ = oracle.norms2_csr(p["rp"], p["val"])
    b = oracle.tick_b(p["b0"], p["Av"], rho, tick)
    x32 = p["x0"]
    ref = oracle.map_reduce_csr(p["rp"], p["ci"], p["val"], p["n"], b, n2, x32)
    assert mv == pytest.approx(ref["maxviol"], rel=1e-12, abs=1e-9)
    assert mn == pytest.approx(ref["maxnorm"], rel=1e-12, abs=1e-9)


def test_sparse_error_codes():
    p = workloads.sparse_system(10, 8, 3, seed=9)
    m, n = 10, 8

    def make(rp, ci, val, storage="f32"):
        return nsli.SparseSolver(m, n, rp, ci, val, p["b0"], p["x0"], storage=storage)

    def code(*a, **k):
        with pytest.raises(nsli.NsliError) as e:
            make(*a, **k)
        return e.value.code

    rp, ci, val = p["rp"].copy(), p["ci"].copy(), p["val"].copy()
    bad = ci.copy()
    bad[1], bad[2] = bad[2], bad[1]                       # not ascending within row 0
    assert code(rp, bad, val) == nsli.ERR_ARG
    bad = ci.copy()
    bad[4] = n                                           # out of range
    assert code(rp, bad, val) == nsli.ERR_ARG
    bad_rp = rp.copy()
    bad_rp[-1] += 1                                      # does not end at nnz
    with pytest.raises((nsli.NsliError, ValueError)):
        make(bad_rp, ci, val)
    v = val.copy()
    v[3:6] = 0.0                                          # row 1 all zero
    assert code(rp, ci, v) == nsli.ERR_ZERO_ROW
    v = val.copy()
    v[7] = np.nan
    assert code(rp, ci, v) == nsli.ERR_NONFINITE
    assert code(rp, ci, val, storage="bf16") == nsli.ERR_UNSUPPORTED
    with make(rp, ci, val) as s:
        assert s.inject_timeout() == nsli.ERR_UNSUPPORTED


def test_sparse_full_size_one_step_sampled():
    """The sparse benchmark shape (4194304 x 1048576, 32 per row, binary32):
    one Map/Reduce against the compressed-row oracle over all rows."""
    p = workloads.sparse_system(1 << 22, 1 << 20, 32, seed=2011)
    with solver(p, "f32") as s:
        check_one_step(s, p, "f32", p["b0"], np.zeros(p["m"]), p["x0"])
