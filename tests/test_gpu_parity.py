"""CUDA path against the FP64 oracle, through the C ABI, on seeded inputs.

Floating point decides an integer in the Map (row violated or not).  Rows
whose oracle residual lies within a rigorous bound of the accumulation
type's rounding error are "ambiguous": either classification is correct,
so the checks accept both and bound their (tiny) contribution; everything
else is compared element by element.
"""
import numpy as np
import pytest

import oracle
import parity
from paper_2003_09956_gb300 import nsli, workloads

pytestmark = pytest.mark.gpu

STORAGES = ["f64", "f32", "bf16", "fp8"]


@pytest.fixture(scope="session", autouse=True)
def built_library():
    from paper_2003_09956_gb300 import _build
    _build.build()
    nsli.load()


def num_sms():
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def stored_values(A32, storage):
    """Exact values the stored matrix holds, from the oracle's quantizers."""
    if storage == "bf16":
        return oracle.quantize_bf16(A32)
    if storage == "fp8":
        q, _ = oracle.quantize_e4m3_rows(A32)
        return q
    return A32


def ambiguity_bound(A, x, b, u):
    """Rigorous bound on the accumulation type's error in r_i (64 levels)."""
    return parity.residual_bound(A, x, b, u, levels=64)


def check_map_reduce(solver, A_eff, b, x, storage):
    """One Map/Reduce through the C ABI against the oracle, element by
    element (tests/parity.py)."""
    y_g, h_g, st_g = solver.map_reduce()
    m, n = A_eff.shape
    ref = parity.check_map_reduce(y_g, h_g, st_g, A_eff, b, x, storage,
                                  depth=parity.dense_y_depth(m, num_sms()),
                                  levels=parity.dot_levels(n))
    return ref.mr, h_g


def step_and_check(solver, A_eff, b_k, storage, lam=1.0, rule="relaxed", rho=0.0, n2=None):
    """One iteration on the device from its own x_k, checked element by
    element against the oracle's step from the same point."""
    xk = solver.get_x()
    y_g, h_g, _ = solver.map_reduce()      # the Map the step takes (same x, same tick)
    solver.iterate(1, lam=lam, rule=rule, rho=rho)
    x1 = solver.get_x()
    m, n = A_eff.shape
    parity.check_step(xk, x1, h_g, A_eff, b_k, storage,
                      depth=parity.dense_y_depth(m, num_sms()), lam=lam, rule=rule, n2=n2,
                      levels=parity.dot_levels(n))
    if rule == "relaxed":                  # and the step is lambda y / h of that Map
        np.testing.assert_allclose(xk - x1, lam / max(h_g, 1) * y_g, rtol=1e-12,
                                   atol=1e-15 * (np.abs(xk).max() + 1))
    return xk, x1


# ------------------------------------------------------------------ Map/Reduce

SHAPES = [(1, 1), (7, 5), (300, 1), (150, 3), (1000, 333), (3001, 1000), (2000, 4100),
          (600, 8192), (333, 8200), (700, 12000), (400, 16384)]


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("m,n", SHAPES)
def test_map_reduce_one_step(storage, m, n):
    if storage == "f64" and n > 8192:
        pytest.skip("binary64 rows are limited to n <= 8192")
    p = workloads.dense_system(m, n, seed=1000 + m + n)
    A_eff = stored_values(p["A"], storage)
    src = p["A"].astype(np.float64) if storage == "f64" else p["A"]
    with nsli.Solver(src, p["b0"], p["x0"], Av=p["Av"], storage=storage) as s:
        if storage in ("bf16", "fp8"):
            np.testing.assert_array_equal(s.stored_rows(), A_eff.astype(np.float64))
        n2, _ = oracle.norms2(A_eff)
        np.testing.assert_allclose(s.norms2(), n2, rtol=1e-13)
        check_map_reduce(s, A_eff, p["b0"], p["x0"], storage)


@pytest.mark.parametrize("n", [3000, 12000])
@pytest.mark.parametrize("big", [40000.0, 2.0 ** 33])
def test_fp8_large_x_and_slice_coefficients(n, big):
    """FP8 storage with a few x entries far outside the typical range (40000
    and 2^33, at odd and even columns): residuals and slice coefficients of
    very different magnitudes in one Map.  Parity as everywhere."""
    m = 1500
    p = workloads.dense_system(m, n, seed=31 + n)
    x = p["x0"].copy()
    x[[1, 7, n // 2, n - 3]] = [big, -big, big, -big]
    A_eff = stored_values(p["A"], "fp8")
    with nsli.Solver(p["A"], p["b0"], x, Av=p["Av"], storage="fp8") as s:
        check_map_reduce(s, A_eff, p["b0"], x, "fp8")


@pytest.mark.parametrize("storage", STORAGES)
def test_map_reduce_after_tick_and_new_b(storage):
    m, n = 2500, 700
    p = workloads.dense_system(m, n, seed=77)
    A_eff = stored_values(p["A"], storage)
    src = p["A"].astype(np.float64) if storage == "f64" else p["A"]
    rng = np.random.default_rng(3)
    b_new = p["b0"] + rng.uniform(-5, 5, m)
    rho, tick = 0.25, 7
    with nsli.Solver(src, p["b0"], p["x0"], Av=p["Av"], storage=storage) as s:
        s.iterate(0, rho=rho)          # sets rho on the device
        s.update_b(b_new, tick=tick)
        b_k = oracle.tick_b(b_new, p["Av"], rho, tick)
        check_map_reduce(s, A_eff, b_k, p["x0"], storage)


# ------------------------------------------------------------------ trajectories

def oracle_trajectory(A_eff, p, rule, lam, rho, K):
    """x_0..x_K of the oracle and the residuals r(x_k, b(k)) of each Map."""
    n2, _ = oracle.norms2(A_eff)
    xs, rs = [p["x0"].copy()], []
    x = p["x0"].copy()
    for k in range(K):
        code, x, st, y, r = oracle.iteration(A_eff, p["b0"], p["Av"], rho, k, n2, x,
                                             lam=lam, rule=rule)
        xs.append(x.copy())
        rs.append(r)
    return xs, rs, n2


@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("rule", ["relaxed", "modap"])
@pytest.mark.parametrize("rho", [0.0, 1e-3])
def test_trajectory_matches_oracle(storage, rule, rho):
    """Every iteration's step, taken on the device from its own x_k, equals
    the oracle's step from that x_k element by element (tests/parity.py:
    1e-5 relative per element, 1e-12 for binary64 storage, plus the column's
    rounding bound), over 30 iterations.  The two independent trajectories
    also agree to the same tolerance relative to ||x|| until the first Map
    with an ambiguous row (one whose oracle residual is within the rounding
    bound plus ||a_i|| times the distance between the two iterates: from
    then on both classifications, hence both trajectories, are correct)."""
    m, n, K = 800, 257, 30
    p = workloads.dense_system(m, n, seed=5 + int(rho * 1e4))
    A_eff = stored_values(p["A"], storage)
    src = p["A"].astype(np.float64) if storage == "f64" else p["A"]
    lam = 1.0 if rule == "relaxed" else 0.5
    orule = oracle.RULE_RELAXED if rule == "relaxed" else oracle.RULE_MODAP
    tol = parity.TOL[storage]
    xs, rs, n2 = oracle_trajectory(A_eff, p, orule, lam, rho, K)
    compared = 0
    together = True
    with nsli.Solver(src, p["b0"], p["x0"], Av=p["Av"], storage=storage) as s:
        xg = s.get_x()
        for k in range(K):
            b_k = oracle.tick_b(p["b0"], p["Av"], rho, k)
            if together:
                drift = np.linalg.norm(xg - xs[k])
                bound = ambiguity_bound(A_eff, xs[k], b_k, parity.U[storage]) / 4 + \
                    np.sqrt(n2) * drift * 1.01
                together = not np.any(np.abs(rs[k]) <= bound)
            _, xg = step_and_check(s, A_eff, b_k, storage, lam=lam, rule=rule, rho=rho, n2=n2)
            if together:
                rel = np.linalg.norm(xg - xs[k + 1]) / np.linalg.norm(xs[k + 1])
                assert rel <= tol, (k, rel)
                compared += 1
        assert compared >= 3, "seeded case became ambiguous too early"
        assert s.result()["tick"] == K


def test_graph_blocks_equal_single_launches():
    """Iterations replayed from a captured graph equal direct launches, bit for bit."""
    p = workloads.dense_system(3000, 515, seed=9)
    with nsli.Solver(p["A"], p["b0"], p["x0"], Av=p["Av"]) as s1, \
            nsli.Solver(p["A"], p["b0"], p["x0"], Av=p["Av"]) as s2:
        s1.iterate(40, rho=1e-3, block_iters=8)   # 5 graph replays
        for _ in range(40):
            s2.iterate(1, rho=1e-3)               # direct launches
        np.testing.assert_array_equal(s1.get_x(), s2.get_x())
        assert s1.result()["tick"] == s2.result()["tick"] == 40


def test_deterministic_runs():
    p = workloads.dense_system(4000, 1000, seed=10)
    xs = []
    for _ in range(3):
        with nsli.Solver(p["A"], p["b0"], p["x0"], Av=p["Av"]) as s:
            s.iterate(25, rho=1e-4)
            xs.append(s.get_x())
    np.testing.assert_array_equal(xs[0], xs[1])
    np.testing.assert_array_equal(xs[0], xs[2])


def test_launch_count_two_kernels_per_iteration():
    p = workloads.dense_system(500, 100, seed=11)
    with nsli.Solver(p["A"], p["b0"], p["x0"]) as s:
        c0 = s.launch_count()
        s.iterate(64, block_iters=32)
        s.sync()
        assert s.launch_count() - c0 == 1 + 2 * 64   # state set-up + 2 per iteration


# ------------------------------------------------------------------ solves

@pytest.mark.parametrize("rule,lam", [("relaxed", 1.0), ("modap", 1.0)])
def test_model_system_solve_f64(rule, lam):
    """n = 256, m = 513 cube-with-cut-corner system, binary64, ||dx|| < 1e-8."""
    p = workloads.model_system(256, seed=0)
    orule = oracle.RULE_RELAXED if rule == "relaxed" else oracle.RULE_MODAP
    ref = oracle.solve(p["A"], p["b0"], p["x0"], rule=orule, lam=lam,
                       stop=oracle.STOP_STEP, eps=1e-8, max_iter=200000)
    with nsli.Solver(p["A"], p["b0"], p["x0"], storage="f64") as s:
        res = s.solve(lam=lam, rule=rule, stop="step", eps=1e-8, max_iter=200000)
        xg = s.get_x()
    assert res["status"] == ref["status"] == nsli.OK
    assert abs(res["iters"] - ref["iters"]) <= max(1, 0.01 * ref["iters"])
    maxb = np.abs(p["b0"]).max()
    assert res["max_viol"] <= 1e-6 * maxb
    assert np.max(p["A"] @ xg - p["b0"]) <= 1e-6 * maxb
    np.testing.assert_allclose(xg, ref["x"], rtol=0, atol=1e-6 * maxb)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_dense_solve_iteration_count_within_one_percent(storage):
    """A small stationary dense system solved to max r_i <= 1e-6 max|b|."""
    p = workloads.dense_system(256, 48, seed=21, grid=None if storage == "f32" else storage,
                               x0_std=1.0)
    A_eff = stored_values(p["A"], storage)
    ref = oracle.solve(A_eff, p["b0"], p["x0"], stop=oracle.STOP_MAXVIOL_REL, eps=1e-6,
                       max_iter=400000)
    assert ref["status"] == oracle.OK
    with nsli.Solver(p["A"], p["b0"], p["x0"], storage=storage) as s:
        res = s.solve(stop="maxviol_rel", eps=1e-6, max_iter=400000, block_iters=64)
    assert res["status"] == nsli.OK
    assert abs(res["iters"] - ref["iters"]) <= max(2, 0.01 * ref["iters"]), (res["iters"], ref["iters"])
    assert res["max_viol"] <= 1e-6 * res["max_abs_b"]


@pytest.mark.parametrize("m,n", [(2048, 256), (1024, 256)])
def test_mid_size_solves_match_oracle_in_binary32_and_bf16(m, n):
    """A stationary dense system drawn on the bf16 grid (so binary32 and
    bf16 storage hold the same values) solved from x0 ~ N(0, 25 I) to the
    binary64-confirmed stop max r_i <= 1e-6 max|b|: both storages end
    within 1 % of the oracle's iteration count (about 10^4 iterations),
    with the oracle's binary64 violation at the device's final iterate
    below the threshold."""
    p = workloads.dense_system(m, n, seed=5000 + n + m, grid="bf16")
    ref = oracle.solve(p["A"], p["b0"], p["x0"], stop=oracle.STOP_MAXVIOL_REL, eps=1e-6, max_iter=2000000)
    assert ref["status"] == oracle.OK
    n2, _ = oracle.norms2(p["A"])
    for storage in ("f32", "bf16"):
        with nsli.Solver(p["A"], p["b0"], p["x0"], storage=storage) as s:
            res = s.solve(stop="maxviol_rel", eps=1e-6, max_iter=2000000, block_iters=256)
            xg = s.get_x()
        assert res["status"] == nsli.OK
        assert abs(res["iters"] - ref["iters"]) <= max(2, 0.01 * ref["iters"]), (storage, res["iters"], ref["iters"])
        mr = oracle.map_reduce(p["A"], p["b0"], n2, xg)
        assert mr["maxviol"] <= 1e-6 * mr["maxb"], (storage, mr["maxviol"], mr["maxb"])
        assert res["max_viol"] == pytest.approx(mr["maxviol"], rel=1e-9, abs=1e-12 * mr["maxb"])


def test_strictly_feasible_start_gpu():
    p = workloads.dense_system(800, 64, seed=3)
    for storage in STORAGES:
        src = p["A"].astype(np.float64) if storage == "f64" else p["A"]
        A_eff = stored_values(p["A"], storage)
        z = p["z"].astype(np.float32).astype(np.float64)
        if np.max(A_eff.astype(np.float64) @ z - p["b0"]) >= -1e-3:
            continue
        with nsli.Solver(src, p["b0"], z, storage=storage) as s:
            res = s.solve(stop="step", eps=1e-8, max_iter=100)
            assert res["status"] == nsli.OK and res["iters"] == 0 and res["h"] == 0
            np.testing.assert_array_equal(s.get_x(), z)


def test_modap_step_length_gpu():
    p = workloads.dense_system(2000, 300, seed=4)
    with nsli.Solver(p["A"], p["b0"], p["x0"]) as s:
        for lam in (0.5, 2.0):
            x0 = s.get_x()
            s.iterate(1, lam=lam, rule="modap")
            x1 = s.get_x()
            assert np.linalg.norm(x1 - x0) == pytest.approx(lam, rel=1e-5)
            assert s.result()["last_step_norm"] == pytest.approx(lam, rel=1e-5)


def test_max_iter_and_not_converged():
    p = workloads.model_system(64, seed=2)
    with nsli.Solver(p["A"], p["b0"], p["x0"], storage="f64") as s:
        res = s.solve(stop="step", eps=1e-12, max_iter=5, block_iters=4)
        assert res["status"] == nsli.NOT_CONVERGED and res["iters"] == 5
        res = s.solve(stop="step", eps=1e-12, max_iter=0)
        assert res["status"] == nsli.NOT_CONVERGED and res["iters"] == 0


# ------------------------------------------------------------------ binary64 check

@pytest.mark.parametrize("storage", STORAGES)
def test_binary64_check_matches_oracle(storage):
    m, n = 3000, 900
    p = workloads.dense_system(m, n, seed=31)
    A_eff = stored_values(p["A"], storage)
    src = p["A"].astype(np.float64) if storage == "f64" else p["A"]
    rng = np.random.default_rng(6)
    x = rng.normal(0, 0.3, n).astype(np.float32).astype(np.float64)
    rho, tick = 1e-2, 11
    with nsli.Solver(src, p["b0"], p["x0"], Av=p["Av"], storage=storage) as s:
        s.set_x(x)
        s.iterate(0, rho=rho)
        s.update_b(None, tick=tick)
        mv, mn = s.residual_max()
    n2, _ = oracle.norms2(A_eff)
    mr = oracle.map_reduce(A_eff, oracle.tick_b(p["b0"], p["Av"], rho, tick), n2, x)
    assert mv == pytest.approx(mr["maxviol"], rel=1e-12, abs=1e-9)
    assert mn == pytest.approx(mr["maxnorm"], rel=1e-12, abs=1e-9)


# ------------------------------------------------------------------ errors

def test_error_codes():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((20, 8)).astype(np.float32)
    b = np.ones(20)
    x = np.zeros(8)
    bad = A.copy()
    bad[3] = 0.0
    with pytest.raises(nsli.NsliError) as e:
        nsli.Solver(bad, b, x)
    assert e.value.code == nsli.ERR_ZERO_ROW
    bad = A.copy()
    bad[2, 2] = np.nan
    for storage in ("f32", "bf16", "fp8"):
        with pytest.raises(nsli.NsliError) as e:
            nsli.Solver(bad, b, x, storage=storage)
        assert e.value.code == nsli.ERR_NONFINITE
    bb = b.copy()
    bb[0] = np.inf
    with pytest.raises(nsli.NsliError) as e:
        nsli.Solver(A, bb, x)
    assert e.value.code == nsli.ERR_NONFINITE
    xx = x.copy()
    xx[1] = np.nan
    with pytest.raises(nsli.NsliError) as e:
        nsli.Solver(A, b, xx)
    assert e.value.code == nsli.ERR_NONFINITE
    with pytest.raises(nsli.NsliError) as e:
        nsli.Solver(np.ones((2, 4), np.float64), np.ones(2), np.zeros(4), storage="bf16")
    assert e.value.code == nsli.ERR_ARG
    with nsli.Solver(A, b, x) as s:
        with pytest.raises(nsli.NsliError) as e:
            s.iterate(1, lam=-1.0)
        assert e.value.code == nsli.ERR_ARG
        with pytest.raises(nsli.NsliError) as e:
            s.update_b(np.full(20, np.nan))
        assert e.value.code == nsli.ERR_NONFINITE


# ------------------------------------------------------------------ full sizes

@pytest.fixture(scope="module")
def cfg2_system():
    return workloads.dense_system(32768, 8192, seed=2004)


@pytest.mark.parametrize("storage", ["f32", "bf16", "fp8"])
def test_full_size_32768x8192_one_step(cfg2_system, storage):
    p = cfg2_system
    A_eff = stored_values(p["A"], storage)
    with nsli.Solver(p["A"], p["b0"], p["x0"], Av=p["Av"], storage=storage) as s:
        s.iterate(0, rho=1e-4)
        check_map_reduce(s, A_eff, p["b0"], p["x0"], storage)


@pytest.fixture(scope="module")
def cfg3_system():
    return workloads.dense_system(131072, 16384, seed=2005)


def test_full_size_131072x16384_f32_one_step_and_fejer(cfg3_system):
    """The benchmark's workload and launch shape: one Map/Reduce against the
    oracle, then 6 stationary iterations whose distance to the interior point
    z must not grow (Fejer property, any size)."""
    p = cfg3_system
    with nsli.Solver(p["A"], p["b0"], p["x0"], Av=p["Av"], storage="f32") as s:
        check_map_reduce(s, p["A"], p["b0"], p["x0"], "f32")
        d_prev = np.linalg.norm(s.get_x() - p["z"])
        for _ in range(6):
            s.iterate(1, rho=0.0)
            d = np.linalg.norm(s.get_x() - p["z"])
            assert d <= d_prev * (1 + 1e-6)
            d_prev = d


@pytest.mark.parametrize("storage", ["bf16", "fp8"])
def test_full_size_131072x16384_quantized_one_step(cfg3_system, storage):
    """The bf16 and fp8 storage of the benchmark system: stored values and
    one Map/Reduce against the oracle on the oracle's own quantization."""
    p = cfg3_system
    A_eff = stored_values(p["A"], storage)
    with nsli.Solver(p["A"], p["b0"], p["x0"], Av=p["Av"], storage=storage) as s:
        rows = np.random.default_rng(5).integers(0, 131072, 64)
        for r in rows:
            np.testing.assert_array_equal(s.stored_rows(int(r), 1)[0], A_eff[r].astype(np.float64))
        s.iterate(0, rho=1e-4)
        check_map_reduce(s, A_eff, p["b0"], p["x0"], storage)


# ------------------------------------------------------------------ long rows

# four rows per group (the default L2 budget) for all but the last two (two
# and one rows); partial sums in shared memory except fp8 70000 and the
# binary32 rows of 60000 columns and more
LONG = [("f32", 600, 20000), ("bf16", 300, 40000), ("fp8", 200, 70000), ("f64", 200, 9000),
        ("f32", 153, 16388), ("f32", 400, 60000), ("bf16", 40, 40000), ("f32", 200, 54000),
        ("f32", 200, 70000), ("f32", 160, 140000)]


@pytest.mark.parametrize("budget_mb", ["8", "30", "512"])
@pytest.mark.parametrize("storage,m,n", [("f32", 600, 20000), ("bf16", 300, 40000)])
def test_long_rows_every_group_size(monkeypatch, budget_mb, storage, m, n):
    """The two-pass long-row kernel (clusters turned off): the L2 budget for
    the rows of a group (NSLI_LONG_L2_MB) picks one, two or four rows per
    group; all give the oracle's step, with the partial sums in shared
    memory."""
    monkeypatch.setenv("NSLI_LONG_CLUSTER", "0")
    monkeypatch.setenv("NSLI_LONG_L2_MB", budget_mb)
    test_long_rows_one_step_and_trajectory(storage, m, n)


@pytest.mark.parametrize("storage,m,n", [("f32", 200, 54000), ("bf16", 300, 40000), ("f64", 200, 9000),
                                         ("fp8", 200, 70000)])
def test_long_rows_two_pass_kernel(monkeypatch, storage, m, n):
    """The two-pass kernel (NSLI_LONG_CLUSTER=0) keeps the same parity bar."""
    monkeypatch.setenv("NSLI_LONG_CLUSTER", "0")
    test_long_rows_one_step_and_trajectory(storage, m, n)


@pytest.mark.parametrize("storage,m,n,size", [("bf16", 300, 40000, "4"), ("fp8", 200, 70000, "8"),
                                             ("f32", 400, 60000, "8"), ("f64", 200, 9000, "4")])
def test_long_rows_cluster_kernel_every_storage_and_size(monkeypatch, storage, m, n, size):
    """The cluster kernel at cluster sizes other than the default choice:
    same parity bar."""
    monkeypatch.setenv("NSLI_LONG_CLUSTER", "1")
    monkeypatch.setenv("NSLI_LONG_CLUSTER_SIZE", size)
    test_long_rows_one_step_and_trajectory(storage, m, n)


@pytest.mark.parametrize("storage,m,n,lag", [("bf16", 300, 40000, "1"), ("fp8", 200, 70000, "1"),
                                            ("bf16", 37, 54000, "2"), ("fp8", 150, 54000, "1"),
                                            ("fp8", 43, 54000, "2")])
def test_long_rows_cluster_one_and_two_rows_per_group_agree(monkeypatch, storage, m, n, lag):
    """bf16 rows take two rows per block barrier on clusters and FP8 rows
    four (the last group of a cluster's block may hold fewer); one row per
    barrier (NSLI_LONG_CLUSTER_RG=1) does the same arithmetic in the same
    order, so every group size gives the same bits, and the one-row form
    keeps the parity bar."""
    p = workloads.dense_system(m, n, seed=4100 + n)
    monkeypatch.setenv("NSLI_LONG_CLUSTER_LAG", lag)
    out = []
    for rg in (["4", "2", "1"] if storage == "fp8" else ["2", "1"]):
        monkeypatch.setenv("NSLI_LONG_CLUSTER_RG", rg)
        with nsli.Solver(p["A"], p["b0"], p["x0"], Av=p["Av"], storage=storage) as s:
            y, h, st = s.map_reduce()
            s.iterate(4, rho=1e-3)
            out.append((y, h, st, s.get_x()))
    for o in out[1:]:
        np.testing.assert_array_equal(out[0][0], o[0])
        assert out[0][1] == o[1] and out[0][2] == o[2]
        np.testing.assert_array_equal(out[0][3], o[3])
    test_long_rows_one_step_and_trajectory(storage, m, n)


def test_long_rows_cluster_kernel_equals_two_pass_kernel_and_is_deterministic(monkeypatch):
    """n = 54000 (the paper's size) on clusters of four CTAs: repeated runs
    give the same bits, and the iterate agrees with the two-pass kernel's to
    the parity tolerance after a few steps."""
    p = workloads.dense_system(400, 54000, seed=3999)
    xs = []
    for cluster in ("1", "1", "0"):
        monkeypatch.setenv("NSLI_LONG_CLUSTER", cluster)
        with nsli.Solver(p["A"], p["b0"], p["x0"], Av=p["Av"], storage="f32") as s:
            s.iterate(5, rho=1e-3)
            xs.append(s.get_x())
    np.testing.assert_array_equal(xs[0], xs[1])
    assert np.linalg.norm(xs[0] - xs[2]) <= 1e-5 * np.linalg.norm(xs[2] - p["x0"])


@pytest.mark.parametrize("storage,m,n", LONG)
def test_long_rows_one_step_and_trajectory(storage, m, n):
    """Rows beyond the register-resident limit take the chunked two-pass
    Map (violated rows re-read from L2); same parity bar, element by
    element, for one Map/Reduce and three steps."""
    p = workloads.dense_system(m, n, seed=3000 + n)
    A_eff = stored_values(p["A"], storage)
    src = p["A"].astype(np.float64) if storage == "f64" else p["A"]
    with nsli.Solver(src, p["b0"], p["x0"], Av=p["Av"], storage=storage) as s:
        check_map_reduce(s, A_eff, p["b0"], p["x0"], storage)
        n2, _ = oracle.norms2(A_eff)
        for k in range(3):
            step_and_check(s, A_eff, oracle.tick_b(p["b0"], p["Av"], 1e-3, k), storage, rho=1e-3, n2=n2)


# ------------------------------------------------------------------ step-size table

@pytest.mark.parametrize("kind", ["dense-f64", "dense-f32", "sparse-f64-grid"])
def test_step_size_changes_between_runs(monkeypatch, kind):
    """The relaxed step reads lambda / h from a table filled when a run
    begins with a new lambda: alternating lambda on one handle must give the
    oracle's step every time (one step from the device's own x_k; rows within
    rounding of zero would make the step ambiguous, and the seeds avoid them)."""
    monkeypatch.setenv("NSLI_SPARSE_RESIDENT", "0")
    if kind.startswith("dense"):
        storage = kind.split("-")[1]
        p = workloads.dense_system(700, 300, seed=61)
        A = p["A"].astype(np.float64) if storage == "f64" else stored_values(p["A"], storage)
        src = p["A"].astype(np.float64) if storage == "f64" else p["A"]
        make = lambda: nsli.Solver(src, p["b0"], p["x0"], Av=p["Av"], storage=storage)
    else:
        storage = "f64"
        p = workloads.sparse_system(700, 300, 8, seed=62)
        A = workloads.csr_to_dense(p["rp"], p["ci"], p["val"], p["n"])
        make = lambda: nsli.SparseSolver(p["m"], p["n"], p["rp"], p["ci"], p["val"], p["b0"], p["x0"],
                                         Av=p["Av"], storage="f64")
    n2, _ = oracle.norms2(A)
    with make() as s:
        for k, lam in enumerate([1.0, 0.5, 0.5, 1.7, 1.0]):
            xk = s.get_x()
            s.iterate(1, lam=lam, rule="relaxed", rho=0.0)
            x1 = s.get_x()
            depth = parity.dense_y_depth(700, num_sms()) if kind.startswith("dense") else 700
            parity.check_step(xk, x1, None, A, p["b0"], storage, depth=depth, lam=lam, n2=n2,
                              levels=parity.dot_levels(300))
