"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these checks re-types the oracle's formulas: each compares it with a
hand-worked example, an exact rational recurrence, a geometric property
(projection onto a hyperplane, Fejer monotonicity, fixed length of the ModAP
step), brute-force vertex enumeration, an invariance, or a library routine.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2003_09956_gb300 import workloads
from conftest import load_golden


# ---------------------------------------------------------------- worked examples

def test_hand_worked_2d_relaxed_and_modap():
    """Eq. 7, Eq. 8 and Eq. 12 on the hand-worked 2-D fixture."""
    g = load_golden("hand_worked_2d.txt")
    A = np.array([[1.0, 0.0], [0.0, 1.0], [-1.0, -1.0]])
    b = np.array([1.0, 1.0, 10.0])
    n2, zero = oracle.norms2(A)
    assert zero == 0
    mr = oracle.map_reduce(A, b, n2, g["case1.x0"])
    np.testing.assert_allclose(mr["y"], g["case1.y"], rtol=0, atol=1e-15)
    assert mr["h"] == int(g["case1.h"][0])
    assert mr["maxviol"] == pytest.approx(g["case1.maxviol"][0], abs=1e-15)
    assert mr["maxnorm"] == pytest.approx(g["case1.maxnorm"][0], abs=1e-15)
    code, x1, st, _, _ = oracle.iteration(A, b, None, 0.0, 0, n2, g["case1.x0"],
                                          lam=1.0, rule=oracle.RULE_RELAXED)
    assert code == oracle.IT_STEPPED
    np.testing.assert_allclose(x1, g["case1.relaxed_x1"], rtol=0, atol=1e-15)
    code, x1, st, _, _ = oracle.iteration(A, b, None, 0.0, 0, n2, g["case1.x0"],
                                          lam=1.0, rule=oracle.RULE_MODAP)
    np.testing.assert_allclose(x1, g["case1.modap_x1"], rtol=0, atol=1e-15)


def test_hand_worked_single_row_projection():
    g = load_golden("hand_worked_2d.txt")
    A = np.array([[3.0, 4.0]])
    b = np.array([5.0])
    n2, _ = oracle.norms2(A)
    mr = oracle.map_reduce(A, b, n2, g["case2.x0"])
    np.testing.assert_allclose(mr["y"], g["case2.y"], rtol=1e-15)
    assert mr["h"] == 1
    assert mr["maxnorm"] == pytest.approx(g["case2.maxnorm"][0], rel=1e-15)
    _, x1, _, _, _ = oracle.iteration(A, b, None, 0.0, 0, n2, g["case2.x0"])
    np.testing.assert_allclose(x1, g["case2.relaxed_x1"], rtol=1e-15)


# ---------------------------------------------------------------- geometry

@pytest.mark.parametrize("seed", range(5))
def test_single_violated_row_is_orthogonal_projection(seed):
    """With one violated row and lambda = 1 the step is the orthogonal
    projection onto its hyperplane (Section 2): the new point satisfies the
    row with equality and moved along the row's normal."""
    rng = np.random.default_rng(100 + seed)
    n = 7
    a = rng.standard_normal(n)
    x0 = rng.standard_normal(n)
    b_violated = float(a @ x0) - 2.5          # r = 2.5 > 0
    # a second, satisfied row (r < 0)
    a2 = rng.standard_normal(n)
    b2 = float(a2 @ x0) + 10.0
    A = np.stack([a, a2])
    b = np.array([b_violated, b2])
    n2, _ = oracle.norms2(A)
    code, x1, st, y, r = oracle.iteration(A, b, None, 0.0, 0, n2, x0)
    assert st["h"] == 1
    assert abs(float(a @ x1) - b_violated) < 1e-12 * (1 + abs(b_violated))
    d = x0 - x1
    cosang = abs(d @ a) / (np.linalg.norm(d) * np.linalg.norm(a))
    assert cosang == pytest.approx(1.0, abs=1e-14)
    # distance moved equals the distance to the hyperplane
    assert np.linalg.norm(d) == pytest.approx(2.5 / np.linalg.norm(a), rel=1e-13)


@pytest.mark.parametrize("lam", [0.5, 1.0, 1.5, 1.9])
def test_fejer_monotone_relaxed(lam):
    """x - phi(x) is M-Fejer for fixed t (Section 2): the distance to every
    feasible point never grows (lambda in (0, 2))."""
    p = workloads.small_polytope(n=6, m=30, seed=7)
    A, b = p["A"], p["b0"]
    n2, _ = oracle.norms2(A)
    zs = [p["z"]]
    rng = np.random.default_rng(3)
    # a few more feasible points: z moved a little inside
    for _ in range(3):
        cand = p["z"] + rng.uniform(-0.01, 0.01, p["n"])
        if np.all(A @ cand <= b):
            zs.append(cand)
    x = p["x0"].copy()
    for k in range(300):
        code, xn, st, _, _ = oracle.iteration(A, b, None, 0.0, k, n2, x, lam=lam)
        for z in zs:
            assert np.linalg.norm(xn - z) <= np.linalg.norm(x - z) * (1 + 1e-14)
        x = xn


def test_y_points_away_from_feasible_points():
    """<y, x - z> > 0 for feasible z whenever h > 0, because a_i.(x - z) > r_i > 0
    on every violated row."""
    p = workloads.small_polytope(n=5, m=25, seed=11)
    A, b, z = p["A"], p["b0"], p["z"]
    n2, _ = oracle.norms2(A)
    rng = np.random.default_rng(5)
    for _ in range(50):
        x = z + rng.normal(0, 4, p["n"])
        mr = oracle.map_reduce(A, b, n2, x)
        if mr["h"] > 0:
            assert mr["y"] @ (x - z) > 0


@pytest.mark.parametrize("lam", [0.25, 1.0, 3.0])
def test_modap_step_has_length_lambda(lam):
    """psi(x) = lambda phi / ||phi|| has length lambda (Eq. 12)."""
    p = workloads.small_polytope(n=8, m=40, seed=2)
    A, b = p["A"], p["b0"]
    n2, _ = oracle.norms2(A)
    x = p["x0"].copy()
    for k in range(20):
        code, xn, st, _, _ = oracle.iteration(A, b, None, 0.0, k, n2, x, lam=lam,
                                              rule=oracle.RULE_MODAP)
        if st["h"] == 0:
            break
        assert np.linalg.norm(xn - x) == pytest.approx(lam, rel=1e-13)
        assert st["dx_norm"] == pytest.approx(lam, rel=1e-13)
        x = xn


def test_strictly_feasible_start_is_a_fixed_point():
    p = workloads.small_polytope(n=4, m=20, seed=4)
    for rule in (oracle.RULE_RELAXED, oracle.RULE_MODAP):
        for stop in (oracle.STOP_STEP, oracle.STOP_EPSMEM, oracle.STOP_MAXVIOL_REL):
            res = oracle.solve(p["A"], p["b0"], p["z"], rule=rule, stop=stop,
                               eps=1e-9, max_iter=10)
            assert res["status"] == oracle.OK
            assert res["iters"] == 0
            assert res["h"] == 0
            np.testing.assert_array_equal(res["x"], p["z"])


# ---------------------------------------------------------------- exact recurrence

def test_model_system_exact_rational_recurrence():
    """Cube-with-cut-corner system, Algorithm 1 with lambda = 1.

    While exactly the n upper bounds and the sum row are violated, the slices
    are e_j * unit_j (r_j = e_j = x_j - 200, ||a||^2 = 1) and (s/n) * 1 with
    s = sum_j e_j + 100 (||a||^2 = n), h = n + 1, so
    e <- e - (e + (s/n) 1) / (n + 1).  Iterated exactly in rationals."""
    n = 12
    p = workloads.model_system(n, seed=0)
    x0 = np.array([390.0, 395.0, 399.0, 392.0, 397.0, 391.0, 398.0, 393.0,
                   396.0, 394.0, 399.0, 390.0])
    e = [Fraction(int(v)) - 200 for v in x0]
    n2, _ = oracle.norms2(p["A"])
    x = x0.copy()
    steps = 0
    for k in range(60):
        if not all(ej > 0 for ej in e):
            break
        s = sum(e) + 100
        if s <= 0:
            break
        e = [ej - (ej + s / n) / (n + 1) for ej in e]
        code, x, st, _, _ = oracle.iteration(p["A"], p["b0"], None, 0.0, k, n2, x)
        assert st["h"] == n + 1
        exact = np.array([float(ej + 200) for ej in e])
        np.testing.assert_allclose(x, exact, rtol=1e-13, atol=0)
        steps += 1
    assert steps >= 10


# ---------------------------------------------------------------- brute force

def _vertices(A, b):
    m, n = A.shape
    verts = []
    for rows in itertools.combinations(range(m), n):
        S = A[list(rows)]
        if abs(np.linalg.det(S)) < 1e-12:
            continue
        v = np.linalg.solve(S, b[list(rows)])
        if np.all(A @ v <= b + 1e-9):
            verts.append(v)
    return np.array(verts)


@pytest.mark.parametrize("n,m,seed", [(2, 10, 0), (2, 14, 1), (3, 12, 2), (3, 16, 3)])
@pytest.mark.parametrize("rule", [oracle.RULE_RELAXED, oracle.RULE_MODAP])
def test_brute_force_vertex_enumeration(n, m, seed, rule):
    """Vertex enumeration certifies M is non-empty and gives an interior point
    (the vertex centroid); the oracle then reaches eps-membership (Eq. 10)
    and the final point satisfies every row to within eps * ||a_i||."""
    p = workloads.small_polytope(n=n, m=m, seed=seed)
    A, b = p["A"], p["b0"]
    V = _vertices(A, b)
    assert len(V) >= n + 1
    c = V.mean(axis=0)
    assert np.all(A @ c <= b + 1e-9)
    eps = 1e-7
    lam = 1.0 if rule == oracle.RULE_RELAXED else 1e-3
    res = oracle.solve(A, b, p["x0"], rule=rule, stop=oracle.STOP_EPSMEM,
                       eps=eps, max_iter=2_000_000, lam=lam)
    assert res["status"] == oracle.OK
    viol = (A @ res["x"] - b) / np.linalg.norm(A, axis=1)
    assert viol.max() < eps
    # Fejer: the final point is not farther from the centroid than the start
    if rule == oracle.RULE_RELAXED:
        assert np.linalg.norm(res["x"] - c) <= np.linalg.norm(p["x0"] - c)


# ---------------------------------------------------------------- invariances

def test_row_scaling_and_permutation_invariance():
    p = workloads.small_polytope(n=6, m=30, seed=9)
    A, b = p["A"], p["b0"]
    rng = np.random.default_rng(1)
    scale = rng.uniform(0.1, 10.0, A.shape[0])
    perm = rng.permutation(A.shape[0])
    A2 = (A * scale[:, None])[perm]
    b2 = (b * scale)[perm]
    r1 = oracle.solve(A, b, p["x0"], stop=oracle.STOP_NONE, max_iter=50)
    r2 = oracle.solve(A2, b2, p["x0"], stop=oracle.STOP_NONE, max_iter=50)
    np.testing.assert_allclose(r1["x"], r2["x"], rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("rule", [oracle.RULE_RELAXED, oracle.RULE_MODAP])
def test_tick_is_a_translation(rule):
    """b(k) = b0 + k rho A v translates M by k rho v (Section 5): one iteration
    at tick k from x equals one stationary iteration from x - k rho v,
    shifted back by k rho v."""
    p = workloads.small_polytope(n=6, m=30, seed=12)
    A, b0 = p["A"], p["b0"]
    rng = np.random.default_rng(8)
    v = rng.standard_normal(p["n"])
    v /= np.linalg.norm(v)
    Av = A @ v
    n2, _ = oracle.norms2(A)
    rho, k = 0.37, 5
    x = p["x0"]
    _, x_moving, st1, _, _ = oracle.iteration(A, b0, Av, rho, k, n2, x, rule=rule)
    shift = k * rho * v
    _, x_static, st2, _, _ = oracle.iteration(A, b0, None, 0.0, 0, n2, x - shift, rule=rule)
    assert st1["h"] == st2["h"]
    np.testing.assert_allclose(x_moving, x_static + shift, rtol=1e-12, atol=1e-12)


def test_translation_equivariance_of_the_trajectory():
    """Shifting the system by A d and the start by d shifts every iterate by d."""
    p = workloads.small_polytope(n=5, m=20, seed=13)
    A, b = p["A"], p["b0"]
    d = np.array([0.5, -1.0, 2.0, 0.25, -0.75])
    r1 = oracle.solve(A, b, p["x0"], stop=oracle.STOP_NONE, max_iter=40)
    r2 = oracle.solve(A, b + A @ d, p["x0"] + d, stop=oracle.STOP_NONE, max_iter=40)
    np.testing.assert_allclose(r2["x"], r1["x"] + d, rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- stopping rules

def test_epsmem_threshold_is_eq10():
    """Eq. 10: stop iff every violated row is closer than eps to its half-space."""
    A = np.array([[3.0, 4.0], [0.0, -1.0]])
    b = np.array([5.0, 10.0])
    # distance of x to the first half-space = (3x1 + 4x2 - 5) / 5
    x_in = np.array([1.0 / 3.0 * 0 + 0.6, 0.8 + 0.5e-7 * 5 / 4 * 0.99])
    dist = (A[0] @ x_in - 5.0) / 5.0
    assert 0 < dist < 1e-7
    res = oracle.solve(A, b, x_in, stop=oracle.STOP_EPSMEM, eps=1e-7, max_iter=0)
    assert res["status"] == oracle.OK and res["iters"] == 0
    x_out = np.array([0.6, 0.8 + 2e-7])
    res = oracle.solve(A, b, x_out, stop=oracle.STOP_EPSMEM, eps=1e-7, max_iter=0)
    assert res["status"] == oracle.NOT_CONVERGED


def test_max_iter_not_converged_and_counts():
    p = workloads.model_system(16, seed=1)
    res = oracle.solve(p["A"], p["b0"], p["x0"], stop=oracle.STOP_STEP, eps=1e-8,
                       max_iter=7)
    assert res["status"] == oracle.NOT_CONVERGED
    assert res["iters"] == 7
    assert res["tick"] == 7


def test_model_system_converges_feasible():
    p = workloads.model_system(32, seed=3)
    res = oracle.solve(p["A"], p["b0"], p["x0"], stop=oracle.STOP_STEP, eps=1e-8,
                       max_iter=200000)
    assert res["status"] == oracle.OK
    viol = p["A"] @ res["x"] - p["b0"]
    assert viol.max() <= 1e-6


def test_maxviol_rel_rule():
    p = workloads.small_polytope(n=4, m=16, seed=21)
    res = oracle.solve(p["A"], p["b0"], p["x0"], stop=oracle.STOP_MAXVIOL_REL,
                       eps=1e-6, max_iter=100000)
    assert res["status"] == oracle.OK
    viol = (p["A"] @ res["x"] - p["b0"]).max()
    assert viol <= 1e-6 * np.abs(p["b0"]).max()
    assert res["maxviol"] == pytest.approx(viol, abs=1e-12)


# ---------------------------------------------------------------- norms and storage

def test_norms_match_library():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((37, 53))
    n2, zero = oracle.norms2(A)
    np.testing.assert_allclose(n2, np.einsum("ij,ij->i", A, A), rtol=1e-14)
    A[5] = 0.0
    _, zero = oracle.norms2(A)
    assert zero == 1


def _bf16_library(a):
    import torch
    return torch.from_numpy(a).to(torch.bfloat16).to(torch.float32).numpy()


def test_bf16_rounding_matches_library_bit_exact():
    rng = np.random.default_rng(0)
    a = rng.standard_normal(200000).astype(np.float32) * np.float32(3.0)
    # ties: values exactly halfway between two bf16 neighbours, both parities
    base = np.arange(1, 2001, dtype=np.uint32) << np.uint32(16)
    ties = ((base | np.uint32(0x3f800000)) + np.uint32(0x8000)).view(np.float32)
    special = np.array([0.0, -0.0, 1e-40, -1e-40, 3.3895314e38, 1.0, -1.0,
                        65504.0, 1.17549435e-38], np.float32)
    for arr in (a, ties, special):
        got = oracle.quantize_bf16(arr)
        np.testing.assert_array_equal(got.view(np.uint32), _bf16_library(arr).view(np.uint32))


def test_e4m3_rounding_matches_library_bit_exact():
    import torch
    rng = np.random.default_rng(1)
    A = rng.standard_normal((64, 300)).astype(np.float32)
    A[3, 7] = 0.0
    A[4] *= np.float32(1e-3)      # pushes many codes into the subnormal range
    q, s = oracle.quantize_e4m3_rows(A)
    # scales are powers of two with max |a| / s in (224, 448]
    amax = np.abs(A).max(axis=1)
    ratio = amax / s
    assert np.all((ratio > 224) & (ratio <= 448))
    assert np.all(np.frexp(s)[0] == 0.5)
    lib = torch.from_numpy(A / s[:, None]).to(torch.float8_e4m3fn).to(torch.float32).numpy()
    np.testing.assert_array_equal(q, lib * s[:, None])
    # every e4m3 code exactly, and every midpoint between neighbours (ties)
    codes = torch.arange(0, 256, dtype=torch.uint8).view(torch.float8_e4m3fn).to(torch.float32).numpy()
    finite = np.sort(np.unique(codes[np.isfinite(codes) & (np.abs(codes) <= 448)]))
    mids = ((finite[:-1].astype(np.float64) + finite[1:]) / 2).astype(np.float32)
    for arr in (finite, mids):
        row = arr[None, :].astype(np.float32)
        # scale 1 is chosen whenever max |a| is in (224, 448]
        row = np.concatenate([row, np.array([[448.0]], np.float32)], axis=1)
        q, s = oracle.quantize_e4m3_rows(row)
        assert s[0] == 1.0
        lib = torch.from_numpy(row).to(torch.float8_e4m3fn).to(torch.float32).numpy()
        np.testing.assert_array_equal(q, lib)


def test_binary32_entry_points_match_double_entry_points():
    """The binary32-input Map/Reduce and norms read the same exact values."""
    rng = np.random.default_rng(4)
    A32 = rng.standard_normal((60, 45)).astype(np.float32)
    b = rng.standard_normal(60)
    x = rng.standard_normal(45) * 3
    n2a, _ = oracle.norms2(A32)
    n2b, _ = oracle.norms2(A32.astype(np.float64))
    np.testing.assert_array_equal(n2a, n2b)
    m1 = oracle.map_reduce(A32, b, n2a, x)
    m2 = oracle.map_reduce(A32.astype(np.float64), b, n2b, x)
    np.testing.assert_array_equal(m1["y"], m2["y"])
    np.testing.assert_array_equal(m1["r"], m2["r"])
    assert m1["h"] == m2["h"]


def test_maxviol_rel_threshold_is_relative_to_max_b():
    """The relative rule stops when max_i r_i <= eps * max_i |b_i|: with
    max|b| = 1000 and eps = 1e-6 the threshold is 1e-3, so a point violating
    one row by 5e-4 is accepted at once and one violating it by 2e-3 is not."""
    A = np.array([[1.0, 0.0], [0.0, 1.0]])
    b = np.array([1000.0, 1.0])
    res = oracle.solve(A, b, np.array([1000.0 + 5e-4, 0.0]), stop=oracle.STOP_MAXVIOL_REL,
                       eps=1e-6, max_iter=0)
    assert res["status"] == oracle.OK and res["iters"] == 0
    res = oracle.solve(A, b, np.array([1000.0 + 2e-3, 0.0]), stop=oracle.STOP_MAXVIOL_REL,
                       eps=1e-6, max_iter=0)
    assert res["status"] == oracle.NOT_CONVERGED


def test_only_strictly_violated_rows_count():
    """Eq. 7 / Eq. 8: a row contributes iff r_i > 0.  Rows with r_i = 0
    exactly or slightly negative add nothing to y and are not counted in h."""
    A = np.array([[1.0, 0.0], [0.0, 1.0], [0.0, 1.0]])
    b = np.array([1.0, 1.0, 1.0 + 5e-4])
    n2, _ = oracle.norms2(A)
    mr = oracle.map_reduce(A, b, n2, np.array([3.0, 1.0]))   # r = (2, 0, -5e-4)
    assert mr["h"] == 1
    np.testing.assert_array_equal(mr["y"], [2.0, 0.0])
    assert mr["maxviol"] == 2.0


# ---- compressed-row (sparse) form ---------------------------------------------

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_csr_map_reduce_equals_dense_oracle_bitwise(seed):
    """Leaving out the zero entries changes no sum (a zero product adds
    nothing), so the compressed-row Map/Reduce is the dense one bit for bit
    on the same matrix, including ragged rows and unused columns."""
    from paper_2003_09956_gb300 import workloads
    g = np.random.default_rng(seed)
    m, n = 300, 90
    lengths = g.integers(1, 40, m)
    p = workloads.sparse_system(m, n, 0, seed=seed, lengths=lengths)
    A = workloads.csr_to_dense(p["rp"], p["ci"], p["val"], n)
    n2d, zd = oracle.norms2(A)
    n2s, zs = oracle.norms2_csr(p["rp"], p["val"])
    np.testing.assert_array_equal(n2s, n2d)
    assert zs == zd == 0
    b = oracle.tick_b(p["b0"], p["Av"], 0.3, 5)
    x = g.normal(0.0, 2.0, n)
    d = oracle.map_reduce(A, b, n2d, x)
    c = oracle.map_reduce_csr(p["rp"], p["ci"], p["val"], n, b, n2s, x)
    np.testing.assert_array_equal(c["y"], d["y"])
    np.testing.assert_array_equal(c["r"], d["r"])
    assert (c["h"], c["maxviol"], c["maxnorm"], c["maxb"]) == \
        (d["h"], d["maxviol"], d["maxnorm"], d["maxb"])
    assert 0 < c["h"] < m


def test_csr_model_system_is_the_model_system():
    from paper_2003_09956_gb300 import workloads
    p = workloads.model_system_csr(7, seed=4)
    q = workloads.model_system(7, seed=4)
    np.testing.assert_array_equal(workloads.csr_to_dense(p["rp"], p["ci"], p["val"], 7), q["A"])
    np.testing.assert_array_equal(p["b0"], q["b0"])
    n2, zero = oracle.norms2_csr(p["rp"], p["val"])
    np.testing.assert_array_equal(n2, np.r_[np.ones(14), 7.0])
    assert zero == 0


# ------------------------------------------------------------------ ModAPL exchange

def _split_records(A, b, n2, x, bounds):
    """Each worker's Map and local Reduce over its contiguous block of rows."""
    return [oracle.map_reduce(np.ascontiguousarray(A[a:c]), b[a:c], n2[a:c], x) for a, c in bounds]


@pytest.mark.parametrize("bounds", [[(0, 1), (1, 3)], [(0, 2), (2, 3)], [(0, 1), (1, 2), (2, 3)],
                                    [(0, 0), (0, 3)]])
def test_combine_hand_worked_2d_split_over_workers(bounds):
    """The hand-worked 2-D example (tests/golden/hand_worked_2d.txt) with its
    rows split among workers: the global Reduce of ModAPL (Section 3) gives
    the worked y, h, maxima and both steps, whatever the split."""
    g = load_golden("hand_worked_2d.txt")
    A = np.array([[1.0, 0.0], [0.0, 1.0], [-1.0, -1.0]])
    b = np.array([1.0, 1.0, 10.0])
    n2 = np.array([1.0, 1.0, 2.0])
    x0 = np.array(g["case1.x0"])
    recs = _split_records(A, b, n2, x0, bounds)
    code, x1, st, y = oracle.combine_step(recs, x0, lam=1.0, rule=oracle.RULE_RELAXED)
    assert code == oracle.IT_STEPPED
    np.testing.assert_array_equal(y, g["case1.y"])
    assert st["h"] == g["case1.h"][0]
    assert st["maxviol"] == g["case1.maxviol"][0] and st["maxnorm"] == g["case1.maxnorm"][0]
    np.testing.assert_array_equal(x1, g["case1.relaxed_x1"])
    _, x1m, _, _ = oracle.combine_step(recs, x0, lam=1.0, rule=oracle.RULE_MODAP)
    np.testing.assert_allclose(x1m, g["case1.modap_x1"], rtol=0, atol=1e-15)


def test_combine_one_worker_equals_iteration():
    """One worker holding every row: the combined step is oracle.iteration's
    step bit for bit (same arithmetic in the same order)."""
    p = workloads.dense_system(400, 37, seed=71)
    A = p["A"].astype(np.float64)
    n2, _ = oracle.norms2(A)
    for rule in (oracle.RULE_RELAXED, oracle.RULE_MODAP):
        code, x1, st, y, _ = oracle.iteration(A, p["b0"], p["Av"], 1e-2, 3, n2, p["x0"], lam=0.7, rule=rule)
        b = oracle.tick_b(p["b0"], p["Av"], 1e-2, 3)
        c2, x2, st2, y2 = oracle.combine_step(_split_records(A, b, n2, p["x0"], [(0, 400)]), p["x0"],
                                              lam=0.7, rule=rule)
        assert c2 == code
        np.testing.assert_array_equal(x2, x1)
        np.testing.assert_array_equal(y2, y)
        assert st2 == st


@pytest.mark.parametrize("R", [2, 3, 7])
def test_combine_contiguous_splits_match_unsplit(R):
    """R workers over contiguous balanced row blocks: h and the maxima are
    exact, y and the step equal the unsplit ones to rounding (only the order
    of the sums differs)."""
    p = workloads.dense_system(501, 40, seed=72 + R)
    A = p["A"].astype(np.float64)
    n2, _ = oracle.norms2(A)
    m = A.shape[0]
    edges = [m * w // R for w in range(R + 1)]
    bounds = list(zip(edges[:-1], edges[1:]))
    full = oracle.map_reduce(A, p["b0"], n2, p["x0"])
    recs = _split_records(A, p["b0"], n2, p["x0"], bounds)
    code, x1, st, y = oracle.combine_step(recs, p["x0"])
    assert st["h"] == full["h"] and st["maxviol"] == full["maxviol"]
    assert st["maxnorm"] == full["maxnorm"] and st["maxb"] == full["maxb"]
    np.testing.assert_allclose(y, full["y"], rtol=1e-13, atol=1e-13 * np.abs(full["y"]).max())
    # reversed worker order: the same up to rounding
    _, xr, str_, yr = oracle.combine_step(recs[::-1], p["x0"])
    np.testing.assert_allclose(xr, x1, rtol=1e-13)
    assert str_["h"] == st["h"]


def test_combine_decisions_follow_the_stop_rules():
    """The stop decision after the exchange: all workers feasible (h = 0)
    stops under any rule but NONE; max r <= eps max|b| over ALL workers."""
    A = np.array([[1.0, 0.0], [0.0, 1.0]])
    n2 = np.ones(2)
    x = np.array([0.5, 2.0])
    b = np.array([1.0, 1.0])
    recs = _split_records(A, b, n2, x, [(0, 1), (1, 2)])
    assert recs[0]["h"] == 0 and recs[1]["h"] == 1
    code, x1, _, _ = oracle.combine_step(recs, x, stop=oracle.STOP_MAXVIOL_REL, eps=0.5)
    assert code == oracle.IT_STEPPED                  # max r = 1 > 0.5 * max|b| = 0.5
    np.testing.assert_array_equal(x1, [0.5, 1.0])
    code, x2, _, _ = oracle.combine_step(recs, x, stop=oracle.STOP_MAXVIOL_REL, eps=1.0)
    assert code == oracle.IT_CONVERGED
    np.testing.assert_array_equal(x2, x)
    feas = _split_records(A, b, n2, np.array([0.5, 0.5]), [(0, 1), (1, 2)])
    assert oracle.combine_step(feas, np.array([0.5, 0.5]), stop=oracle.STOP_STEP, eps=1e-9)[0] == \
        oracle.IT_CONVERGED
    assert oracle.combine_step(feas, np.array([0.5, 0.5]), stop=oracle.STOP_NONE)[0] == oracle.IT_STEPPED
