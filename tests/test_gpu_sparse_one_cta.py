"""Small sparse systems run whole blocks of iterations in one CTA (one
launch per block).  Against the FP64 oracle (one step from the same point,
ambiguity-aware as in test_gpu_sparse.py), across launch boundaries, and
for the path selection itself."""
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


def make(monkeypatch, p, storage, path="one-cta", x0=None):
    monkeypatch.setenv("NSLI_SPARSE_RESIDENT", {"one-cta": "1", "grid": "0", "auto": ""}[path])
    if path == "auto":
        monkeypatch.delenv("NSLI_SPARSE_RESIDENT")
    return nsli.SparseSolver(p["m"], p["n"], p["rp"], p["ci"], p["val"], p["b0"],
                             p["x0"] if x0 is None else x0, Av=p["Av"], storage=storage)


def launches_for(s, iters, block):
    c0 = s.launch_count()
    s.iterate(iters, block_iters=block)
    s.sync()
    return s.launch_count() - c0


def shapes():
    g = np.random.default_rng(11)
    long_rows = np.full(400, 5)
    long_rows[::50] = 2500                      # rows for a warp each
    return {
        "ragged": workloads.sparse_system(3000, 500, 0, seed=2, lengths=g.integers(1, 40, 3000)),
        "long-rows": workloads.sparse_system(400, 3000, 0, seed=4, lengths=long_rows),
        "long-cols": workloads.sparse_system(5000, 1500, 0, seed=5, lengths=g.integers(3, 12, 5000),
                                             dense_cols=2),
        "short-rows": workloads.sparse_system(5000, 2000, 3, seed=3),
        "one-by-one": workloads.sparse_system(1, 1, 1, seed=1),
    }


SHAPES = shapes()


def test_path_selection(monkeypatch):
    """The model system (768 non-zeros) runs on one CTA by default; a system
    whose matrix outgrows the SM's on-chip memory does not; =0 and =1
    override within the shared-memory limit; a system whose iterate does
    not fit in shared memory never does."""
    model = workloads.model_system_csr(256, seed=0)
    with make(monkeypatch, model, "f64", "auto") as s:
        assert launches_for(s, 64, 32) == 1 + 2
    with make(monkeypatch, model, "f64", "grid") as s:
        assert launches_for(s, 64, 32) == 1 + 2 * 64
    big = SHAPES["short-rows"]                  # 15000 non-zeros: past the on-chip budget
    with make(monkeypatch, big, "f32", "auto") as s:
        assert launches_for(s, 64, 32) == 1 + 2 * 64
    with make(monkeypatch, big, "f32", "one-cta") as s:
        assert launches_for(s, 64, 32) == 1 + 2
    wide = workloads.sparse_system(100, 30000, 4, seed=8)   # 30000 columns: too large for shared memory
    with make(monkeypatch, wide, "f32", "one-cta") as s:
        assert launches_for(s, 8, 8) == 1 + 2 * 8


def csr_step_check(s, p, storage, k, rho, rule, lam):
    """One more iteration from the device's own x_k (tick k) against the
    oracle's step from that x_k, element by element (tests/parity.py)."""
    xk = s.get_x()
    shift = oracle.tick_b(p["b0"], p["Av"], rho, k) - p["b0"]
    s.iterate(1, rule=rule, lam=lam, rho=rho)
    x1 = s.get_x()
    ref = parity.CsrMapRef(p["rp"], p["ci"], p["val"], p["n"], p["b0"] + shift,
                           parity.to_accumulation(xk, storage), storage, b_parts=(p["b0"], shift))
    parity.check_dx(ref, xk, x1, None, lam, rule, parity.TOL[storage])


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("rule", ["relaxed", "modap"])
@pytest.mark.parametrize("name", list(SHAPES))
def test_one_step_matches_oracle(monkeypatch, storage, rule, name):
    """After 3 iterations on one CTA, one more from the device's own x_k
    agrees with the oracle's step element by element (1e-5 relative, 1e-12
    for binary64, plus the column's rounding bound)."""
    p = SHAPES[name]
    rho, lam = 1e-3, (1.0 if rule == "relaxed" else 0.5)
    with make(monkeypatch, p, storage) as s:
        s.iterate(3, rule=rule, lam=lam, rho=rho)
        assert s.result()["tick"] == 3
        csr_step_check(s, p, storage, 3, rho, rule, lam)


@pytest.mark.parametrize("rule", ["relaxed", "modap"])
def test_launch_splits_are_bitwise_equal(monkeypatch, rule):
    """40 iterations as one launch, as blocks of 7, and as 40 calls of one:
    identical bits (only x, x64 and the state cross a launch boundary), and
    identical again on a second solver."""
    p = SHAPES["long-cols"]
    xs = []
    for block in (40, 7, 1, 40):
        with make(monkeypatch, p, "f32") as s:
            if block == 1:
                for _ in range(40):
                    s.iterate(1, rho=1e-3, rule=rule, lam=0.5)
            else:
                s.iterate(40, rho=1e-3, rule=rule, lam=0.5, block_iters=block)
            xs.append(s.get_x())
            assert s.result()["tick"] == 40
    for x in xs[1:]:
        np.testing.assert_array_equal(xs[0], x)


@pytest.mark.parametrize("stop,eps", [("maxviol_rel", 1e-6), ("epsmem", 1e-7), ("step", 1e-9)])
def test_solve_stop_rules_match_grid(monkeypatch, stop, eps):
    """Every stop rule (binary32 candidates confirmed by the binary64
    check, the step rule in binary64) ends after the oracle's iteration
    count within 1%, on one CTA and on the grid kernels alike."""
    p = workloads.sparse_system(600, 150, 6, seed=41, x0_std=1.0)
    A = workloads.csr_to_dense(p["rp"], p["ci"], p["val"], p["n"])
    ostop = {"maxviol_rel": oracle.STOP_MAXVIOL_REL, "epsmem": oracle.STOP_EPSMEM,
             "step": oracle.STOP_STEP}[stop]
    ref = oracle.solve(A, p["b0"], p["x0"], stop=ostop, eps=eps, max_iter=400000)
    assert ref["status"] == oracle.OK
    res = {}
    for path in ("one-cta", "grid"):
        with make(monkeypatch, p, "f64", path) as s:
            res[path] = s.solve(stop=stop, eps=eps, max_iter=400000, block_iters=256)
        assert res[path]["status"] == nsli.OK
        assert abs(res[path]["iters"] - ref["iters"]) <= max(2, 0.01 * ref["iters"]), \
            (path, res[path]["iters"], ref["iters"])


def test_iteration_cap_and_model_system_x(monkeypatch):
    """max_iter ends a one-CTA run with NOT_CONVERGED after exactly max_iter
    updates; the model system's solved x equals the oracle's."""
    p = workloads.model_system_csr(256, seed=3)
    with make(monkeypatch, p, "f64") as s:
        res = s.solve(stop="step", eps=1e-8, max_iter=1000, block_iters=300)
        assert res["status"] == nsli.NOT_CONVERGED and res["iters"] == 1000
    A = workloads.csr_to_dense(p["rp"], p["ci"], p["val"], p["n"])
    ref = oracle.solve(A, p["b0"], p["x0"], stop=oracle.STOP_STEP, eps=1e-8, max_iter=200000)
    with make(monkeypatch, p, "f64") as s:
        res = s.solve(stop="step", eps=1e-8, max_iter=200000)
        xg = s.get_x()
    assert res["status"] == nsli.OK
    assert abs(res["iters"] - ref["iters"]) <= max(1, 0.01 * ref["iters"])
    np.testing.assert_allclose(xg, ref["x"], rtol=0, atol=1e-6 * np.abs(p["b0"]).max())


def test_shared_memory_limit(monkeypatch):
    """The largest binary32 system whose x64, y, x, c and step table fit the
    one-CTA shared-memory limit (8000 x 6000: 216008 of 221184 bytes) runs on
    one CTA and matches the oracle's step; 300 more columns (222008 bytes)
    fall back to the grid kernels even when the one-CTA path is forced."""
    p = workloads.sparse_system(8000, 6000, 4, seed=17)
    with make(monkeypatch, p, "f32") as s:
        assert launches_for(s, 4, 4) == 1 + 1
    with make(monkeypatch, p, "f32") as s:
        s.iterate(2, rule="relaxed", lam=1.0, rho=1e-3)
        csr_step_check(s, p, "f32", 2, 1e-3, "relaxed", 1.0)
    wider = workloads.sparse_system(8000, 6300, 4, seed=18)
    with make(monkeypatch, wider, "f32") as s:
        assert launches_for(s, 4, 4) == 1 + 2 * 4
