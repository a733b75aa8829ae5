"""Checkpoint and resume through the C ABI.

The state of a run is the binary64 iterate x and the tick k (plus the
constant system and parameters).  Saving them with nsli_get_x and the
result's tick, then giving them to another handle of the same system with
nsli_set_x and nsli_update_b(NULL, k), continues the run exactly: K1 + K2
iterations in two handles equal K1 + K2 iterations in one, bit for bit."""
import numpy as np
import pytest

from paper_2003_09956_gb300 import nsli, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session", autouse=True)
def built_library():
    from paper_2003_09956_gb300 import _build
    _build.build()
    nsli.load()


def dense(p, storage):
    src = p["A"].astype(np.float64) if storage == "f64" else p["A"]
    return nsli.Solver(src, p["b0"], p["x0"], Av=p["Av"], storage=storage)


def sparse(p, storage):
    return nsli.SparseSolver(p["m"], p["n"], p["rp"], p["ci"], p["val"], p["b0"], p["x0"], Av=p["Av"],
                             storage=storage)


@pytest.mark.parametrize("kind,storage,rule", [("dense", "f32", "relaxed"), ("dense", "bf16", "modap"),
                                               ("dense", "f64", "relaxed"), ("sparse", "f32", "modap")])
def test_resume_from_saved_x_and_tick_is_exact(kind, storage, rule):
    K1, K2, rho = 13, 9, 1e-3
    lam = 1.0 if rule == "relaxed" else 0.5
    if kind == "dense":
        p, make = workloads.dense_system(3000, 700, seed=71), dense
    else:
        p, make = workloads.sparse_system(5000, 900, 10, seed=72), sparse
    with make(p, storage) as s:
        s.iterate(K1 + K2, rule=rule, lam=lam, rho=rho, block_iters=4)
        x_once = s.get_x()
        assert s.result()["tick"] == K1 + K2
    with make(p, storage) as s:
        s.iterate(K1, rule=rule, lam=lam, rho=rho, block_iters=4)
        x_saved, tick = s.get_x(), s.result()["tick"]
    assert tick == K1
    with make(p, storage) as s:
        s.set_x(x_saved)
        s.update_b(None, tick=tick)
        s.iterate(K2, rule=rule, lam=lam, rho=rho, block_iters=4)
        np.testing.assert_array_equal(s.get_x(), x_once)
        assert s.result()["tick"] == K1 + K2
