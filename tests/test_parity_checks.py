"""The element-by-element checker of tests/parity.py, on the CPU: a binary32
emulation of the Map/Reduce (the arithmetic the kernels do, in another
order) passes it, and results with a planted mistake fail it."""
import numpy as np
import pytest

import oracle
import parity
from paper_2003_09956_gb300 import workloads


def emulate_f32(A, b, x, G=8):
    """Binary32 Map (dots in float32) and Reduce (per-block float32 partial
    sums, then binary64 over the blocks), as the kernels are structured."""
    A32 = np.asarray(A, np.float32)
    x32 = np.asarray(x, np.float32)
    r = (A32 @ x32).astype(np.float32) - np.asarray(b, np.float32)
    n2 = (A32.astype(np.float64) ** 2).sum(1)
    inv = (1.0 / n2).astype(np.float32)
    c = np.where(r > 0, r * inv, np.float32(0)).astype(np.float32)
    parts = [(c[i::G, None] * A32[i::G]).sum(0, dtype=np.float32) for i in range(G)]
    y = np.sum(np.array(parts, np.float64), axis=0)
    return y, int((r > 0).sum()), float(r.max())


@pytest.fixture(scope="module")
def case():
    p = workloads.dense_system(600, 97, seed=17)
    y, h, mv = emulate_f32(p["A"], p["b0"], p["x0"])
    return p, y, h, mv


def check(p, y, h, mv):
    parity.check_map_reduce(y, h, {"maxviol": mv}, p["A"], p["b0"], p["x0"], "f32",
                            depth=parity.dense_y_depth(600, 8), levels=parity.dot_levels(97))


def test_binary32_emulation_passes(case):
    check(*case)


def test_dropped_row_fails(case):
    p, y, h, mv = case
    n2, _ = oracle.norms2(p["A"])
    r = oracle.map_reduce(p["A"], p["b0"], n2, p["x0"])["r"]
    i = int(np.argmax(r))
    y_bad = y - r[i] / n2[i] * p["A"][i].astype(np.float64)
    with pytest.raises(AssertionError):
        check(p, y_bad, h, mv)
    with pytest.raises(AssertionError):
        check(p, y, h - 1, mv)


def test_one_element_off_by_1e3_relative_fails(case):
    p, y, h, mv = case
    y_bad = y.copy()
    j = int(np.argmax(np.abs(y)))
    y_bad[j] *= 1 + 1e-3
    with pytest.raises(AssertionError):
        check(p, y_bad, h, mv)


def test_transposed_or_sign_errors_fail(case):
    p, y, h, mv = case
    with pytest.raises(AssertionError):
        check(p, -y, h, mv)
    with pytest.raises(AssertionError):
        check(p, np.roll(y, 1), h, mv)


def test_step_check_relaxed_and_modap(case):
    p, y, h, _ = case
    x = p["x0"].astype(np.float32).astype(np.float64)
    for rule, lam in (("relaxed", 1.0), ("modap", 0.5)):
        s = lam / h if rule == "relaxed" else lam / np.linalg.norm(y)
        x1 = x - s * y
        parity.check_step(x, x1, h, p["A"], p["b0"], "f32", depth=parity.dense_y_depth(600, 8),
                          lam=lam, rule=rule, levels=parity.dot_levels(97))
        with pytest.raises(AssertionError):
            parity.check_step(x, x - 1.001 * s * y, h, p["A"], p["b0"], "f32",
                              depth=parity.dense_y_depth(600, 8), lam=lam, rule=rule,
                              levels=parity.dot_levels(97))
