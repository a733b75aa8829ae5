"""Catch-up rate search (host logic) and its closed forms on the oracle.

On the one-dimensional model system (rows -x <= 0, x <= 200, x <= 100)
moved by -rho per iteration, both rules can be followed by hand from
x0 in (300, 400):
* ModAP (Eq. 12): while x is above the box y > 0, so every step has length
  exactly lambda and x_k = x0 - k lambda.  The test at tick k passes when
  x_k - (100 - k rho) < eps, so within K updates the iteration catches the
  box iff rho < lambda - (x0 - 100 - eps) / K.
* Algorithm 1 with lambda = 1 (Eq. 8): the first step averages two
  projections and lands on 150, the second projects onto x = 100 - rho;
  from then on every step projects onto the face x = 100 - k rho, which
  moves on by rho before the next test.  The lag is exactly rho, so the
  iteration catches the box iff rho < eps (a Fejer process trails a moving
  polytope)."""
import math

import numpy as np
import pytest

import oracle
from paper_2003_09956_gb300 import catchup


def oracle_trial(p, rule, lam, eps, K):
    def trial(rho):
        r = oracle.solve(p["A"], p["b0"], p["x0"], Av=p["Av"], rho=rho, lam=lam, rule=rule,
                         stop=oracle.STOP_EPSMEM, eps=eps, max_iter=K)
        return r["status"] == oracle.OK
    return trial


@pytest.mark.parametrize("thr", [0.37, 1e-9, 123.0])
def test_max_rate_brackets_a_threshold(thr):
    lo, hi, trials = catchup.max_rate(lambda r: r < thr, 1e-3, steps=12)
    assert lo < thr <= hi
    assert hi / lo <= 2.0 ** (2.0 ** -12) * (1 + 1e-12)
    assert all(ok == (r < thr) for r, ok in trials)


def test_max_rate_degenerate_cases():
    lo, hi, _ = catchup.max_rate(lambda r: False, 1.0, limit=10)
    assert lo == 0.0 and hi == 2.0 ** -10
    lo, hi, _ = catchup.max_rate(lambda r: True, 1.0, limit=10)
    assert lo == 2.0 ** 10 and math.isinf(hi)


def test_model_system_translation_direction():
    p = catchup.model_system_translated(5, seed=3)
    v = -np.ones(5)
    np.testing.assert_array_equal(p["Av"], p["A"] @ v)
    # at tick k the box is [-k rho, 200 - k rho]^n: it moves away from x0
    rho, k = 0.5, 7
    b = oracle.tick_b(p["b0"], p["Av"], rho, k)
    np.testing.assert_allclose(b[:5], k * rho)
    np.testing.assert_allclose(b[5:10], 200.0 - k * rho)
    assert b[10] == pytest.approx(200.0 * 4 + 100.0 - 5 * k * rho)


@pytest.mark.parametrize("lam,K", [(1.0, 500), (10.0, 40), (3.0, 1000)])
def test_oracle_modap_catchup_closed_form_1d(lam, K):
    p = catchup.model_system_translated(1, seed=11)
    eps = 1e-7
    exact = lam - (p["x0"][0] - 100.0 - eps) / K
    lo, hi, _ = catchup.max_rate(oracle_trial(p, oracle.RULE_MODAP, lam, eps, K), 1e-3, steps=14)
    assert lo <= exact * (1 + 1e-9) and exact <= hi * (1 + 1e-9), (lo, exact, hi)


def test_oracle_relaxed_lags_by_exactly_rho_1d():
    p = catchup.model_system_translated(1, seed=12)
    eps = 1e-7
    lo, hi, _ = catchup.max_rate(oracle_trial(p, oracle.RULE_RELAXED, 1.0, eps, 50), 1e-3,
                                 steps=14)
    assert lo <= eps * (1 + 1e-6) and eps <= hi * (1 + 1e-6), (lo, hi)


def test_oracle_modap_outruns_relaxed_on_model_system():
    """On a 16-dimensional model system ModAP catches a polytope moving
    orders of magnitude faster than Algorithm 1 does, and never one moving
    faster than its own step: rho sqrt(n) <= lambda."""
    n, eps, K = 16, 1e-7, 2000
    p = catchup.model_system_translated(n, seed=5)
    lam = 4.0
    lo_m, _, _ = catchup.max_rate(oracle_trial(p, oracle.RULE_MODAP, lam, eps, K), 1e-3, steps=8)
    lo_r, _, _ = catchup.max_rate(oracle_trial(p, oracle.RULE_RELAXED, 1.0, eps, K), 1e-9, steps=8)
    assert 0 < lo_m * math.sqrt(n) <= lam
    assert lo_r < 1e-3 * lo_m


def test_sparse_model_system_translation_matches_dense():
    from paper_2003_09956_gb300 import workloads
    p = catchup.model_system_translated_csr(6, seed=1)
    q = catchup.model_system_translated(6, seed=1)
    np.testing.assert_array_equal(workloads.csr_to_dense(p["rp"], p["ci"], p["val"], 6), q["A"])
    np.testing.assert_array_equal(p["Av"], q["Av"])
    np.testing.assert_array_equal(p["x0"], q["x0"])


def test_time_vs_rate_curve_host_logic():
    """The curve takes the median of the repeats at each fraction of the
    catch-up rate and reports whether every repeat reached the polytope."""
    calls = []

    def timed(rho):
        calls.append(rho)
        k = len(calls)
        return rho < 0.95, 10 + int(100 * rho), [0.3, 0.1, 0.2][k % 3]

    pts = catchup.time_vs_rate(timed, 1.0, fractions=(0.0, 0.5, 1.0), repeats=3)
    assert [q["fraction_of_rho_max"] for q in pts] == [0.0, 0.5, 1.0]
    assert calls == [0.0] * 3 + [0.5] * 3 + [1.0] * 3
    assert all(q["solve_ms"] == pytest.approx(200.0) for q in pts)
    assert [q["reached"] for q in pts] == [True, True, False]
    assert pts[1]["iterations"] == 60
