"""Catch-up rate measured through the C ABI against the oracle: the 1-D
closed forms (see test_catchup.py) and, on a 16-dimensional model system,
the same bracket as the oracle's search over the same trial rates."""
import math

import numpy as np
import pytest

import oracle
from paper_2003_09956_gb300 import catchup, nsli

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="session", autouse=True)
def built_library():
    from paper_2003_09956_gb300 import _build
    _build.build()
    nsli.load()


def oracle_trial(p, rule, lam, eps, K):
    def trial(rho):
        r = oracle.solve(p["A"], p["b0"], p["x0"], Av=p["Av"], rho=rho, lam=lam, rule=rule,
                         stop=oracle.STOP_EPSMEM, eps=eps, max_iter=K)
        return r["status"] == oracle.OK
    return trial


def test_gpu_modap_catchup_closed_form_1d():
    p = catchup.model_system_translated(1, seed=11)
    lam, K, eps = 1.0, 500, 1e-7
    exact = lam - (p["x0"][0] - 100.0 - eps) / K
    with catchup.GpuTrials(p, "modap", lam, eps, K, storage="f64") as t:
        lo, hi, _ = catchup.max_rate(t, 1e-3, steps=14)
    assert lo <= exact * (1 + 1e-9) and exact <= hi * (1 + 1e-9), (lo, exact, hi)


def test_gpu_relaxed_lags_by_exactly_rho_1d():
    p = catchup.model_system_translated(1, seed=12)
    eps = 1e-7
    with catchup.GpuTrials(p, "relaxed", 1.0, eps, 50, storage="f64") as t:
        lo, hi, _ = catchup.max_rate(t, 1e-3, steps=14)
    assert lo <= eps * (1 + 1e-6) and eps <= hi * (1 + 1e-6), (lo, hi)


# Algorithm 1's catch-up rate is eps-sized (it trails the moving face by
# rho), far below the binary32 resolution of coordinates near 200 (ulp
# 1.5e-5): in binary32 arithmetic the rounding of x, not rho, decides whether
# the binary64 iterate lands inside.  It is compared in binary64 only.
@pytest.mark.parametrize("rule,lam,rho0,storage", [("modap", 4.0, 1e-3, "f64"),
                                                   ("modap", 4.0, 1e-3, "f32"),
                                                   ("relaxed", 1.0, 1e-9, "f64")])
def test_gpu_catchup_bracket_matches_oracle(rule, lam, rho0, storage):
    n, eps, K = 16, 1e-7, 2000
    p = catchup.model_system_translated(n, seed=5)
    rid = oracle.RULE_MODAP if rule == "modap" else oracle.RULE_RELAXED
    lo_o, hi_o, tr_o = catchup.max_rate(oracle_trial(p, rid, lam, eps, K), rho0, steps=8)
    with catchup.GpuTrials(p, rule, lam, eps, K, storage=storage) as t:
        lo_g, hi_g, tr_g = catchup.max_rate(t, rho0, steps=8)
    width = math.log(hi_o / lo_o)
    assert lo_o > 0 and lo_g > 0
    assert abs(math.log(lo_g / lo_o)) <= 2 * width + 1e-9, (tr_o, tr_g)
    # away from the boundary both sides take the same decisions
    for (r_o, ok_o), (r_g, ok_g) in zip(tr_o, tr_g):
        if r_o != r_g:
            break
        if abs(math.log(r_o / lo_o)) > 2 * width:
            assert ok_o == ok_g, (r_o, ok_o, ok_g)


def test_gpu_catchup_report_fields():
    p = catchup.model_system_translated(64, seed=2)
    p["name"] = "model-64"
    r = catchup.catchup(p, "modap", 8.0, eps=1e-7, max_iter=3000, storage="f64", steps=4)
    assert r["rho_max_per_iteration"] > 0
    assert r["rho_max_per_iteration"] * 8.0 <= 8.0  # rho sqrt(n) <= lambda
    assert r["iterations_at_rho_max"] <= 3000
    assert r["units_per_s_total"] == pytest.approx(r["units_per_s_per_coordinate"] * 8.0)
