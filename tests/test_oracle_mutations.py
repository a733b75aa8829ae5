"""Each planted mistake in the oracle (on the CPU, in a temporary copy of
its C source) must make at least one pin fail: the pins are not blind to a
dropped term, a wrong sign or index, a transposed operand or a wrong
rounding rule."""
import os

import pytest

import oracle
import test_oracle_pins as pins

# (name, text in nsli_oracle.c, replacement, occurrence to replace: 0 = first)
MUTATIONS = [
    ("residual sign of b", "double ri = dot - b[i];", "double ri = dot + b[i];"),
    ("dot uses x[0]", "dot = dot + a[j] * x[j];", "dot = dot + a[j] * x[0];"),
    ("norm drops the square", "s = s + a * a;", "s = s + (a < 0 ? -a : a);"),
    ("slice divides by ||a||", "double c = ri / n2[i];", "double c = ri / sqrt(n2[i]);"),
    ("slice adds a[0]", "y[j] = y[j] + c * a[j];", "y[j] = y[j] + c * a[0];"),
    ("relaxed step divides by h + 1", "s = lambda / (double)h;", "s = lambda / (double)(h + 1);"),
    ("ModAP step drops lambda", "s = (ynorm > 0.0) ? lambda / ynorm : 0.0;", "s = (ynorm > 0.0) ? 1.0 / ynorm : 0.0;"),
    ("step added, not subtracted", "x[j] = x[j] - d;", "x[j] = x[j] + d;"),
    ("translation sign", "shift = t * Av[i];", "shift = -t * Av[i];"),
    ("Eq. 10 on r instead of r/||a||", "return maxnorm < eps; /* Eq. 10 over all rows */", "return maxviol < eps;"),
    ("max violation relative to 1", "return maxviol <= eps * maxb;", "return maxviol <= eps;"),
    ("violated test includes ties and negatives", "if (ri > 0.0) {\n            /* positive slice", "if (ri > -1e-3) {\n            /* positive slice"),
    ("violated test includes ties", "if (ri > 0.0) {\n            /* positive slice", "if (ri >= 0.0) {\n            /* positive slice"),
    ("bf16 rounds half up", "u = u + 0x7fffu + keep_lsb;", "u = u + 0x8000u;"),
    ("e4m3 scale target 480", "while (ldexp(amax, -e) > 448.0)", "while (ldexp(amax, -e) > 480.0)"),
    ("e4m3 subnormal quantum", "quantum = ldexp(1.0, -9); /* subnormal spacing */", "quantum = ldexp(1.0, -8);"),
    ("exchange takes h as a maximum", "h = h + hs[w];", "h = (hs[w] > h) ? hs[w] : h;"),
    ("exchange drops worker 0's y", "y_out[j] = y_out[j] + yw[j];", "y_out[j] = (w > 0) ? y_out[j] + yw[j] : 0.0;"),
    ("exchange keeps the first worker's maximum", "if (maxviols[w] > mv)", "if (w == 0 && maxviols[w] > mv)"),
]

PIN_CALLS = [
    pins.test_hand_worked_2d_relaxed_and_modap,
    pins.test_hand_worked_single_row_projection,
    pins.test_only_strictly_violated_rows_count,
    lambda: pins.test_single_violated_row_is_orthogonal_projection(0),
    lambda: pins.test_fejer_monotone_relaxed(1.0),
    lambda: pins.test_modap_step_has_length_lambda(0.25),
    pins.test_strictly_feasible_start_is_a_fixed_point,
    pins.test_model_system_exact_rational_recurrence,
    lambda: pins.test_brute_force_vertex_enumeration(2, 10, 0, oracle.RULE_RELAXED),
    lambda: pins.test_tick_is_a_translation(oracle.RULE_RELAXED),
    pins.test_epsmem_threshold_is_eq10,
    pins.test_maxviol_rel_rule,
    pins.test_maxviol_rel_threshold_is_relative_to_max_b,
    pins.test_norms_match_library,
    pins.test_bf16_rounding_matches_library_bit_exact,
    pins.test_e4m3_rounding_matches_library_bit_exact,
    lambda: pins.test_combine_hand_worked_2d_split_over_workers([(0, 1), (1, 3)]),
    lambda: pins.test_combine_hand_worked_2d_split_over_workers([(0, 2), (2, 3)]),
    lambda: pins.test_combine_hand_worked_2d_split_over_workers([(0, 0), (0, 3)]),
]


def test_unmutated_copy_passes_every_pin(tmp_path):
    src = open(oracle._SRC).read()
    path = os.path.join(tmp_path, "orig.c")
    open(path, "w").write(src)
    lib = oracle.compile_source(path, os.path.join(tmp_path, "orig.so"))
    with oracle.library(lib):
        for call in PIN_CALLS:
            call()


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, name, old, new):
    src = open(oracle._SRC).read()
    assert old in src, "mutation anchor missing: %s" % name
    path = os.path.join(tmp_path, "mut.c")
    open(path, "w").write(src.replace(old, new, 1))
    lib = oracle.compile_source(path, os.path.join(tmp_path, "mut.so"))
    caught = []
    with oracle.library(lib):
        for call in PIN_CALLS:
            try:
                call()
            except Exception as e:  # noqa: BLE001 - any failure of a pin counts
                caught.append(type(e).__name__)
                break
    assert caught, "no pin caught the planted mistake: %s" % name
