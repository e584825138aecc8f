"""Planted mistakes in copies of the oracle must be caught by the pins.

Each case edits the oracle's C source in a temporary copy (the committed oracle
is never touched), compiles it, and runs the pins cheapest-first until one
fails.  A case passes when some pin rejects the planted mistake, which shows
the pins would notice that class of error in the real oracle.
"""
import functools

import pytest

import oracle
import pins

MUTATIONS = {
    # constants
    "coefficient_digit": [("(float)0.0796819754", "(float)0.0796818754")],
    "scale_one_over_pi": [("(1.0 / (2.0 * 3.1415926536))", "(1.0 / (3.1415926536))")],
    "swap_ss2_ss3": [("fmaf(q2, fmaf(q2, ss4, ss3), ss2)", "fmaf(q2, fmaf(q2, ss4, ss2), ss3)")],
    "drop_ss4_term": [("fmaf(q2, fmaf(q2, fmaf(q2, ss4, ss3), ss2), ss1)",
                       "fmaf(q2, fmaf(q2, ss3, ss2), ss1)")],
    "cos_constant_term": [("fmaf(q2, fmaf(q2, fmaf(q2, cc3, cc2), cc1), 1.0f)",
                           "fmaf(q2, fmaf(q2, fmaf(q2, cc3, cc2), cc1), 0.5f)")],
    # reduction
    "floor_not_round": [("float r = rintf(x1);\n    return x1 - r;",
                         "float r = floorf(x1);\n    return x1 - r;")],
    "round_half_away": [("float r = rintf(x1);\n    return x1 - r;",
                         "float r = roundf(x1);\n    return x1 - r;")],
    "dropped_square": [("float q2 = q1 * q1;", "float q2 = q1;")],
    "compensated_no_low_part": [("q = fmaf(x, klo, q);", "")],
    "compensated_low_part_sign": [("q = fmaf(x, klo, q);", "q = fmaf(-x, klo, q);")],
    # doubling
    "doubling_sign": [("float c2 = fmaf(-s1, s1, c1 * c1);", "float c2 = fmaf(s1, s1, c1 * c1);")],
    "doubling_transposed": [("float s2 = 2.0f * (s1 * c1);", "float s2 = 2.0f * (s1 * s1);")],
    "doubling_eq2": [("float c2 = fmaf(-s1, s1, c1 * c1);",
                      "float c2 = fmaf(-2.0f * s1, s1, 1.0f);")],
    "second_doubling_missing": [("float c3 = fmaf(-s2, s2, c2 * c2);\n    float s3 = 2.0f * (s2 * c2);",
                                 "float c3 = c2;\n    float s3 = s2;")],
    # amplitude correction
    "drift_correction_dropped": [("fixmag = fmaf(-s2, s2, fmaf(-c2, c2, 2.0f));", "fixmag = 1.0f;")],
    "drift_correction_wrong_pair": [("fixmag = fmaf(-s2, s2, fmaf(-c2, c2, 2.0f));",
                                     "fixmag = fmaf(-s1, s1, fmaf(-c1, c1, 2.0f));")],
    "dagger_no_reciprocal": [("fixmag = 1.0f / mag2;", "fixmag = 1.0f;")],
    # output rounding
    "bf16_truncates": [("u += 0x7fffu + keep_lsb;", "u += 0u * keep_lsb;")],
    "f16_ties_up": [("if (rem > 0x1000u || (rem == 0x1000u && (h & 1u)))", "if (rem >= 0x1000u)")],
    "f16_subnormal_ties_up": [("if (rem > halfway || (rem == halfway && (h & 1u)))",
                               "if (rem >= halfway)")],
    # backward
    "backward_sign": [("gx[i] = fmaf(gs[i], c[i], -(gc[i] * s[i]));",
                       "gx[i] = fmaf(gs[i], c[i], gc[i] * s[i]);")],
    "backward_swapped_operands": [("gx[i] = fmaf(gs[i], c[i], -(gc[i] * s[i]));",
                                   "gx[i] = fmaf(gs[i], s[i], -(gc[i] * c[i]));")],
    "backward_null_gc_sign": [("gx[i] = gs[i] * c[i];", "gx[i] = -(gs[i] * c[i]);")],
    # Huygens sum
    "huygens_conjugate": [("float pi = fmaf(ar[j], s, ai[j] * c);",
                           "float pi = fmaf(ar[j], -s, ai[j] * c);")],
    "huygens_no_falloff": [("ure = fmaf(w, pr, ure);\n            uim = fmaf(w, pi, uim);",
                            "ure = pr + ure;\n            uim = pi + uim;")],
    "huygens_dropped_dz": [("float r = sqrtf(fmaf(dz, dz, fmaf(dy, dy, dx * dx)));",
                            "float r = sqrtf(fmaf(dy, dy, dx * dx));")],
    # threaded driver: a split that drops each thread's last element, and the
    # coefficient set passed where the reduction belongs
    "mt_split_drops_last": [("job[t].hi = n * (t + 1) / nthreads;",
                             "job[t].hi = n * (t + 1) / nthreads - 1;")],
    "mt_coef_as_reduction": [("job[t].reduction = reduction; job[t].coef = coef;",
                              "job[t].reduction = coef; job[t].coef = coef;")],
}

# cheapest first; the expensive statistics run only if nothing cheaper fails
PIN_ORDER = [
    pins.pin_special_values, pins.pin_symmetry, pins.pin_ties_to_even,
    pins.pin_exact_at_whole_turns, pins.pin_quarter_turns, pins.pin_periodicity,
    pins.pin_backward, pins.pin_threaded_driver, pins.pin_bf16_rounding, pins.pin_f16_rounding,
    pins.pin_16bit_outputs, pins.pin_compensated, pins.pin_plain_reduction_bound,
    pins.pin_drift_correction,
    functools.partial(pins.pin_e1_normalized, n=1 << 22),
    functools.partial(pins.pin_e2_dagger, n=1 << 22),
    pins.pin_huygens_fp64, pins.pin_huygens_edges,
    pins.pin_bruteforce,
]


def _build(tmp_path, name, edits):
    with open(oracle.SOURCE) as f:
        src = f.read()
    for old, new in edits:
        assert src.count(old) == 1, f"mutation {name}: anchor not unique or missing: {old!r}"
        src = src.replace(old, new)
    path = tmp_path / f"{name}.c"
    path.write_text(src)
    so = oracle.compile_source(str(path), str(tmp_path / f"lib{name}.so"))
    return src, oracle.OracleLib(so)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    src, lib = _build(tmp_path, name, MUTATIONS[name])
    try:
        pins.pin_coefficients_source(src)
    except AssertionError:
        return
    for pin in PIN_ORDER:
        try:
            pin(lib)
        except (AssertionError, FloatingPointError):
            return
    pytest.fail(f"no pin caught the planted mistake {name!r}")


def test_unmutated_copy_passes_every_pin(tmp_path):
    """The harness itself: an untouched copy passes all pins (so the cases
    above fail for the planted mistake, not for the copying)."""
    src, lib = _build(tmp_path, "identity", [])
    pins.pin_coefficients_source(src)
    for pin in PIN_ORDER:
        pin(lib)
