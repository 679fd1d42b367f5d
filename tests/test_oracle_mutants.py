"""Planted mistakes in the oracle (CPU only): each mutant is a copy of
oracle/shaken_oracle.c with one plausible error -- a dropped term, a wrong sign,
a wrong neighbour index, a transposed bit order, a wrong constant -- compiled on
its own and swapped in for the oracle.  The pins of test_oracle_pins.py must
reject every mutant (at least one pin fails) and accept the unmodified source.
"""
import os

import pytest

from oracle import core
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(core.__file__), "shaken_oracle.c")

# name -> (text of the correct line, text of the planted mistake)
MUTANTS = {
    "field_drops_q_sigma": ("  double b = q * (double)sigma;",
                            "  double b = 0.0 * q * (double)sigma;"),
    "field_lambda_sign": ("  return (a + b) + lambda;", "  return (a + b) - lambda;"),
    "threshold_exponent_sign": ("  double e = orc_exp(-2.0 * y);",
                                "  double e = orc_exp(2.0 * y);"),
    "threshold_drops_factor_2": ("  double e = orc_exp(-2.0 * y);", "  double e = orc_exp(-y);"),
    "exp_drops_taylor_term": (
        "    0x1.5555555555555p-3,  0x1.5555555555555p-5,  0x1.1111111111111p-7,",
        "    0x1.5555555555555p-3,  0.0,  0x1.1111111111111p-7,"),
    "dl_reads_up_row": ("    ya = ((i - 1 + L) % L) * L + j;", "    ya = ((i + 1) % L) * L + j;"),
    "ur_reads_left_column": ("    yb = i * L + (j + 1) % L;", "    yb = i * L + (j - 1 + L) % L;"),
    "philox_multiplier": ("#define ORC_PH_M0 0xD2511F53u", "#define ORC_PH_M0 0xD2511F55u"),
    "philox_products_swapped": ("    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;",
                                "    uint32_t n0 = (uint32_t)(p0 >> 32) ^ c1 ^ k0;"),
    "plane_bit_order_transposed": ("    u |= ((w >> k) & 1u) << (31 - j);",
                                   "    u |= ((w >> k) & 1u) << j;"),
    "lattice_decision_inverted": ("  return ((uint64_t)u < T) ? 1 : -1;",
                                  "  return ((uint64_t)u >= T) ? 1 : -1;"),
    "graph_coupling_sign_dropped": ("      s += (J[e] > 0 ? 1 : -1) * (int64_t)sr[y];",
                                    "      s += (int64_t)sr[y];"),
    "graph_real_drops_q": ("    h = (acc + q * (double)sr[x]) + lambda[x];",
                           "    h = acc + lambda[x];"),
    "graph_plane_draw_wrong_group": (
        "    return orc_draw_plane(seed, (uint32_t)x, (uint32_t)(r >> 5), t, (uint32_t)half, (int)(r & 31));",
        "    return orc_draw_plane(seed, (uint32_t)x, (uint32_t)r, t, (uint32_t)half, (int)(r & 31));"),
    "graph_field_reads_wrong_end": (
        "      int32_t y = half == 0 ? tail[e] : head[e];\n      acc += J[e] * (double)sr[y];",
        "      int32_t y = half == 0 ? head[e] : head[e];\n      acc += J[e] * (double)sr[y];"),
    "graph_pair_sum_uses_sigma": (
        "    out[3] += J[e] * (double)(s[tail[e]] * sp[head[e]]);",
        "    out[3] += J[e] * (double)(s[tail[e]] * s[head[e]]);"),
    "lattice_pair_sum_wrong_row": (
        "      int64_t up = ((i + 1) % L) * L + j, rt = i * L + (j + 1) % L;",
        "      int64_t up = ((i - 1 + L) % L) * L + j, rt = i * L + (j + 1) % L;"),
}


def _pins():
    """The pins as plain calls, cheapest first; each raises AssertionError on failure."""
    return [
        ("philox_curand", pins.test_philox_matches_curand_host_generator),
        ("draw_layouts", pins.test_draw_layouts_match_definition),
        ("threshold_points", pins.test_threshold_exact_points_and_saturation),
        ("threshold_precision", pins.test_threshold_against_high_precision),
        ("exp_libm", pins.test_exp_close_to_libm),
        ("field_rounding", pins.test_field_rounding_order),
        ("worked_thm33", lambda: pins.test_worked_trajectory_thm33(8, 2, 3, core.MODE_SINGLE)),
        ("worked_graph", pins.test_worked_trajectory_through_graph_path),
        ("first_exit", pins.test_first_exit_probability_from_minus),
        ("lattice_sums", pins.test_lattice_sums_match_numpy_hamiltonians),
        ("graph_sums", pins.test_graph_sums_match_numpy_hamiltonians),
        ("lattice_law", lambda: pins.test_lattice_chain_follows_exact_law(core.MODE_SINGLE, None)),
        ("graph_law_int", lambda: pins.test_graph_chain_follows_exact_law(True,
                                                                          core.DRAW_DIRECT)),
        ("graph_law_real", lambda: pins.test_graph_chain_follows_exact_law(False,
                                                                           core.DRAW_DIRECT)),
        ("graph_law_plane", lambda: pins.test_graph_chain_follows_exact_law(True,
                                                                            core.DRAW_PLANE)),
        ("graph_fields_dense", pins.test_graph_fields_match_dense_form),
        ("philox_independent", pins.test_philox_matches_independent_implementation),
    ]


def _failing_pin(so_path, stop_at_first=True):
    """Names of the pins that reject the library at so_path (the first one only by
    default); pins that skip (a missing optional package) do not count."""
    failed = []
    with core.using(so_path):
        for name, pin in _pins():
            try:
                pin()
            except AssertionError:
                failed.append(name)
                if stop_at_first:
                    break
            except pytest.skip.Exception:
                continue
    return failed


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_planted_mistake(name):
    src = open(SRC).read()
    good, bad = MUTANTS[name]
    assert good in src, f"mutation site of {name} not found"
    so = core.build_variant(src.replace(good, bad, 1), name)
    assert _failing_pin(so), f"no pin rejects the mutant {name}"


def test_pins_accept_unmodified_source():
    so = core.build_variant(open(SRC).read(), "unmodified")
    assert _failing_pin(so, stop_at_first=False) == []
