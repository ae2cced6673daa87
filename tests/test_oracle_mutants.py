"""The oracle pins catch planted mistakes. Each case copies the oracle source,
plants one plausible error (a swapped term, a wrong sign, index or tie rule, a
transposed operand, an off-by-one), compiles the copy on the CPU and runs the
pins that should notice: at least one must fail. The committed oracle is not
modified."""
from __future__ import annotations

import os

import pytest

import oracle
import tests.test_oracle_pins as pins

MUTANTS = {
    "bhattacharyya_branches_swapped": (
        "tmp[2 * t] = 2.0 * zt - zt * zt;\n      tmp[2 * t + 1] = zt * zt;",
        "tmp[2 * t] = zt * zt;\n      tmp[2 * t + 1] = 2.0 * zt - zt * zt;",
        ["test_bhattacharyya_matches_bec_bruteforce", "test_frozen_set_n32"]),
    "H_rows_are_G_rows": (
        "H[(size_t)r * N + j] = G[(size_t)j * N + frozen[r]];",
        "H[(size_t)r * N + j] = G[(size_t)frozen[r] * N + j];",
        ["test_parity_matrix_annihilates_code"]),
    "binary_labels_not_gray": (
        "static int gray(int l) { return l ^ (l >> 1); }",
        "static int gray(int l) { return l; }",
        ["test_demod_packs_gray_labels"]),
    "labels_lsb_first": (
        "if (pos < N) bits[pos] = (uint8_t)((label >> (nb - 1 - k)) & 1);",
        "if (pos < N) bits[pos] = (uint8_t)((label >> k) & 1);",
        ["test_demod_packs_gray_labels"]),
    "outside_distance_sign": (
        "else d = outside ? 256 + mag : 256 - mag;",
        "else d = outside ? 256 - mag : 256 - mag;",
        ["test_demod_hand_vectors"]),
    "tie_direction_at_lowest_level": (
        "else dir = (l == 0) ? +1 : -1;",
        "else dir = -1;",
        ["test_demod_hand_vectors"]),
    "truncating_quantiser": (
        "int32_t aq = (int32_t)nearbyintf(x);",
        "int32_t aq = (int32_t)x;",
        ["test_demod_hand_vectors", "test_demod_hard_point_is_nearest_point"]),
    "threshold_goes_down": (
        "int l = (t < 0) ? 0 : (int)(t / 512);",
        "int l = (t <= 0) ? 0 : (int)((t - 1) / 512);",
        ["test_demod_hand_vectors", "test_demod_hard_point_is_nearest_point"]),
    "colex_reset_off_by_one": (
        "for (int i = 0; i < j; ++i) p[i] = i;\n      return 1;",
        "for (int i = 0; i < j; ++i) p[i] = i + 1;\n      return 1;",
        ["test_tep_order_all_neighbours", "test_grand_ab_is_ml_within_radius"]),
    "alpha_digit_most_significant_first": (
        "for (int j = 0; j < w; ++j) { /* digit j belongs to the j-th smallest rank */",
        "for (int j = w - 1; j >= 0; --j) { /* digit j belongs to the j-th smallest rank */",
        ["test_tep_order_all_neighbours"]),
    "invalid_teps_counted": (
        "        if (!valid) continue;\n        ++count;",
        "        ++count;\n        if (!valid) continue;",
        ["test_tep_order_partial_neighbours", "test_symbol_level_matches_codebook_bruteforce"]),
    "syndrome_parity_not_reduced": (
        "parity ^= __builtin_popcountll(Hrows[(size_t)r * NW + w] & x[w]) & 1;",
        "parity ^= __builtin_popcountll(Hrows[(size_t)r * NW + w] & x[w]);",
        ["test_decode_noise_free", "test_grand_ab_is_ml_within_radius"]),
    "cap_off_by_one": (
        "  return count >= c->cap;\n}",
        "  return count > c->cap;\n}",
        ["test_cap_boundary"]),
    "sort_ties_to_higher_index": (
        "if (best < 0 || s[i].key < s[best].key) best = i; /* ties: lower index first */",
        "if (best < 0 || s[i].key <= s[best].key) best = i; /* ties: lower index first */",
        ["test_symbol_level_matches_codebook_bruteforce", "test_selection_ties_break_by_index"]),
    "nearer_axis_tie_counts_as_vertical": (
        "if (s->Q.dq < s->I.dq) m |= 32;",
        "if (s->Q.dq <= s->I.dq) m |= 32;",
        ["test_demod_hand_vectors"]),
    "nearer_axis_order_reversed": (
        "if (order == ORDER_NNE_DSORT && t->Q.dq < t->I.dq) {",
        "if (order == ORDER_NNE_DSORT && t->Q.dq > t->I.dq) {",
        ["test_nearer_axis_first_single_error", "test_order_variants_match_codebook_bruteforce"]),
    "five_point_away_on_the_near_side": (
        "int aI = lI - t->I.dir, aQ = lQ - t->Q.dir;",
        "int aI = lI + t->I.dir, aQ = lQ - t->Q.dir;",
        ["test_order_variants_match_codebook_bruteforce"]),
    "five_point_walk_in_base_3": (
        "walk_teps(Sp, order == ORDER_NNE5 ? 4 : 3, exists, qam_visit, &c);",
        "walk_teps(Sp, order == ORDER_NNE5 ? 3 : 3, exists, qam_visit, &c);",
        ["test_five_point_away_error", "test_order_variants_match_codebook_bruteforce"]),
    "level_not_clamped_to_the_top": (
        "  if (l > sqrtM - 1) l = sqrtM - 1;\n",
        "  if (0) l = sqrtM - 1;\n",
        ["test_demod_hard_point_is_nearest_point"]),
    "q_label_before_i_label": (
        "  int label = (gI << m) | gQ;\n  int nb = 2 * m;",
        "  int label = (gQ << m) | gI;\n  int nb = 2 * m;",
        ["test_demod_packs_gray_labels", "test_decode_noise_free"]),
    "literal_distance_not_clamped_at_zero": (
        "  if (d < 0) d = 0;\n",
        "  if (0) d = 0;\n",
        ["test_demod_hand_vectors"]),
    "nonfinite_not_read_as_zero": (
        "  if (s.nonfinite) { a = 0.0f; b = 0.0f; }",
        "  if (0) { a = 0.0f; b = 0.0f; }",
        ["test_nonfinite_coordinate_reads_as_zero"]),
    "neighbour_direction_flipped": (
        "  if (delta > 0) dir = -1;\n  else if (delta < 0) dir = +1;",
        "  if (delta > 0) dir = +1;\n  else if (delta < 0) dir = -1;",
        ["test_demod_hand_vectors", "test_injected_error_at_least_reliable_symbol"]),
    "diagonal_with_either_neighbour": (
        "((ex_h && ex_v) ? 4 : 0)",
        "((ex_h || ex_v) ? 4 : 0)",
        ["test_symbol_level_matches_codebook_bruteforce"]),
    "key_sum_of_distances": (
        "  s.key = (uint32_t)s.I.dq * (uint32_t)s.I.dq + (uint32_t)s.Q.dq * (uint32_t)s.Q.dq;",
        "  s.key = (uint32_t)s.I.dq + (uint32_t)s.Q.dq;",
        ["test_demod_hand_vectors"]),
    "bit_level_zero_is_one": (
        "    ybits[j] = (uint8_t)(v < 0.0f);",
        "    ybits[j] = (uint8_t)(v <= 0.0f);",
        ["test_bit_level_hard_decision_of_zero"]),
}


def _call(name, lib):
    fn = getattr(pins, name)
    import inspect

    params = inspect.signature(fn).parameters
    marks = getattr(fn, "pytestmark", [])
    grids = [m for m in marks if m.name == "parametrize"]
    calls = [{}]
    for mk in grids:
        argnames = [a.strip() for a in mk.args[0].split(",")] if isinstance(mk.args[0], str) else list(mk.args[0])
        new = []
        for c in calls:
            for val in mk.args[1]:
                vals = val if len(argnames) > 1 else (val,)
                d = dict(c)
                d.update(dict(zip(argnames, vals)))
                new.append(d)
        calls = new
    for kw in calls:
        if "oracle_lib" in params:
            kw = dict(kw, oracle_lib=lib)
        fn(**kw)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new, tests = MUTANTS[name]
    src = oracle.source_text()
    assert src.count(old) == 1, f"mutation anchor not found exactly once: {name}"
    so = oracle.build_variant(src.replace(old, new), str(tmp_path / "mutant.so"))
    caught = []
    oracle.use_library(so)
    try:
        for t in tests:
            try:
                _call(t, oracle)
            except (AssertionError, ValueError, IndexError) as e:
                caught.append((t, type(e).__name__))
    finally:
        oracle.use_library(None)
    assert caught, f"no pin failed for the planted mistake {name}"
