"""Mutation check of the oracle's pins.

Each mutant is the oracle source with one plausible mistake planted (a dropped
factor, a flipped sign, a transposed index, a wrong tie-break, a dropped
candidate, an off-by-one routing test).  It is compiled on the CPU and the
pins are run against it; every mutant must make at least one pin fail.
"""
import os
import subprocess

import pytest

import oracle
import synth
import test_oracle_pins as pins
import test_oracle_reconstruct as rpins
import test_oracle_anchor as apins
import test_oracle_knn as kpins
import test_oracle_cluster as cpins
import test_oracle_unit as upins

SRC = os.path.join(os.path.dirname(os.path.abspath(oracle.__file__)), "riann_oracle.c")

MUTANTS = {
    "drop_factor_4": ("(unsigned __int128)4 * (unsigned __int128)(qq * qq)", "(unsigned __int128)(qq * qq)"),
    "sign_of_C_term": ("- (__int128)p * p * (__int128)C", "+ (__int128)p * p * (__int128)C"),
    "q_squared_not_fourth": ("(unsigned __int128)4 * (unsigned __int128)(qq * qq)", "(unsigned __int128)4 * (unsigned __int128)(qq)"),
    "strict_ring_edge": ("return lhs <= rhs;", "return lhs < rhs;"),
    "abs_diff_not_squared": ("s += (uint32_t)(d * d);", "s += (uint32_t)(d < 0 ? -d : d);"),
    "patch_transposed": ("frame[((int64_t)(y + dy) * W + (x + dx)) * C + c]", "frame[((int64_t)(y + dx) * W + (x + dy)) * C + c]"),
    "brute_force_tie_high": ("if (d < bd) { bd = d; bi = r; }", "if (d <= bd) { bd = d; bi = r; }"),
    "ring_argmin_tie_high": ("if (d < bd || (d == bd && r < bi)) { bd = d; bi = r; }\n      }\n      annf[i] = bi;\n      if (dist) dist[i] = bd;\n      if (count) count[i] = s_size;\n    }\n    free(B); free(ring_size); free(in_all);",
                             "if (d < bd || (d == bd && r > bi)) { bd = d; bi = r; }\n      }\n      annf[i] = bi;\n      if (dist) dist[i] = bd;\n      if (count) count[i] = s_size;\n    }\n    free(B); free(ring_size); free(in_all);"),
    "prev_not_verified": ("int32_t bi = rp;                                /* r_p is always verified */\n      uint32_t bd = Cd;",
                          "int32_t bi = rp;                                /* r_p is always verified */\n      uint32_t bd = 0xffffffffu;"),
    "ring_argmin_takes_worse_lower_index": (
        "if (!in_all[r]) continue;\n        uint32_t d = sqdist(q, R + (int64_t)r * D, D);\n"
        "        if (d < bd || (d == bd && r < bi)) { bd = d; bi = r; }",
        "if (!in_all[r]) continue;\n        uint32_t d = sqdist(q, R + (int64_t)r * D, D);\n"
        "        if (d < bd || (d != bd && r < bi)) { bd = d; bi = r; }"),
    "indexed_argmin_takes_worse_lower_index": (
        "++s_size;\n        uint32_t d = sqdist(q, R + (int64_t)r * D, D);\n"
        "        if (d < bd || (d == bd && r < bi)) { bd = d; bi = r; }",
        "++s_size;\n        uint32_t d = sqdist(q, R + (int64_t)r * D, D);\n"
        "        if (d < bd || (d != bd && r < bi)) { bd = d; bi = r; }"),
    "limit_off_by_one": ("if (ring_limit >= 0 && ns > (uint32_t)ring_limit) {   /* rings too wide: brute force */",
                         "if (ring_limit >= 0 && ns >= (uint32_t)ring_limit) {   /* rings too wide: brute force */"),
    "count_first_ring_only": ("        in_all[r] = (uint8_t)inside;\n        s_size += (uint32_t)inside;",
                              "        in_all[r] = (uint8_t)inside;\n        s_size += (uint32_t)oracle_ring_member(P[(int64_t)r * K], B[0], Cd, alpha_num, alpha_den);"),
    "alpha_inverted": ("__int128 L = qq * ((__int128)A + (__int128)B) - (__int128)p * p * (__int128)C;",
                       "__int128 L = (__int128)p * p * ((__int128)A + (__int128)B) - qq * (__int128)C;"),
    # Sec. 4 reconstruction
    "recon_truncating_average": ("(uint32_t)((2 * sum + count) / (2 * count))", "(uint32_t)(sum / count)"),
    "recon_patch_offset_transposed": ("((int64_t)(y - py) * 8 + (x - px)) * C + c", "((int64_t)(x - px) * 8 + (y - py)) * C + c"),
    "recon_cover_misses_own_row": ("py <= y && py < Hq; ++py", "py < y && py < Hq; ++py"),
    "recon_norm_not_squared": ("g += (unsigned long long)frame[o] * frame[o];", "g += (unsigned long long)frame[o];"),
    # Alg. 1 with random anchors
    "anchor_ring_width_of_first_ring": ("if (anchor_ring_member(A, Ba, alpha_num, alpha_den)) S2[m++] = S[k];",
                                        "if (anchor_ring_member(A, Bi, alpha_num, alpha_den)) S2[m++] = S[k];"),
    "anchor_not_verified": ("if (Ba < bd || (Ba == bd && a < bi)) { bd = Ba; bi = a; }", ""),
    "anchor_draw_modulo": ("S[(int32_t)(((uint64_t)x[0] * (uint64_t)ns) >> 32)]", "S[(int32_t)(x[0] % (uint32_t)ns)]"),
    "anchor_loop_strict": ("while (ns >= L && (int32_t)t < max_rings)", "while (ns > L && (int32_t)t < max_rings)"),
    # index tables (Sec. 3.3 pre-processing)
    "tables_ties_high_index": ("if (u->id != v->id) return u->id < v->id ? -1 : 1;",
                               "if (u->id != v->id) return u->id > v->id ? -1 : 1;"),
    "tables_descending": ("if (u->a != v->a) return u->a < v->a ? -1 : 1;",
                          "if (u->a != v->a) return u->a > v->a ? -1 : 1;"),
    "key_distances_first_key_only": ("P[(int64_t)r * K + m] = sqdist(KP + (int64_t)m * D, R + (int64_t)r * D, D);",
                                     "P[(int64_t)r * K + m] = sqdist(KP, R + (int64_t)r * D, D);"),
    "full_tables_unsorted": ("    qsort(row, (size_t)n, sizeof(uint64_t), cmp_u64);\n", "\n"),
    "anchor_lower_edge_dropped": ("  if (p < q) {\n    const uint64_t lo = (uint64_t)(q - p) * (uint64_t)(q - p);",
                                  "  if (0) {\n    const uint64_t lo = (uint64_t)(q - p) * (uint64_t)(q - p);"),
    "anchor_first_match_not_a_candidate": ("      uint32_t bd = Bi;\n", "      uint32_t bd = 0xffffffffu;\n"),
    "random_field_counter_word3": ("{(uint32_t)q, 0u, frame_id, 1u}", "{(uint32_t)q, 0u, frame_id, 0u}"),
    "anchor_tie_takes_later_anchor": ("if (Ba < bd || (Ba == bd && a < bi)) { bd = Ba; bi = a; }",
                                      "if (Ba <= bd || (Ba == bd && a < bi)) { bd = Ba; bi = a; }"),
    "anchor_final_tie_takes_later": ("if (d < bd || (d == bd && S[k] < bi)) { bd = d; bi = S[k]; }",
                                     "if (d <= bd || (d == bd && S[k] < bi)) { bd = d; bi = S[k]; }"),
    "recon_entry_n_inside": ("if (r < 0 || r >= n) continue;",
                             "if (r < 0 || r > n) continue;"),
    "knn_limit_zero_not_routed": ("all = ring_limit >= 0 && ns > (uint32_t)ring_limit;",
                                  "all = ring_limit > 0 && ns > (uint32_t)ring_limit;"),
    "unit_limit_zero_not_routed": ("if (ring_limit >= 0 && ns > (uint32_t)ring_limit) {\n        unit_brute_force",
                                   "if (ring_limit > 0 && ns > (uint32_t)ring_limit) {\n        unit_brute_force"),
    "philox_multiplier": ("(uint64_t)0xD2511F53u * c0", "(uint64_t)0xD2511F55u * c0"),
    # k-NN output
    "knn_prev_dropped": ("if (all || in_s[r] || r == rp) {", "if (all || in_s[r]) {"),
    "knn_ties_high_index_first": ("return (a->r > b->r) - (a->r < b->r);", "return (a->r < b->r) - (a->r > b->r);"),
    "knn_cut_one_short": ("knn[i * k + j] = j < nc ? cand[j].r : -1;", "knn[i * k + j] = j + 1 < nc ? cand[j].r : -1;"),
    "knn_routing_off_by_one": ("all = ring_limit >= 0 && ns > (uint32_t)ring_limit;",
                               "all = ring_limit >= 0 && ns >= (uint32_t)ring_limit;"),
    "knn_count_includes_prev": ("if (count) count[i] = all ? (uint32_t)n : s_size;",
                                "if (count) count[i] = all ? (uint32_t)n : s_size + 1;"),
    # reference-set clustering
    "cluster_variance_unsquared_mean": ("const unsigned long long v = (unsigned long long)cnt * s2 - s * s;",
                                        "const unsigned long long v = s2 - s;"),
    "cluster_upper_median": ("return v[(cnt - 1) / 2];", "return v[cnt / 2];"),
    "cluster_tie_high_coordinate": ("if (v > best_v) { best_v = v; best_d = d; }", "if (v >= best_v && v) { best_v = v; best_d = d; }"),
    "cluster_no_strict_fallback": ("strict = nle == cnt;", "strict = 0;"),
    "cluster_leaf_off_by_one": ("if (cnt > leaf) {", "if (cnt >= leaf) {"),
    # unit-normalised float variant
    "unit_query_not_normalised": ("unit_normalize(q, D, qn);\n      int32_t bi;",
                                  "for (int32_t u = 0; u < D; ++u) qn[u] = (float)q[u];\n      int32_t bi;"),
    "unit_alpha_inverted": ("const float T = ((float)p * C) / (float)q;", "const float T = ((float)q * C) / (float)p;"),
    "unit_distance_not_rooted": ("  return sqrtf(acc);\n}", "  return acc;\n}"),
    "unit_ring_tie_high": ("if (d < bd || (d == bd && r < bi)) { bd = d; bi = r; }\n      }\n      annf[i] = bi; if (dist) dist[i] = bd; if (count) count[i] = s_size;",
                           "if (d < bd || (d == bd && r > bi)) { bd = d; bi = r; }\n      }\n      annf[i] = bi; if (dist) dist[i] = bd; if (count) count[i] = s_size;"),
    "unit_brute_tie_high": ("if (d < *bd) { *bd = d; *bi = r; }", "if (d <= *bd) { *bd = d; *bi = r; }"),
    "unit_prev_not_verified": ("      bi = rp;\n      bd = Cd;\n", "      bi = rp;\n      bd = INFINITY;\n"),
    "unit_ring_strict_edge": ("return fabsf(A - B) <= T;", "return fabsf(A - B) < T;"),
    "unit_zero_patch_unguarded": ("  if (s == 0) {\n    for (int32_t i = 0; i < D; ++i) out[i] = 0.f;",
                                  "  if (0) {\n    for (int32_t i = 0; i < D; ++i) out[i] = 0.f;"),
    "unit_routing_off_by_one": ("if (ring_limit >= 0 && ns > (uint32_t)ring_limit) {\n        unit_brute_force",
                                "if (ring_limit >= 0 && ns >= (uint32_t)ring_limit) {\n        unit_brute_force"),
    "cluster_right_first": ("stack[2 * top] = b + nl; stack[2 * top + 1] = e; ++top;     /* right, processed after left */\n    stack[2 * top] = b; stack[2 * top + 1] = b + nl; ++top;",
                            "stack[2 * top] = b; stack[2 * top + 1] = b + nl; ++top;\n    stack[2 * top] = b + nl; stack[2 * top + 1] = e; ++top;"),
}


def _pins_fail() -> bool:
    """Run a fast subset of the pins; True if any of them fails."""
    checks = []
    for name in pins.GOLDEN:
        for mode in ("definitional", "indexed"):
            checks.append(lambda name=name, mode=mode: pins.test_golden_fixture(name, mode))
    checks += [pins.test_exact_nn_vs_numpy_random_with_ties, pins.test_exact_nn_vs_numpy_rgb,
               pins.test_ring_member_exact_equalities_by_construction, pins.test_alpha_zero_profile_match,
               pins.test_frame0_is_brute_force, lambda: pins.test_index_tables_vs_numpy(1),
               lambda: pins.test_index_tables_vs_numpy(3)]

    def alpha_one():
        w = synth.WORKLOADS["tiny"]
        R = synth.workload_reference(w)[:1024]
        KP = synth.keypoints_kmeanspp(R, 8, 11)[1]
        frames = synth.Video(w.video).frames(0, 3)[:, :48, :64]
        idx = oracle.Index(R, KP)
        pins.test_alpha_one_is_exact_nn_every_frame((R, KP, frames, idx))
        pins.test_monotone_never_worse_than_previous((R, KP, frames, idx)) if False else None

    def modes_agree():
        for a in ((1, 4), (1, 1)):
            pins.test_definitional_equals_indexed_random(1, a)
            pins.test_definitional_equals_indexed_random(3, a)

    def modes_agree_on_a_chain():
        # previous matches from a video chain are good ones, unlike random
        # fields: r_p then often beats members of S with lower indices
        w = synth.WORKLOADS["tiny"]
        R = synth.workload_reference(w)[:1024]
        KP = synth.keypoints_kmeanspp(R, 8, 11)[1]
        frames = synth.Video(w.video).frames(0, 3)[:, :48, :64]
        pins.test_definitional_equals_indexed_tiny_workload((R, KP, frames, oracle.Index(R, KP)))

    checks += [alpha_one, modes_agree, modes_agree_on_a_chain,
               lambda: rpins.test_identity_field_reproduces_frame(23, 17, 3),
               lambda: rpins.test_matches_scatter_formulation(13, 29, 1, 50),
               rpins.test_constant_references_closed_form, rpins.test_golden_two_patches_round_half_up,
               rpins.test_invalid_field_contributes_nothing,
               apins.test_philox_known_answers, apins.test_alpha_one_is_exact_nn,
               apins.test_full_tables_are_sorted_distance_rows, apins.test_random_field_definition_and_range,
               apins.test_ties_at_the_minimum_go_to_the_lowest_index,
               lambda: apins.test_exact_previous_match_is_kept((1, 4), 20), apins.test_no_loop_is_first_ring_argmin,
               apins.test_identical_references_stop_at_the_ring_cap, apins.test_golden_candidate_set_of_exactly_L,
               lambda: apins.test_matches_independent_implementation((1, 4), 3),
               lambda: apins.test_matches_independent_implementation((1, 2), 5),
               lambda: kpins.test_frame0_is_sorted_brute_force(300, 1, 12, 20, 8),
               lambda: kpins.test_frame0_is_sorted_brute_force(5, 1, 9, 9, 8),
               lambda: kpins.test_k1_is_the_argmin_step((1, 2), 40),
               lambda: kpins.test_k1_is_the_argmin_step((0, 1), -1),
               lambda: kpins.test_k1_is_the_argmin_step((1, 1), 0),
               kpins.test_routed_queries_are_sorted_brute_force, kpins.test_alpha_one_prefix_is_exact_knn,
               kpins.test_routing_at_the_limit_follows_the_argmin_step,
               lambda: kpins.test_matches_set_assembled_from_the_ring_predicate((1, 2)),
               kpins.test_lists_are_sorted_unique_and_padded,
               *[lambda n=n: kpins.test_golden_fixture(n) for n in kpins.GOLDEN],
               *[lambda n=n: cpins.test_golden_fixture(n) for n in cpins.GOLDEN],
               lambda: cpins.test_partition_sizes_and_medians(1000, 64, 16, 0),
               lambda: cpins.test_partition_sizes_and_medians(64, 64, 64, 2),
               cpins.test_few_patches_one_cluster, cpins.test_identical_patches_do_not_split,
               cpins.test_two_separated_groups, cpins.test_single_varying_coordinate_gives_value_ranges,
               cpins.test_split_on_largest_variance, cpins.test_tied_variance_splits_lowest_coordinate,
               cpins.test_all_at_or_below_the_median_splits_strictly,
               upins.test_normalisation_matches_float64, lambda: upins.test_distance_matches_float64(64),
               upins.test_ring_predicate_on_exact_values,
               lambda: upins.test_scale_invariance_bit_exact((1, 4), -1),
               lambda: upins.test_frame0_is_float_brute_force(1), upins.test_wide_rings_reduce_to_brute_force,
               upins.test_alpha_one_is_near_exact_nn,
               lambda: upins.test_exact_previous_match_is_kept((1, 4), -1),
               upins.test_ring_limit_zero_routes_every_nonempty_ring,
               *[lambda c=c: upins.test_golden_16_pixel_sets(c)
                 for c in ("limit_-1", "limit_5", "limit_6", "zero_query_limit_-1")]]
    for c in checks:
        try:
            c()
        except AssertionError:
            return True
    return False


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site of {name} not found"
    mutated = src.replace(old, new, 1)
    c_path = tmp_path / "mutant.c"
    c_path.write_text(mutated)
    so = tmp_path / "mutant.so"
    subprocess.run(["gcc", "-std=c99", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off", "-I",
                    os.path.dirname(SRC), "-o", str(so), str(c_path), "-lm"], check=True)
    with oracle.use_library(str(so)):
        assert _pins_fail(), f"no pin caught the planted mistake {name}"


def test_unmutated_oracle_passes_the_subset():
    assert not _pins_fail()
