"""Plant plausible mistakes in a copy of the oracle (CPU only) and check that
at least one pin of tests/test_oracle.py fails for each: the pins are strong
enough to catch a dropped term, a wrong sign, a wrong index or a wrong bound
anywhere in the oracle."""
import numpy as np
import pytest

import oracle
from tests import test_oracle as T

PINS = [
    T.test_splitmix64_published_values,
    T.test_init_positions_distinct_and_in_range,
    T.test_dist_symmetric_bitwise,
    T.test_dist_f32_within_rounding_bound,
    T.test_list_insert_is_topk_of_unique_union,
    T.test_exact_matches_scipy_kdtree,
    lambda: T.test_exact_golden_hand_worked("square_ties_k2.txt"),
    lambda: T.test_exact_golden_hand_worked("tiny_1d_k2.txt"),
    T.test_exact_integer_ties_broken_by_id,
    T.test_exact_sample_rows_equal_full_rows,
    T.test_tree_depth_closed_form,
    lambda: T.test_partition_invariants(777, 3, 40),
    T.test_partition_of_points_on_a_line_is_contiguous_runs,
    T.test_partition_orientation_one_dimension,
    T.test_partition_separates_two_far_clusters,
    T.test_partition_split_is_lloyd_fixed_point,
    T.test_partition_of_identical_points_is_by_ascending_id,
    T.test_partition_centroids_are_fp64_means_rounded_to_fp32,
    T.test_init_positions_depend_on_segment_level_and_seed,
    T.test_one_leaf_build_is_exact_graph,
    T.test_leaf_update_is_exact_within_each_leaf,
    lambda: T.test_refine_round_matches_pull_formulation(oracle.FWD),
    lambda: T.test_refine_round_matches_pull_formulation(oracle.FWD_REV),
    T.test_reverse_lists_match_brute_force,
    T.test_recall_hand_example,
    T.test_partition_depends_on_pass_seed_only_through_init,
    lambda: T.test_build_is_its_passes_then_its_rounds(oracle.FWD_REV),
]

# (name, text in the oracle source, planted replacement)
MUTATIONS = [
    ("splitmix constant", "0xBF58476D1CE4E5B9ull", "0xBF58476D1CE4E5B8ull"),
    ("dist drops first dim", "for (int j = 0; j < D; ++j) {\n        float t", "for (int j = 1; j < D; ++j) {\n        float t"),
    ("dist plain square of sum", "acc = fmaf(t, t, acc);", "acc = fmaf(t, 1.0f, acc);"),
    ("tie order reversed", "return (uint32_t)ia < (uint32_t)ib;\n}\n\nstatic void list_clear",
     "return (uint32_t)ia > (uint32_t)ib;\n}\n\nstatic void list_clear"),
    ("list keeps duplicates", "if (ids[t] == cid) return;", "if (ids[t] == cid && 0) return;"),
    ("exact includes self", "if (j == i) continue;\n            orc_list_insert", "orc_list_insert"),
    ("depth off by one", "while ((n + ((int64_t)1 << L) - 1) / ((int64_t)1 << L) > leaf_max) ++L;",
     "while ((n + ((int64_t)1 << L) - 1) / ((int64_t)1 << L) > leaf_max) ++L;\n    ++L;"),
    ("projection sign", "w[j] = c1[j] - c0[j];", "w[j] = c0[j] - c1[j];"),
    ("cut at ceil", "int64_t K = m / 2, h, h2;", "int64_t K = (m + 1) / 2, h, h2;"),
    ("right centroid not updated", "mean_of(X, D, tmp + K, m - K, acc, c1);", ""),
    ("left ids not re-sorted", "qsort(tmp, (size_t)K, sizeof(int32_t), id_cmp);", ""),
    ("leaf updates only G[i]",
     "orc_list_insert(ids + (int64_t)j * k, dists + (int64_t)j * k, k, d, i);\n            }\n        }\n    }\n    return 0;",
     "}\n        }\n    }\n    return 0;"),
    ("join skips adjacent pairs", "for (int b = a + 1; b < cnt; ++b) {", "for (int b = a + 2; b < cnt; ++b) {"),
    ("reverse list stores wrong id", "dists[j * k + t], (int32_t)j);", "dists[j * k + t], (int32_t)i);"),
    ("join ignores reverse lists", "if (rev_ids[i * k + t] >= 0) memb[cnt++] = rev_ids[i * k + t];", ""),
    ("recall tie bound strict", "if (dists[i * k + a] <= kth) ++tie;", "if (dists[i * k + a] < kth) ++tie;"),
    ("centroid sums in FP32", "for (int j = 0; j < D; ++j) acc[j] += (double)X[(int64_t)ids[t] * D + j];",
     "for (int j = 0; j < D; ++j) acc[j] = (double)((float)acc[j] + X[(int64_t)ids[t] * D + j]);"),
    ("mean divided in FP32", "for (int j = 0; j < D; ++j) c[j] = (float)(acc[j] / (double)cnt);",
     "for (int j = 0; j < D; ++j) c[j] = (float)acc[j] / (float)cnt;"),
    ("sum rounded to FP32 before the division", "for (int j = 0; j < D; ++j) c[j] = (float)(acc[j] / (double)cnt);",
     "for (int j = 0; j < D; ++j) c[j] = (float)((float)acc[j] / (double)cnt);"),
    ("projection ties by descending id", "    return (x->id > y->id) - (x->id < y->id);\n}\n\nstatic int id_cmp",
     "    return (x->id < y->id) - (x->id > y->id);\n}\n\nstatic int id_cmp"),
    ("exact sample rows ignored", "        int64_t i = sample ? sample[r] : r;\n        int32_t *li = out_ids + r * k;\n        float *ld",
     "        int64_t i = r;\n        int32_t *li = out_ids + r * k;\n        float *ld"),
    ("recall reads graph rows by sample position", "            int32_t g = ids[i * k + a];", "            int32_t g = ids[r * k + a];"),
    ("build repeats pass 0", "        if (orc_partition(X, n, D, leaf_max, iters, seed, p, perm, off) < 0) {",
     "        if (orc_partition(X, n, D, leaf_max, iters, seed, 0, perm, off) < 0) {"),
    ("build one round fewer", "    for (int r = 0; r < rounds; ++r)\n        if (orc_refine_round",
     "    for (int r = 1; r < rounds; ++r)\n        if (orc_refine_round"),
    ("build rounds in forward mode only", "if (orc_refine_round(X, n, D, k, mode, out_ids, out_d) != 0) return -1;",
     "if (orc_refine_round(X, n, D, k, 0, out_ids, out_d) != 0) return -1;"),
    ("pass seed ignores the pass", "return orc_splitmix64(seed ^ (uint64_t)pass);", "return orc_splitmix64(seed);"),
    ("first position ignores the segment",
     "orc_splitmix64(orc_splitmix64(orc_splitmix64(pass_seed) ^ (uint64_t)level) ^ (uint64_t)seg)",
     "orc_splitmix64(orc_splitmix64(orc_splitmix64(pass_seed) ^ (uint64_t)level))"),
]


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(name, old, new, tmp_path, monkeypatch):
    src = oracle.source_text()
    assert src.count(old) == 1, "mutation anchor must occur once: " + name
    lib = oracle.compile_variant(src.replace(old, new), str(tmp_path / "mutant.so"))
    monkeypatch.setattr(oracle, "_lib", lib)
    caught = []
    for pin in PINS:
        try:
            pin()
        except Exception as e:   # an assertion or a crash-free error both count
            caught.append(getattr(pin, "__name__", "pin"))
            break
    assert caught, "no pin caught the planted mistake: " + name


# the search (Alg. 2) and the residue-quantisation index (Sec. 4)
from tests import test_oracle_rvq as V    # noqa: E402
from tests import test_oracle_search as Sr  # noqa: E402

PINS_SEARCH_RVQ = [
    Sr.test_no_iterations_rank_the_seeds,
    Sr.test_one_iteration_over_a_complete_graph_is_brute_force,
    lambda: Sr.test_path_graph_frontier_moves_one_node_per_iteration(2, 3),
    lambda: Sr.test_path_graph_frontier_moves_one_node_per_iteration(4, 40),
    Sr.test_repeated_and_out_of_range_seeds_count_once,
    Sr.test_rows_are_sorted_unique_and_carry_canonical_distances,
    lambda: Sr.test_every_top_entry_is_expanded_not_only_the_first(2, [2, 0]),
    V.test_init_positions_one_per_stratum,
    V.test_zero_iterations_give_each_stage_its_drawn_vectors,
    V.test_a_word_without_members_keeps_its_value,
    V.test_assign_is_the_brute_force_argmin_with_ties_to_the_smaller_index,
    V.test_one_iteration_from_separated_clusters_gives_their_means,
    lambda: V.test_converged_training_is_a_fixed_point_of_both_stages(0),
    V.test_quantisation_error_never_grows_over_iterations,
    V.test_one_word_per_point_and_a_single_word,
    V.test_index_is_a_stable_sort_by_key,
    lambda: V.test_seeds_follow_eqn2_with_pruning_by_the_first_term(3, 40),
    lambda: V.test_seeds_follow_eqn2_with_pruning_by_the_first_term(12, 300),
    lambda: V.test_seeds_follow_eqn2_with_pruning_by_the_first_term(12, 5000),
    V.test_seeds_tie_by_key_when_the_query_norm_absorbs_the_differences,
    V.test_seeds_on_float_data_follow_the_direct_distance_up_to_rounding,
]

MUTATIONS_SEARCH_RVQ = [
    ("search expands only the top entry", "int ntop = nr < ks ? (int)nr : ks;", "int ntop = nr < 1 ? (int)nr : 1;"),
    ("search seeds not marked visited", "visited[id] = 1;\n            R[nr].d", "R[nr].d"),
    ("search drops the last neighbour slot", "for (int e = 0; e < k; ++e) {\n                    int32_t nb",
     "for (int e = 0; e + 1 < k; ++e) {\n                    int32_t nb"),
    ("search expands the final order", "/* the ks first entries of R as it stands at the iteration's start */\n"
     "            qsort(R, (size_t)nr, sizeof(rank_t), rank_cmp);", ""),
    ("rvq ties to the larger word", "if (d < best) { best = d; bc = c; }", "if (d <= best) { best = d; bc = c; }"),
    ("rvq residue sign", "R[i * D + j] = X[i * D + j] - w1[", "R[i * D + j] = X[i * D + j] + w1["),
    ("rvq mean off by one", "/ (double)cnt[c]);", "/ (double)(cnt[c] + 1));"),
    ("rvq stage 2 trained on the points", "rc = lloyd(R, n, D, W2", "rc = lloyd(X, n, D, W2"),
    ("rvq draw outside its stratum", "pos[c] = lo + (int64_t)(h % (uint64_t)(hi - lo));",
     "pos[c] = lo + (int64_t)(h % (uint64_t)(hi - lo + 1));"),
    ("rvq term 2 cross-product sign", "fmaf(2.0f, x12[", "fmaf(-2.0f, x12["),
    ("rvq pruning without the word norm", "t1[a].d = (t + n1[a]) + 0.0f;", "t1[a].d = t + 0.0f;"),
    ("rvq lists in descending ids", "for (int64_t i = 0; i < n; ++i) ids[fill",
     "for (int64_t i = n - 1; i >= 0; --i) ids[fill"),
    ("rvq seeds skip a list's first id", "for (int32_t t = offsets[cand[e].key];",
     "for (int32_t t = offsets[cand[e].key] + 1;"),
    ("rvq empty word reset to zero", "            if (cnt[c] == 0) continue;\n",
     "            if (cnt[c] == 0) { for (int j = 0; j < D; ++j) words[(int64_t)c * D + j] = 0.0f; continue; }\n"),
    ("rvq stage 2 drawn like stage 1", "rc = lloyd(R, n, D, W2, iters, seed, 2, w2, codes);",
     "rc = lloyd(R, n, D, W2, iters, seed, 1, w2, codes);"),
    ("rvq term 1 without the query norm", "float t = fmaf(-2.0f, dot_f32(q, w1 + (int64_t)a * D, D), qq);",
     "float t = fmaf(-2.0f, dot_f32(q, w1 + (int64_t)a * D, D), 0.0f);"),
    ("rvq seeds padded with 0", "for (; cnt < s; ++cnt) S[qi * s + cnt] = -1;", "for (; cnt < s; ++cnt) S[qi * s + cnt] = 0;"),
]


@pytest.mark.parametrize("name,old,new", MUTATIONS_SEARCH_RVQ, ids=[m[0] for m in MUTATIONS_SEARCH_RVQ])
def test_planted_mistake_in_search_or_index_is_caught(name, old, new, tmp_path, monkeypatch):
    src = oracle.source_text()
    assert src.count(old) == 1, "mutation anchor must occur once: " + name
    lib = oracle.compile_variant(src.replace(old, new), str(tmp_path / "mutant.so"))
    monkeypatch.setattr(oracle, "_lib", lib)
    caught = False
    for pin in PINS_SEARCH_RVQ:
        try:
            pin()
        except Exception:
            caught = True
            break
    assert caught, "no pin caught the planted mistake: " + name


# the sampled refinement round (nearest-neighbour descent with sampling)
from tests import test_oracle_sampled as Sm  # noqa: E402

PINS_SAMPLED = [
    Sm.test_priority_is_splitmix_of_the_stated_key,
    Sm.test_no_samples_or_no_new_entries_change_nothing,
    lambda: Sm.test_unlimited_sample_joins_every_new_pair(3),
    lambda: Sm.test_limited_sample_joins_the_sampled_members(4, 2),
    Sm.test_the_sample_is_the_least_priorities,
    Sm.test_lists_only_improve_and_stay_canonical,
]

MUTATIONS_SAMPLED = [
    ("sampled entries stay new", "isnew[v * k + t] = 1;\n                flags[v * k + t] = 0;",
     "isnew[v * k + t] = 1;"),
    ("new x old pairs skipped", "for (int b = a + 1; b < cn_ + co_; ++b) {", "for (int b = a + 1; b < cn_; ++b) {"),
    ("inserted entries flagged old", "if (found < 0) { f = 1; ++changed; }", "if (found < 0) { f = 0; ++changed; }"),
    ("reverse new lists ignored", "if (!has_id(nn, cn_, buf[a])) nn[cn_++] = buf[a];", ""),
    ("sample keeps the greatest priorities", "if (x->h != y->h) return x->h < y->h ? -1 : 1;",
     "if (x->h != y->h) return x->h > y->h ? -1 : 1;"),
    ("priority ignores the round", "orc_splitmix64(seed ^ (uint64_t)(uint32_t)round)", "orc_splitmix64(seed)"),
    ("priority without the id bits", "return (h & 0xFFFFFFFF00000000ull) | (uint32_t)u;",
     "return h & 0xFFFFFFFF00000000ull;"),
    ("old members drawn from unsampled new entries",
     "if (u >= 0 && !isnew[v * k + t] && !flags[v * k + t] && !has_id(nn, cn_, u)) no[co_++] = u;",
     "if (u >= 0 && !isnew[v * k + t] && !has_id(nn, cn_, u)) no[co_++] = u;"),
]


@pytest.mark.parametrize("name,old,new", MUTATIONS_SAMPLED, ids=[m[0] for m in MUTATIONS_SAMPLED])
def test_planted_mistake_in_the_sampled_round_is_caught(name, old, new, tmp_path, monkeypatch):
    src = oracle.source_text()
    assert src.count(old) == 1, "mutation anchor must occur once: " + name
    lib = oracle.compile_variant(src.replace(old, new), str(tmp_path / "mutant.so"))
    monkeypatch.setattr(oracle, "_lib", lib)
    caught = False
    for pin in PINS_SAMPLED:
        try:
            pin()
        except Exception:
            caught = True
            break
    assert caught, "no pin caught the planted mistake: " + name
