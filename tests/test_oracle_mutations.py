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
    T.test_tree_depth_closed_form,
    lambda: T.test_partition_invariants(777, 3, 40),
    T.test_partition_of_points_on_a_line_is_contiguous_runs,
    T.test_partition_orientation_one_dimension,
    T.test_partition_separates_two_far_clusters,
    T.test_partition_split_is_lloyd_fixed_point,
    T.test_one_leaf_build_is_exact_graph,
    T.test_leaf_update_is_exact_within_each_leaf,
    lambda: T.test_refine_round_matches_pull_formulation(oracle.FWD),
    lambda: T.test_refine_round_matches_pull_formulation(oracle.FWD_REV),
    T.test_reverse_lists_match_brute_force,
    T.test_recall_hand_example,
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
