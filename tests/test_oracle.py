"""Pins for the CPU oracle (test infrastructure), checked against facts that
do not come from the oracle itself: library routines (scipy's k-d tree),
closed forms, published generator values, hand-worked fixtures, error bounds
and brute force in a different formulation.

Citations: problem statement (Sec. 1), Alg. 1 and Sec. 3.1 of arXiv 1701.08475;
refinement is the neighbour-of-neighbour prior art cited in Sec. 1.
"""
import os

import numpy as np
import pytest

import datagen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _is_valid_graph(ids, d, n, full=True):
    k = ids.shape[1]
    for i in range(n):
        row = ids[i]
        real = row[row >= 0]
        assert i not in real, "self loop"
        assert len(set(real.tolist())) == len(real), "duplicate id"
        if full:
            assert len(real) == k
        keys = [(float(d[i, t]), int(np.uint32(ids[i, t]))) for t in range(k)]
        assert keys == sorted(keys), "row not sorted by (d, id)"


def _load_golden(name):
    """Fixture format: lines 'i: id:d id:d ...' after a header of '#' lines and 'X' rows."""
    X, rows = [], {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("x "):
                X.append([float(v) for v in line[2:].split()])
            else:
                i, rest = line.split(":", 1)
                rows[int(i)] = [(int(a), float(b)) for a, b in (t.split("/") for t in rest.split())]
    return np.array(X, np.float32), rows


# ---------------------------------------------------------------- generator
def test_splitmix64_published_values():
    # SplitMix64 with seed 0 (Steele, Lea & Flood 2014): first three outputs.
    assert oracle.splitmix64(0) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4
    assert oracle.splitmix64((2 * 0x9E3779B97F4A7C15) % 2**64) == 0x06C45D188009454F


def test_init_positions_distinct_and_in_range():
    ps = oracle.pass_seed(1234, 0)
    for m in (2, 3, 5, 64, 1000):
        for seg in range(20):
            h, h2 = oracle.init_positions(ps, 3, seg, m)
            assert 0 <= h < m and 0 <= h2 < m and h != h2


def test_init_positions_depend_on_segment_level_and_seed():
    # The first position is a hash of (pass seed, level, segment): over 200
    # segments (levels, seeds) of 1,000 points it takes well over 100 values
    # (a uniform draw takes about 181 on average).
    ps = oracle.pass_seed(1234, 0)
    assert len({oracle.init_positions(ps, 3, seg, 1000)[0] for seg in range(200)}) > 150
    assert len({oracle.init_positions(ps, lev, 5, 1000)[0] for lev in range(200)}) > 150
    assert len({oracle.init_positions(oracle.pass_seed(s, 0), 3, 5, 1000)[0] for s in range(200)}) > 150
    # and the second one, given the first, varies too
    seconds = {}
    for seg in range(2000):
        h, h2 = oracle.init_positions(ps, 3, seg, 50)
        seconds.setdefault(h, set()).add(h2)
    assert max(len(v) for v in seconds.values()) > 10


# ---------------------------------------------------------------- distances
def test_dist_symmetric_bitwise():
    rng = np.random.default_rng(0)
    for D in (1, 7, 32, 129):
        for _ in range(20):
            x = rng.standard_normal(D).astype(np.float32) * 10
            y = rng.standard_normal(D).astype(np.float32) * 10
            assert np.float32(oracle.dist_f32(x, y)).tobytes() == np.float32(oracle.dist_f32(y, x)).tobytes()
            assert oracle.dist_f32(x, x) == 0.0


def test_dist_f32_within_rounding_bound():
    # Each difference rounds once (relative error u = 2^-24) and each of the D
    # fused adds rounds once: |d32 - d| <= ((D + 2) u + O(u^2)) d  (Higham, Ch. 3).
    rng = np.random.default_rng(1)
    u = 2.0 ** -24
    for D in (3, 32, 128, 960):
        for _ in range(10):
            x = rng.standard_normal(D).astype(np.float32)
            y = rng.standard_normal(D).astype(np.float32)
            exact = float(np.sum((x.astype(np.float64) - y.astype(np.float64)) ** 2))
            assert abs(oracle.dist_f32(x, y) - exact) <= (D + 3) * u * exact
            assert abs(oracle.dist_f64(x, y) - exact) <= 1e-12 * exact


def test_dist_integer_data_is_exact():
    # Integers 0..255 in D = 128: every partial sum is an integer < 2^24, so the
    # canonical FP32 distance equals the exact integer sum of squares.
    X = datagen.sift_like(200, seed=3)
    Xi = X.astype(np.int64)
    for i in range(0, 200, 7):
        for j in range(0, 200, 11):
            assert oracle.dist_f32(X[i], X[j]) == float(np.sum((Xi[i] - Xi[j]) ** 2))


# ---------------------------------------------------------------- bounded lists
def test_list_insert_is_topk_of_unique_union():
    rng = np.random.default_rng(2)
    for trial in range(50):
        k = int(rng.integers(1, 12))
        pool_d = rng.integers(0, 6, size=40).astype(np.float32)   # many equal d
        ids, d = oracle.new_graph(1, k)
        offered = {}
        for _ in range(int(rng.integers(0, 80))):
            cid = int(rng.integers(-1, 40))
            if cid < 0:
                oracle.list_insert(ids[0], d[0], 0.0, cid)   # empty-slot id is ignored
                continue
            offered[cid] = float(pool_d[cid])
            oracle.list_insert(ids[0], d[0], pool_d[cid], cid)
        want = sorted((dd, i) for i, dd in offered.items())[:k]
        got = [(float(d[0, t]), int(ids[0, t])) for t in range(k) if ids[0, t] >= 0]
        assert got == want
        assert all(ids[0, t] == -1 and np.isinf(d[0, t]) for t in range(len(want), k))


# ---------------------------------------------------------------- exact graph
def test_exact_matches_scipy_kdtree():
    scipy_spatial = pytest.importorskip("scipy.spatial")
    rng = np.random.default_rng(4)
    X = rng.standard_normal((1500, 8)).astype(np.float32)
    k = 10
    ids64, d64 = oracle.exact_f64(X, k)
    ids32, d32 = oracle.exact_f32(X, k)
    tree = scipy_spatial.cKDTree(X.astype(np.float64))
    dd, jj = tree.query(X.astype(np.float64), k=k + 1)
    assert np.array_equal(jj[:, 0], np.arange(1500))        # self first (continuous data)
    assert np.array_equal(ids64, jj[:, 1:])
    assert np.allclose(d64, dd[:, 1:] ** 2, rtol=1e-12, atol=0)
    assert np.array_equal(ids32, ids64)
    assert np.allclose(d32, d64, rtol=1e-5, atol=0)


def test_exact_sample_rows_equal_full_rows():
    X = datagen.gaussian_mixture(600, 16, 10, seed=5)
    ids, d = oracle.exact_f32(X, 7)
    smp = datagen.sample_rows(600, 50, seed=1)
    sids, sd = oracle.exact_f32(X, 7, smp)
    assert np.array_equal(sids, ids[smp]) and np.array_equal(sd, d[smp])


def test_exact_one_dimension_is_sorted_window():
    # In 1-D the k nearest of a point are the k closest of its sorted neighbours,
    # taken by a two-pointer walk outward (distinct values, no ties here).
    rng = np.random.default_rng(6)
    vals = rng.permutation(np.arange(300) * 3 + rng.integers(0, 2, 300)).astype(np.float32)
    # make gaps distinct so no two distances tie
    vals = (vals * 1.0 + np.arange(300, dtype=np.float32) * 1e-3).astype(np.float32)
    X = vals[:, None]
    k = 6
    ids, _ = oracle.exact_f64(X, k)
    order = np.argsort(vals, kind="stable")
    rank = np.empty(300, int)
    rank[order] = np.arange(300)
    for i in range(300):
        lo, hi, got = rank[i] - 1, rank[i] + 1, []
        while len(got) < k:
            dl = vals[i] - vals[order[lo]] if lo >= 0 else np.inf
            dh = vals[order[hi]] - vals[i] if hi < 300 else np.inf
            if dl <= dh:
                got.append(order[lo]); lo -= 1
            else:
                got.append(order[hi]); hi += 1
        assert set(got) == set(ids[i].tolist())


@pytest.mark.parametrize("name", ["tiny_1d_k2.txt", "square_ties_k2.txt"])
def test_exact_golden_hand_worked(name):
    X, rows = _load_golden(name)
    k = len(next(iter(rows.values())))
    ids, d = oracle.exact_f32(X, k)
    for i, want in rows.items():
        assert [(int(a), float(b)) for a, b in zip(ids[i], d[i])] == want


def test_exact_integer_ties_broken_by_id():
    # Integer data with many equal distances: the list must be exactly the first
    # k of all (d, j) pairs sorted lexicographically (exact int64 distances).
    rng = np.random.default_rng(7)
    X = rng.integers(0, 3, size=(120, 4)).astype(np.float32)
    Xi = X.astype(np.int64)
    k = 9
    ids, d = oracle.exact_f32(X, k)
    for i in range(120):
        dd = ((Xi - Xi[i]) ** 2).sum(1)
        pairs = sorted((int(dd[j]), j) for j in range(120) if j != i)[:k]
        assert [(int(a), float(b)) for a, b in zip(ids[i], d[i])] == [(j, float(v)) for v, j in pairs]


# ---------------------------------------------------------------- partition
def test_tree_depth_closed_form():
    for n, lm in [(10_000, 64), (1_000_000, 128), (1_000_000, 256), (10_000_000, 128), (50, 64), (65, 64)]:
        L = oracle.tree_depth(n, lm)
        assert -(-n // (1 << L)) <= lm
        assert L == 0 or -(-n // (1 << (L - 1))) > lm
    assert oracle.tree_depth(1_000_000, 128) == 13
    assert oracle.tree_depth(10_000, 64) == 8


@pytest.mark.parametrize("n,D,lm", [(1000, 5, 64), (777, 3, 40), (64, 4, 64), (300, 1, 10)])
def test_partition_invariants(n, D, lm):
    X = datagen.gaussian_mixture(n, D, 7, seed=n)
    perm, off = oracle.partition(X, lm, iters=3, seed=9)
    L = oracle.tree_depth(n, lm)
    assert len(off) == (1 << L) + 1 and off[0] == 0 and off[-1] == n
    assert np.array_equal(np.sort(perm), np.arange(n))
    sizes = np.diff(off)
    assert set(sizes.tolist()) <= {n >> L, -(-n // (1 << L))}
    assert sizes.max() <= lm
    for a, b in zip(off[:-1], off[1:]):
        assert np.all(np.diff(perm[a:b]) > 0)


def test_partition_of_points_on_a_line_is_contiguous_runs():
    # Points t * v on a line: x . (c1 - c0) is monotone in t, so every balanced
    # cut splits the sorted order, and every leaf is a run of consecutive t.
    rng = np.random.default_rng(8)
    n = 1000
    t = rng.permutation(n).astype(np.float32)
    v = np.array([1.0, 2.0, -1.0, 0.5], np.float32)
    X = t[:, None] * v[None, :]
    perm, off = oracle.partition(X, 40, iters=4, seed=3)
    for a, b in zip(off[:-1], off[1:]):
        ts = np.sort(t[perm[a:b]])
        assert np.all(np.diff(ts) == 1.0)


def test_partition_of_identical_points_is_by_ascending_id():
    # Every point the same: every projection is the same key, so each balanced
    # cut takes the floor(m/2) smallest ids of its segment (ties by position,
    # positions ascending ids): the leaves are consecutive id ranges in order,
    # and the permutation is the identity.
    for n, leaf_max in ((1000, 40), (777, 64), (64, 2)):
        X = np.full((n, 3), 2.5, np.float32)
        perm, off = oracle.partition(X, leaf_max, iters=3, seed=9)
        assert np.array_equal(perm, np.arange(n, dtype=np.int32))
        L = oracle.tree_depth(n, leaf_max)
        sizes = np.diff(off)
        assert sizes.min() >= n // (1 << L) and sizes.max() <= -(-n // (1 << L))


def _offset_pairs_data():
    """2,051 points in 2-D, ids shuffled: b = -1 (825 points), 0 (400), +1
    (826); a = B = 1023 + 37/1024 except that 724 of the b = -1 points carry
    B +- 1/2 and every b = 0 point B +- 2^-10, + and - alternating in id
    order.  Every a is an FP32 number and every sum below is exact in FP64;
    1025 B and 1026 B are not FP32 numbers."""
    m, n_neg, n_neg_b, n0 = 2051, 825, 101, 400
    rng = np.random.default_rng(31)
    b = np.array([-1.0] * n_neg + [0.0] * n0 + [1.0] * (m - n_neg - n0), np.float32)
    rng.shuffle(b)
    B = np.float32(1023 + 37 / 1024)
    a = np.full(m, B, np.float32)
    alt = np.flatnonzero(b == -1)[:n_neg - n_neg_b]
    a[alt[0::2]] = B + np.float32(0.5)
    a[alt[1::2]] = B - np.float32(0.5)
    zeros = np.flatnonzero(b == 0)
    a[zeros[0::2]] = B + np.float32(2.0 ** -10)
    a[zeros[1::2]] = B - np.float32(2.0 ** -10)
    return np.stack([a, b], 1), a, b, zeros


def test_partition_centroids_are_fp64_means_rounded_to_fp32():
    # With a pass seed whose initial points are a b = -1 and a b = +1 point of
    # equal a, the first cut is by b: all b = -1 points, then the b = 0 points
    # by ascending id up to floor(m/2) = 1025.  Both sides then have the exact
    # mean B in a (the +- pairs cancel), so the FP64 means rounded to FP32 are
    # equal, the projection ignores a, every b = 0 point ties and the same cut
    # repeats: a closed form.  Means that are not the FP64 mean rounded once
    # (sums accumulated in FP32, or the sum rounded to FP32 before the division)
    # differ in a between the sides (by construction of B, 1025 and 1026), and
    # the cut inside the b = 0 points then follows a, not the ids.
    X, a, b, zeros = _offset_pairs_data()
    m = X.shape[0]
    K = m // 2
    seed = next(s for s in range(3000)
                for h, h2 in [oracle.init_positions(oracle.pass_seed(s, 0), 0, 0, m)]
                if b[h] == -1 and b[h2] == 1 and a[h] == a[h2])
    perm, off = oracle.partition(X, K + 1, iters=3, seed=seed)
    left = np.sort(np.concatenate([np.flatnonzero(b == -1), zeros[:K - 825]]))
    assert np.array_equal(off, [0, K, m])
    assert np.array_equal(perm[:K], left)
    assert np.array_equal(perm[K:], np.setdiff1d(np.arange(m), left))


def test_partition_orientation_one_dimension():
    # With no Lloyd iteration the cut is by x . (c1 - c0) with c0, c1 the points
    # at positions h, h2: in 1-D the left half is the smaller values exactly
    # when x_h < x_h2 (points closer to c0 go left).
    rng = np.random.default_rng(21)
    n = 200
    vals = rng.permutation(n).astype(np.float32)
    X = vals[:, None]
    for seed in range(10):
        perm, off = oracle.partition(X, n // 2, iters=0, seed=seed)
        h, h2 = oracle.init_positions(oracle.pass_seed(seed, 0), 0, 0, n)
        left = np.sort(vals[perm[off[0]:off[1]]])
        small = np.arange(n // 2, dtype=np.float32)
        if vals[h] < vals[h2]:
            assert np.array_equal(left, small)
        else:
            assert np.array_equal(left, small + n // 2)


def test_partition_separates_two_far_clusters():
    # Two equal-size clusters far apart: the first balanced 2-means split
    # must cut exactly along the clusters.
    rng = np.random.default_rng(9)
    m = 200
    A = rng.standard_normal((m, 6)).astype(np.float32)
    B = rng.standard_normal((m, 6)).astype(np.float32) + np.float32(50.0)
    X = np.empty((2 * m, 6), np.float32)
    lab = rng.permutation(np.r_[np.zeros(m, int), np.ones(m, int)])
    X[lab == 0], X[lab == 1] = A, B
    for seed in range(8):
        perm, off = oracle.partition(X, m, iters=3, seed=seed)   # depth 1: one split
        assert len(off) == 3
        left = lab[perm[off[0]:off[1]]]
        assert len(set(left.tolist())) == 1


def test_partition_split_is_lloyd_fixed_point():
    # After many Lloyd iterations on clustered data, the final balanced cut is
    # consistent with its own sides: the projection on mean(right) - mean(left)
    # (FP64, numpy) orders every left point before every right point.
    X = datagen.gaussian_mixture(600, 10, 2, seed=11, lo=-3, hi=3)
    perm, off = oracle.partition(X, 300, iters=30, seed=2)
    Lm = X[perm[off[0]:off[1]]].astype(np.float64)
    Rm = X[perm[off[1]:off[2]]].astype(np.float64)
    w = Rm.mean(0) - Lm.mean(0)
    assert (Lm @ w).max() <= (Rm @ w).min() + 1e-4 * np.abs(Rm @ w).max()


def test_partition_depends_on_pass_seed_only_through_init():
    X = datagen.gaussian_mixture(2000, 8, 20, seed=12)
    p0, _ = oracle.partition(X, 64, seed=5, pass_=0)
    p0b, _ = oracle.partition(X, 64, seed=5, pass_=0)
    p1, _ = oracle.partition(X, 64, seed=5, pass_=1)
    assert np.array_equal(p0, p0b)
    assert not np.array_equal(p0, p1)


# ---------------------------------------------------------------- leaf stage
def test_one_leaf_build_is_exact_graph():
    # leaf_max >= n: a single cluster, Alg. 1 compares every pair: the exact graph.
    X = datagen.gaussian_mixture(300, 12, 5, seed=13)
    ids, d = oracle.build_graph(X, 8, leaf_max=300, passes=1, rounds=0)
    eids, ed = oracle.exact_f32(X, 8)
    assert np.array_equal(ids, eids) and np.array_equal(d, ed)


def test_leaf_update_is_exact_within_each_leaf():
    X = datagen.gaussian_mixture(900, 6, 9, seed=14)
    k = 5
    perm, off = oracle.partition(X, 64, seed=1)
    ids, d = oracle.leaf_update(X, k, perm, off)
    for a, b in zip(off[:-1], off[1:]):
        members = perm[a:b]
        sub_ids, sub_d = oracle.exact_f32(X[members], k)
        assert np.array_equal(ids[members], members[sub_ids]) and np.array_equal(d[members], sub_d)


def test_leaf_update_merges_with_previous_lists():
    X = datagen.gaussian_mixture(500, 5, 6, seed=15)
    k = 6
    g = oracle.new_graph(500, k)
    for p in range(3):
        perm, off = oracle.partition(X, 40, seed=2, pass_=p)
        prev = g
        g = oracle.leaf_update(X, k, perm, off, *g)
        # every row only improves: elementwise (d, id) keys never increase
        for i in range(0, 500, 13):
            old = [(float(a), int(np.uint32(b))) for a, b in zip(prev[1][i], prev[0][i])]
            new = [(float(a), int(np.uint32(b))) for a, b in zip(g[1][i], g[0][i])]
            assert all(nv <= ov for nv, ov in zip(new, old))
    _is_valid_graph(*g, 500)


# ---------------------------------------------------------------- refinement
def _brute_refine(X, ids, d, mode):
    """Pull formulation: P[u] = union over i with u in N_i of N_i - {u}."""
    n, k = ids.shape
    rev = [[] for _ in range(n)]
    for j in range(n):
        for t in range(k):
            if ids[j, t] >= 0:
                rev[ids[j, t]].append((float(d[j, t]), j))
    R = [sorted(r)[:k] for r in rev]
    N = []
    for i in range(n):
        s = [int(v) for v in ids[i] if v >= 0]
        if mode == oracle.FWD_REV:
            s += [j for _, j in R[i]]
        N.append(s)
    members_of = [set() for _ in range(n)]
    for i in range(n):
        for u in N[i]:
            members_of[u].add(i)
    out_ids, out_d = oracle.new_graph(n, k)
    for u in range(n):
        cand = {int(v): float(dd) for v, dd in zip(ids[u], d[u]) if v >= 0}
        for i in members_of[u]:
            for v in N[i]:
                if v != u:
                    cand[v] = oracle.dist_f32(X[u], X[v])
        best = sorted((dd, v) for v, dd in cand.items())[:k]
        for t, (dd, v) in enumerate(best):
            out_ids[u, t], out_d[u, t] = v, dd
    return out_ids, out_d


def _random_graph(X, k, seed):
    n = X.shape[0]
    rng = np.random.default_rng(seed)
    ids, d = oracle.new_graph(n, k)
    for i in range(n):
        for j in rng.choice(np.delete(np.arange(n), i), size=k, replace=False):
            oracle.list_insert(ids[i], d[i], oracle.dist_f32(X[i], X[j]), j)
    return ids, d


@pytest.mark.parametrize("mode", [oracle.FWD, oracle.FWD_REV])
def test_refine_round_matches_pull_formulation(mode):
    # Start from a random graph: one tree pass would leave closed leaf cliques
    # on which a round is a no-op and proves nothing.
    X = datagen.gaussian_mixture(160, 4, 6, seed=16)
    k = 5
    g = _random_graph(X, k, seed=4)
    got = oracle.refine_round(X, *g, mode=mode)
    assert not np.array_equal(got[0], g[0])
    want = _brute_refine(X, *g, mode)
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])


def test_reverse_lists_match_brute_force():
    X = datagen.gaussian_mixture(200, 4, 5, seed=17)
    ids, d = oracle.build_graph(X, 6, 24, passes=1, rounds=0)
    rid, rd = oracle.reverse_lists(ids, d)
    for i in range(200):
        want = sorted((float(d[j, t]), j) for j in range(200) for t in range(6) if ids[j, t] == i)[:6]
        got = [(float(a), int(b)) for a, b in zip(rd[i], rid[i]) if b >= 0]
        assert got == want


def test_refinement_never_worsens_and_raises_recall():
    # One pass with leaves this small leaves disjoint cliques that refinement
    # cannot leave; three passes overlap them and the rounds then climb.
    X = datagen.gaussian_mixture(400, 6, 8, seed=18)
    k = 8
    g = oracle.build_graph(X, k, 20, passes=3, rounds=0)
    eids, ed = oracle.exact_f32(X, k)
    r0 = (g[0] == eids).mean()
    for _ in range(6):
        prev = g
        g = oracle.refine_round(X, *g, mode=oracle.FWD_REV)
        assert np.all(g[1] <= prev[1])
    r6 = (g[0] == eids).mean()
    assert r0 < 0.6 and r6 > 0.9


def test_single_pass_small_leaves_are_closed_cliques():
    # With one pass and k close to the leaf size every list stays inside its
    # leaf, so a refinement round finds nothing new (a property of the method).
    X = datagen.gaussian_mixture(400, 6, 8, seed=18)
    perm, off = oracle.partition(X, 20, seed=0)
    g = oracle.leaf_update(X, 11, perm, off)
    g2 = oracle.refine_round(X, *g, mode=oracle.FWD_REV)
    assert np.array_equal(g[0], g2[0])


# ---------------------------------------------------------------- build, recall
def test_build_invariants_and_recall_small_gmm():
    X = datagen.gaussian_mixture(3000, 32, 50, seed=19)
    k = 10
    ids, d = oracle.build_graph(X, k, 64, passes=2, rounds=2, mode=oracle.FWD_REV, seed=7)
    _is_valid_graph(ids, d, 3000, full=True)
    smp = datagen.sample_rows(3000, 300, seed=2)
    gi, gd = oracle.exact_f32(X, k, smp)
    ri, rt = oracle.recall(ids, d, gi, gd, smp)
    assert 0.97 <= ri <= rt <= 1.0
    # one pass: every list lies inside its leaf, so the rounds change nothing
    g1 = oracle.build_graph(X, k, 64, passes=1, rounds=0, seed=7)
    g1r = oracle.build_graph(X, k, 64, passes=1, rounds=2, seed=7)
    assert np.array_equal(g1[0], g1r[0]) and np.array_equal(g1[1], g1r[1])
    # stored distances are the canonical distances of the listed pairs
    for i in range(0, 3000, 97):
        for t in range(k):
            assert d[i, t] == oracle.dist_f32(X[i], X[ids[i, t]])


@pytest.mark.parametrize("mode", [oracle.FWD, oracle.FWD_REV])
def test_build_is_its_passes_then_its_rounds(mode):
    # Alg. 1's loop: pass p partitions with the pass-p seed and updates G from
    # its leaves, passes 0 .. I_0 - 1 in order; then the refinement rounds, each
    # from the previous one's graph.  The whole build equals that composition of
    # the stages pinned above.
    X = datagen.gaussian_mixture(1200, 8, 12, seed=23)
    k, leaf_max, passes, rounds = 6, 32, 3, 2
    ids, d = oracle.new_graph(1200, k)
    for p in range(passes):
        perm, off = oracle.partition(X, leaf_max, iters=4, seed=5, pass_=p)
        ids, d = oracle.leaf_update(X, k, perm, off, ids, d)
    for _ in range(rounds):
        ids, d = oracle.refine_round(X, ids, d, mode=mode)
    bi, bd = oracle.build_graph(X, k, leaf_max, passes=passes, rounds=rounds, iters=4, mode=mode, seed=5)
    assert np.array_equal(bi, ids) and np.array_equal(bd, d)
    # and the rounds change the graph here (two passes overlap the leaves)
    pi, _ = oracle.build_graph(X, k, leaf_max, passes=passes, rounds=rounds - 1, iters=4, mode=mode, seed=5)
    assert not np.array_equal(pi, bi)


def test_tree_pass_beats_random_partition():
    # The two-means partition puts true neighbours together far more often than
    # a random partition with the same leaf sizes (Sec. 3.1's motivation).
    X = datagen.gaussian_mixture(4000, 16, 40, seed=20)
    k = 10
    perm, off = oracle.partition(X, 64, seed=1)
    g_tree = oracle.leaf_update(X, k, perm, off)
    rperm = np.random.default_rng(0).permutation(4000).astype(np.int32)
    rperm_sorted = np.concatenate([np.sort(rperm[a:b]) for a, b in zip(off[:-1], off[1:])])
    g_rand = oracle.leaf_update(X, k, rperm_sorted, off)
    smp = datagen.sample_rows(4000, 400, seed=3)
    gi, gd = oracle.exact_f32(X, k, smp)
    r_tree, _ = oracle.recall(*g_tree, gi, gd, smp)
    r_rand, _ = oracle.recall(*g_rand, gi, gd, smp)
    assert r_tree > 0.5 and r_rand < 0.1


def test_recall_hand_example():
    ids = np.array([[1, 2], [0, 2], [0, 1]], np.int32)
    d = np.array([[1, 4], [1, 1], [4, 1]], np.float32)
    gt_ids = np.array([[1, 2], [2, 0]], np.int32)
    gt_d = np.array([[1, 4], [1, 1]], np.float32)
    ri, rt = oracle.recall(ids, d, gt_ids, gt_d, np.array([0, 1], np.int32))
    assert ri == 1.0 and rt == 1.0
    ids2 = np.array([[1, -1], [0, 2], [0, 1]], np.int32)
    d2 = np.array([[1, np.inf], [1, 1], [4, 1]], np.float32)
    ri, rt = oracle.recall(ids2, d2, gt_ids, gt_d, np.array([0, 1], np.int32))
    assert ri == 0.75 and rt == 0.75
    # a sample that skips a row: ground-truth row r belongs to graph row sample[r]
    gt3_ids = np.array([[0, 1]], np.int32)       # row 2's exact neighbours
    gt3_d = np.array([[1, 4]], np.float32)
    ids3 = np.array([[1, 2], [0, 2], [1, 0]], np.int32)
    d3 = np.array([[1, 4], [1, 1], [4, 1]], np.float32)
    ri, rt = oracle.recall(ids3, d3, gt3_ids, gt3_d, np.array([2], np.int32))
    assert ri == 1.0 and rt == 1.0
    # the same ground truth given as row 0's: row 0 holds 1 and 2, one of the two
    ri, rt = oracle.recall(ids3, d3, gt3_ids, gt3_d, np.array([0], np.int32))
    assert ri == 0.5
