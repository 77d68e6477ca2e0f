"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Bar (from the graph conventions): ids bit-exact; distances bit-exact (the
canonical FP32 distance is computed in the same order on both sides, so the
1e-5 relative bound is met with zero error).  Where floating point decides
the partition (FP64 centroid sums of non-integer data, summed in another
order), the later stages are compared on the GPU's own partition, and the
partition itself is compared on integer data, where the sums are exact.
"""
import numpy as np
import pytest

import datagen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def knng():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1701_08475_gb300 as m
    m.load()
    return m


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def _np(t):
    return t.cpu().numpy() if hasattr(t, "cpu") else np.asarray(t)


def _assert_graph_equal(g_ids, g_d, o_ids, o_d):
    g_ids, g_d = _np(g_ids), _np(g_d)
    bad = np.argwhere(g_ids != o_ids)
    assert bad.size == 0, "ids differ at %s: gpu %s oracle %s" % (
        bad[:3].tolist(), g_ids[tuple(bad[0])], o_ids[tuple(bad[0])])
    assert np.array_equal(g_d.view(np.uint32), o_d.view(np.uint32)), "distance bits differ"


def _assert_valid(ids, d, full=True):
    ids, d = _np(ids), _np(d)
    n, k = ids.shape
    assert not np.any(ids == np.arange(n)[:, None]), "self loop"
    real = ids >= 0
    if full:
        assert real.all()
    s = np.sort(np.where(real, ids, -1 - np.arange(k)[None, :]), axis=1)
    assert not np.any((s[:, 1:] == s[:, :-1]) & (s[:, 1:] >= 0)), "duplicate id"
    dd = np.where(real, d, np.inf)
    assert np.all(dd[:, 1:] >= dd[:, :-1]), "row not sorted by distance"
    tie = dd[:, 1:] == dd[:, :-1]
    ui = ids.astype(np.int64) & 0xffffffff
    assert not np.any(tie & (ui[:, 1:] < ui[:, :-1])), "equal distances not ordered by id"


# ---------------------------------------------------------------- whole build
BUILD_CASES = [
    # n, D, k, leaf_max, passes, rounds, mode, iters
    (1500, 24, 8, 40, 2, 1, oracle.FWD_REV, 3),
    (3001, 13, 10, 64, 2, 2, oracle.FWD_REV, 4),      # D not a multiple of 4, ragged n
    (2500, 32, 16, 128, 2, 1, oracle.FWD, 2),
    (4097, 8, 12, 256, 1, 1, oracle.FWD_REV, 4),      # largest leaves
    (700, 130, 5, 12, 3, 2, oracle.FWD_REV, 1),       # two dim chunks in the join
    (21, 3, 20, 42, 1, 0, oracle.FWD, 4),             # n = k + 1: one leaf, complete lists
    (900, 16, 33, 68, 1, 0, oracle.FWD, 4),           # k > 32: two list slots per lane
]


@pytest.mark.parametrize("n,D,k,lm,passes,rounds,mode,iters", BUILD_CASES)
def test_build_matches_oracle_on_integer_data(knng, n, D, k, lm, passes, rounds, mode, iters):
    X = datagen.sift_like(n, D=D, n_centres=max(2, n // 60), seed=n + D)
    p = knng.default_params(k=k, leaf_max=lm, tree_passes=passes, refine_rounds=rounds, join_mode=mode,
                            twomeans_iters=iters, seed=1234 + n)
    ids, d = knng.knng_build_ex(_dev(X), p)
    o_ids, o_d = oracle.build_graph(X, k, lm, passes=passes, rounds=rounds, iters=iters, mode=mode, seed=1234 + n)
    _assert_graph_equal(ids, d, o_ids, o_d)
    _assert_valid(ids, d)


def test_plain_build_entry_point(knng):
    X = datagen.sift_like(2000, D=16, n_centres=30, seed=3)
    ids, d = knng.knng_build(_dev(X), k=10, leaf_max=64, rounds=3, seed=99)
    o_ids, o_d = oracle.build_graph(X, 10, 64, passes=3, rounds=0, iters=4, seed=99)
    _assert_graph_equal(ids, d, o_ids, o_d)


@pytest.mark.parametrize("n,D,precision,kind", [(1200, 20, "fp32", "integer"), (1003, 7, "bf16", "integer"),
                                                 (2051, 33, "fp16", "float"), (9, 3, "fp32", "float")])
def test_host_pointers_give_the_same_graph(knng, n, D, precision, kind):
    # host rows come in eight pieces of a multiple of 4 rows (the last one
    # ragged), each checked and converted as it lands; the lists equal the
    # device-buffer build's, and a NaN in the last piece is still refused
    X = (datagen.sift_like(n, D=D, n_centres=15, seed=5) if kind == "integer"
         else datagen.gaussian_mixture(n, D, 10, seed=5))
    prec = {"fp32": knng.KNNG_FP32, "bf16": knng.KNNG_BF16, "fp16": knng.KNNG_FP16}[precision]
    p = knng.default_params(k=6, leaf_max=32, tree_passes=2, refine_rounds=1, seed=8, precision=prec)
    hi, hd = knng.knng_build_ex(X, p)                        # numpy in, numpy out
    di, dd = knng.knng_build_ex(_dev(X), p)
    assert isinstance(hi, np.ndarray)
    _assert_graph_equal(di, dd, hi, hd)
    Xp = torch.from_numpy(X).pin_memory()                    # page-locked host rows
    pi, pd = knng.knng_build_ex(Xp, p)
    _assert_graph_equal(di, dd, _np(pi), _np(pd))
    Xn = X.copy()
    Xn[-1, -1] = np.nan
    with pytest.raises(knng.KnngError):
        knng.knng_build_ex(Xn, p)


# ---------------------------------------------------------------- low precision
def _lp_data(kind, n, D, seed):
    if kind == "integer":      # exact in BF16/FP16: products and sums are exact integers
        return datagen.sift_like(n, D=D, n_centres=max(2, n // 80), seed=seed)
    if kind == "signed":       # signed integers with large norms: the certificate decides
        rng = np.random.default_rng(seed)
        return rng.integers(-250, 250, size=(n, D)).astype(np.float32)
    return datagen.gaussian_mixture(n, D, 30, seed=seed)   # float: quantised, certified re-rank


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
@pytest.mark.parametrize("kind,n,D,k,lm", [("integer", 4000, 128, 20, 128), ("float", 5000, 32, 10, 64),
                                           ("float", 3000, 200, 16, 100), ("signed", 2000, 64, 12, 60),
                                           ("integer", 1500, 24, 40, 128),
                                           ("integer", 5000, 64, 16, 256), ("float", 4000, 96, 12, 200),
                                           ("float", 3000, 320, 10, 160)])   # two 128-row tiles per leaf
def test_low_precision_build_equals_fp32(knng, precision, kind, n, D, k, lm):
    # the certified re-rank makes the BF16/FP16 leaf stage return the FP32 graph
    X = _lp_data(kind, n, D, seed=n + D)
    prec = knng.KNNG_BF16 if precision == "bf16" else knng.KNNG_FP16
    mode = oracle.FWD_REV if 2 * k <= 64 else oracle.FWD   # reverse lists need 2k <= 64
    common = dict(k=k, leaf_max=lm, tree_passes=2, refine_rounds=1, seed=9, join_mode=mode)
    lp_ids, lp_d = knng.knng_build_ex(_dev(X), knng.default_params(precision=prec, **common))
    f_ids, f_d = knng.knng_build_ex(_dev(X), knng.default_params(precision=knng.KNNG_FP32, **common))
    _assert_graph_equal(lp_ids, lp_d, _np(f_ids), _np(f_d))
    if kind == "integer":
        o_ids, o_d = oracle.build_graph(X, k, lm, passes=2, rounds=1, seed=9, mode=mode)
        _assert_graph_equal(lp_ids, lp_d, o_ids, o_d)


# ---------------------------------------------------------------- partition
@pytest.mark.parametrize("n,D,lm,iters,top", [(20000, 12, 64, 3, 255), (5000, 7, 40, 4, 255), (64, 5, 64, 4, 255),
                                               (9000, 1, 100, 2, 255), (20000, 200, 64, 3, 255),
                                               (6000, 33, 50, 4, 255), (20000, 40, 64, 3, 256),
                                               (6000, 33, 50, 4, 256)])
def test_partition_matches_oracle_on_integer_data(knng, n, D, lm, iters, top):
    # n = 20000 takes the multi-CTA selection at the top levels.  Values in
    # [0, 255] take the byte copy (D = 200: two slabs, the second ragged; D
    # not a multiple of 4: padded rows); one value of 256 sends the same data
    # to the FP32 rows
    X = datagen.sift_like(n, D=D, n_centres=50, seed=n)
    if top == 256:
        X[n // 2, D // 2] = 256.0
    perm, off = knng.knng_partition(_dev(X), lm, twomeans_iters=iters, seed=77, pass_=1)
    o_perm, o_off = oracle.partition(X, lm, iters=iters, seed=77, pass_=1)
    assert np.array_equal(_np(off), o_off)
    assert np.array_equal(_np(perm), o_perm)


def test_partition_invariants_on_float_data(knng):
    X = datagen.gaussian_mixture(30000, 20, 100, seed=4)
    perm, off = knng.knng_partition(_dev(X), 100, seed=3)
    perm, off = _np(perm), _np(off)
    L = knng.knng_tree_depth(30000, 100)
    assert len(off) == (1 << L) + 1
    assert np.array_equal(np.sort(perm), np.arange(30000))
    for a, b in zip(off[:-1], off[1:]):
        assert np.all(np.diff(perm[a:b]) > 0)
    o_perm, o_off = oracle.partition(X, 100, seed=3)
    assert np.array_equal(off, o_off)
    # FP64 sums in another order may move a few points at a cut; most leaves agree
    same = sum(np.array_equal(perm[a:b], o_perm[a:b]) for a, b in zip(off[:-1], off[1:]))
    assert same >= 0.9 * (len(off) - 1)


# ---------------------------------------------------------------- leaf stage
@pytest.mark.parametrize("n,D,k,lm", [(6000, 32, 10, 64), (3000, 37, 20, 128), (2000, 300, 8, 256)])
def test_leaf_stage_on_gpu_partition_matches_oracle(knng, n, D, k, lm):
    X = datagen.gaussian_mixture(n, D, 40, seed=D)
    perm, off = knng.knng_partition(_dev(X), lm, seed=5)
    perm_h, off_h = _np(perm), _np(off)
    o_ids, o_d = oracle.leaf_update(X, k, perm_h, off_h)
    ids0, d0 = oracle.new_graph(n, k)
    g_ids, g_d = knng.knng_leaf_update(_dev(X), k, perm, off, _dev(ids0), _dev(d0))
    _assert_graph_equal(g_ids, g_d, o_ids, o_d)
    # the build's first pass is the same computation
    p = knng.default_params(k=k, leaf_max=lm, tree_passes=1, refine_rounds=0, seed=5)
    b_ids, b_d = knng.knng_build_ex(_dev(X), p)
    _assert_graph_equal(b_ids, b_d, o_ids, o_d)


def test_leaf_update_merges_into_an_existing_graph(knng):
    X = datagen.gaussian_mixture(4000, 16, 30, seed=9)
    k = 12
    g = oracle.build_graph(X, k, 64, passes=1, rounds=0, seed=1)
    perm, off = knng.knng_partition(_dev(X), 64, seed=2, pass_=3)
    o_ids, o_d = oracle.leaf_update(X, k, _np(perm), _np(off), *g)
    g_ids, g_d = knng.knng_leaf_update(_dev(X), k, perm, off, _dev(g[0]), _dev(g[1]))
    _assert_graph_equal(g_ids, g_d, o_ids, o_d)


# ---------------------------------------------------------------- refinement
@pytest.mark.parametrize("mode", [oracle.FWD, oracle.FWD_REV])
@pytest.mark.parametrize("n,D,k", [(5000, 24, 10), (3000, 50, 16), (2000, 9, 32)])
def test_refine_round_matches_oracle(knng, mode, n, D, k):
    if mode == oracle.FWD_REV and 2 * k > 64:
        pytest.skip("reverse lists need 2k <= 64")
    X = datagen.gaussian_mixture(n, D, 25, seed=n + k)
    g = oracle.build_graph(X, k, max(64, 2 * (k + 1)), passes=2, rounds=0, seed=3)
    o_ids, o_d = oracle.refine_round(X, *g, mode=mode)
    p = knng.default_params(k=k, refine_rounds=1, join_mode=mode)
    g_ids, g_d = knng.knng_refine(_dev(X), _dev(g[0]), _dev(g[1]), p)
    _assert_graph_equal(g_ids, g_d, o_ids, o_d)


def test_refine_from_random_graph_two_rounds(knng):
    # a random start makes every round propose a lot (stress of the grouping)
    X = datagen.gaussian_mixture(1500, 12, 10, seed=21)
    k = 10
    rng = np.random.default_rng(0)
    ids, d = oracle.new_graph(1500, k)
    for i in range(1500):
        for j in rng.choice(np.delete(np.arange(1500), i), size=k, replace=False):
            oracle.list_insert(ids[i], d[i], oracle.dist_f32(X[i], X[j]), j)
    o = (ids, d)
    for _ in range(2):
        o = oracle.refine_round(X, *o, mode=oracle.FWD_REV)
    p = knng.default_params(k=k, refine_rounds=2, join_mode=knng.KNNG_JOIN_FWD_REV)
    g_ids, g_d = knng.knng_refine(_dev(X), _dev(ids), _dev(d), p)
    _assert_graph_equal(g_ids, g_d, *o)


@pytest.mark.parametrize("mode,k,start", [(oracle.FWD_REV, 8, "tree"), (oracle.FWD_REV, 20, "tree"),
                                          (oracle.FWD, 12, "tree"), (oracle.FWD, 40, "tree"),
                                          (oracle.FWD_REV, 10, "random"), (oracle.FWD, 16, "random")])
def test_refine_rounds_skipping_old_pairs_match_oracle(knng, mode, k, start):
    # rounds after the first skip pairs of two members that the previous round
    # already joined; every round must still equal the oracle's full join
    n, D = 2600, 20
    X = datagen.gaussian_mixture(n, D, 25, seed=k + 31)
    if start == "tree":
        ids, d = oracle.build_graph(X, k, max(64, 2 * (k + 1)), passes=1, rounds=0, seed=6)
    else:
        rng = np.random.default_rng(k)
        ids, d = oracle.new_graph(n, k)
        for i in range(n):
            for j in rng.choice(np.delete(np.arange(n), i), size=k, replace=False):
                oracle.list_insert(ids[i], d[i], oracle.dist_f32(X[i], X[j]), j)
    o = (ids, d)
    for _ in range(4):
        o = oracle.refine_round(X, *o, mode=mode)
    p = knng.default_params(k=k, refine_rounds=4, join_mode=mode)
    g_ids, g_d = knng.knng_refine(_dev(X), _dev(ids), _dev(d), p)
    _assert_graph_equal(g_ids, g_d, *o)


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
@pytest.mark.parametrize("k,mode,kind", [(20, oracle.FWD_REV, "integer"), (12, oracle.FWD, "integer"),
                                         (48, oracle.FWD, "integer"), (16, oracle.FWD_REV, "float"),
                                         (24, oracle.FWD, "float"),
                                         # 16 nodes of 8 member slots per tile (a warp collects two)
                                         (4, oracle.FWD_REV, "integer"), (8, oracle.FWD, "integer"),
                                         (5, oracle.FWD_REV, "integer")])
def test_low_precision_rounds_match_oracle(knng, precision, k, mode, kind):
    # the tensor-core join over four rounds (member flags from the second on):
    # exact on integer data; screening plus canonical distances on float data
    n = 3500
    X = (datagen.sift_like(n, D=96, n_centres=40, seed=k) if kind == "integer"
         else datagen.gaussian_mixture(n, 96, 40, seed=k))
    prec = knng.KNNG_BF16 if precision == "bf16" else knng.KNNG_FP16
    common = dict(k=k, leaf_max=128, tree_passes=1, refine_rounds=4, seed=3, join_mode=mode)
    lp_ids, lp_d = knng.knng_build_ex(_dev(X), knng.default_params(precision=prec, **common))
    o_ids, o_d = oracle.build_graph(X, k, 128, passes=1, rounds=4, seed=3, mode=mode)
    _assert_graph_equal(lp_ids, lp_d, o_ids, o_d)


@pytest.mark.parametrize("k", [4, 20])
def test_exact_join_three_passes_matches_oracle(knng, k):
    # the tensor-core join with three passes' leaf ids (leaf-mate offers
    # dropped), 3 and 16 nodes per tile, four rounds
    n = 6000
    X = datagen.sift_like(n, D=64, n_centres=50, seed=20 + k)
    common = dict(k=k, leaf_max=64, tree_passes=3, refine_rounds=4, seed=5, join_mode=oracle.FWD_REV)
    ids, d = knng.knng_build_ex(_dev(X), knng.default_params(precision=knng.KNNG_BF16, **common))
    o_ids, o_d = oracle.build_graph(X, k, 64, passes=3, rounds=4, seed=5, mode=oracle.FWD_REV)
    _assert_graph_equal(ids, d, o_ids, o_d)


@pytest.mark.parametrize("k", [20, 24])
def test_exact_join_overflow_slots_match_oracle(knng, k):
    # nearly uniform integer data: few mutual neighbours, so many nodes have
    # more members than the tensor-core join's smaller first-launch slot and
    # go through the second launch with full slots
    n = 4000
    X = datagen.sift_like(n, D=48, n_centres=n, seed=31 + k)
    common = dict(k=k, leaf_max=64, tree_passes=2, refine_rounds=3, seed=9, join_mode=oracle.FWD_REV)
    ids, d = knng.knng_build_ex(_dev(X), knng.default_params(precision=knng.KNNG_BF16, **common))
    o_ids, o_d = oracle.build_graph(X, k, 64, passes=2, rounds=3, seed=9, mode=oracle.FWD_REV)
    _assert_graph_equal(ids, d, o_ids, o_d)


@pytest.mark.parametrize("k,D", [(16, 40), (12, 96), (20, 64)])
def test_fp32_join_overflow_slots_match_oracle(knng, k, D):
    # the CTA-wide FP32 join (k = 16 and 12) packs nodes in slots of three
    # quarters of 2k; nearly uniform float data leaves many nodes more members
    # than that, and the second launch with full slots joins them (k = 20: the
    # warp-per-node kernel, on the same data)
    n = 4000
    X = datagen.gaussian_mixture(n, D, n, seed=41 + k)
    common = dict(k=k, leaf_max=64, tree_passes=2, refine_rounds=3, seed=13, join_mode=oracle.FWD_REV)
    ids, d = knng.knng_build_ex(_dev(X), knng.default_params(precision=knng.KNNG_FP32, **common))
    o_ids, o_d = oracle.build_graph(X, k, 64, passes=2, rounds=3, seed=13, mode=oracle.FWD_REV)
    _assert_graph_equal(ids, d, o_ids, o_d)


def test_refine_small_offer_budget_retries_chunks(knng, monkeypatch):
    # a 1 MB offer buffer: chunks sized from the offer estimate overflow and
    # are re-run smaller; the result must not change
    monkeypatch.setenv("KNNG_OFFER_BUDGET_MB", "1")
    n, k = 3000, 12
    X = datagen.gaussian_mixture(n, 16, 20, seed=5)
    rng = np.random.default_rng(2)
    ids, d = oracle.new_graph(n, k)
    for i in range(n):
        for j in rng.choice(np.delete(np.arange(n), i), size=k, replace=False):
            oracle.list_insert(ids[i], d[i], oracle.dist_f32(X[i], X[j]), j)
    o = (ids, d)
    for _ in range(3):
        o = oracle.refine_round(X, *o, mode=oracle.FWD_REV)
    p = knng.default_params(k=k, refine_rounds=3, join_mode=knng.KNNG_JOIN_FWD_REV)
    knng.stats_reset()
    knng.stats_enable(True, False)
    try:
        g_ids, g_d = knng.knng_refine(_dev(X), _dev(ids), _dev(d), p)
    finally:
        knng.stats_enable(False)
    _assert_graph_equal(g_ids, g_d, *o)
    assert knng.stats().get("k5_join_retry", {}).get("items", 0) > 0, "no chunk overflowed"


# ---------------------------------------------------------------- exact, recall
@pytest.mark.parametrize("n,D,k,s", [(3000, 32, 10, None), (5000, 37, 20, 300), (2000, 200, 50, 150),
                                     (129, 4, 3, None)])
def test_exact_matches_oracle(knng, n, D, k, s):
    X = datagen.gaussian_mixture(n, D, 20, seed=n)
    smp = None if s is None else datagen.sample_rows(n, s, seed=1)
    g_ids, g_d = knng.knng_exact(_dev(X), k, None if smp is None else _dev(smp))
    o_ids, o_d = oracle.exact_f32(X, k, smp)
    _assert_graph_equal(g_ids, g_d, o_ids, o_d)


def test_exact_integer_ties(knng):
    rng = np.random.default_rng(2)
    X = rng.integers(0, 3, size=(1000, 4)).astype(np.float32)     # heavy ties
    g_ids, g_d = knng.knng_exact(_dev(X), 15)
    o_ids, o_d = oracle.exact_f32(X, 15)
    _assert_graph_equal(g_ids, g_d, o_ids, o_d)


def test_recall_matches_oracle(knng):
    X = datagen.gaussian_mixture(4000, 16, 40, seed=31)
    k = 10
    ids, d = oracle.build_graph(X, k, 64, passes=1, rounds=0, seed=4)
    smp = datagen.sample_rows(4000, 500, seed=2)
    gi, gd = oracle.exact_f32(X, k, smp)
    want = oracle.recall(ids, d, gi, gd, smp)
    got = knng.knng_recall(_dev(ids), _dev(d), _dev(gi), _dev(gd), _dev(smp))
    assert got == want
    got_host = knng.knng_recall(ids, d, gi, gd, smp)
    assert got_host == want


# ---------------------------------------------------------------- edge cases
def test_duplicate_points_and_zero_vectors(knng):
    X = np.zeros((600, 8), np.float32)
    X[300:] = datagen.sift_like(300, D=8, n_centres=3, seed=1)[np.arange(300) % 7]   # many duplicates
    p = knng.default_params(k=9, leaf_max=32, tree_passes=2, refine_rounds=1, seed=2)
    ids, d = knng.knng_build_ex(_dev(X), p)
    o_ids, o_d = oracle.build_graph(X, 9, 32, passes=2, rounds=1, seed=2)
    _assert_graph_equal(ids, d, o_ids, o_d)


def test_non_finite_input_is_rejected(knng):
    X = datagen.gaussian_mixture(500, 8, 5, seed=1)
    X[123, 4] = np.nan
    with pytest.raises(knng.KnngError) as e:
        knng.knng_build_ex(_dev(X), knng.default_params(k=5, leaf_max=32))
    assert e.value.code == -1 and "non-finite" in str(e.value)
    X[123, 4] = np.inf
    with pytest.raises(knng.KnngError):
        knng.knng_exact(_dev(X), 5)


def test_empty_sample_and_zero_passes(knng):
    X = datagen.gaussian_mixture(300, 8, 5, seed=1)
    ids, d = knng.knng_build_ex(_dev(X), knng.default_params(k=4, tree_passes=0))
    assert np.all(_np(ids) == -1) and np.all(np.isinf(_np(d)))
    gi, gd = knng.knng_exact(_dev(X), 4, _dev(np.zeros(0, np.int32)))
    assert _np(gi).shape == (0, 4)


# ---------------------------------------------------------------- batched instances
@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_batched_build_equals_single_builds(knng, precision):
    # instances of several sizes, dims and cluster bounds in one forest build:
    # each result equals the instance built alone
    specs = [(2000, 64, 64), (5003, 64, 128), (777, 128, 40), (12000, 64, 64), (3000, 128, 128), (150, 64, 40)]
    k = 12
    datas = [datagen.gaussian_mixture(n, D, 20, seed=n + D) if i % 2 else
             datagen.sift_like(n, D=D, n_centres=30, seed=n) for i, (n, D, _) in enumerate(specs)]
    prec = {"fp32": knng.KNNG_FP32, "bf16": knng.KNNG_BF16}[precision]
    p = knng.default_params(k=k, leaf_max=64, tree_passes=2, refine_rounds=2, seed=21, precision=prec)
    outs = knng.knng_build_batched([_dev(X) for X in datas], p, leaf_maxes=[lm for _, _, lm in specs])
    for (n, D, lm), X, (ids, d) in zip(specs, datas, outs):
        q = knng.default_params(k=k, leaf_max=lm, tree_passes=2, refine_rounds=2, seed=21, precision=prec)
        ids1, d1 = knng.knng_build_ex(_dev(X), q)
        _assert_graph_equal(ids, d, _np(ids1), _np(d1))


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_batched_plan_equals_direct_batched(knng, precision):
    # the batched build recorded into one CUDA graph: every replay equals a
    # direct knng_build_batched call, also after the instances' data change
    specs = [(2000, 64, 64, 3), (5003, 64, 128, 3), (777, 128, 40, 2), (3000, 128, 128, 2), (150, 32, 40, 4)]
    k = 12
    datas = [_dev(datagen.gaussian_mixture(n, D, 20, seed=n + D) if i % 2 else
                  datagen.sift_like(n, D=D, n_centres=30, seed=n)) for i, (n, D, _, _) in enumerate(specs)]
    prec = {"fp32": knng.KNNG_FP32, "bf16": knng.KNNG_BF16}[precision]
    p = knng.default_params(k=k, leaf_max=64, tree_passes=2, refine_rounds=3, seed=21, precision=prec)
    lms, its = [lm for _, _, lm, _ in specs], [t for _, _, _, t in specs]
    want = knng.knng_build_batched(datas, p, leaf_maxes=lms, twomeans_iters=its)
    with knng.BatchedPlan(datas, p, leaf_maxes=lms, twomeans_iters=its) as plan:
        assert plan.kernels > 0
        for _ in range(2):
            outs = plan.launch()
            plan.check()
            for (ids, d), (wi, wd) in zip(outs, want):
                _assert_graph_equal(ids, d, _np(wi), _np(wd))
        for i, (n, D, _, _) in enumerate(specs):
            datas[i].copy_(torch.from_numpy(datagen.gaussian_mixture(n, D, 25, seed=7 * n + D)))
        want2 = knng.knng_build_batched(datas, p, leaf_maxes=lms, twomeans_iters=its)
        outs = plan.launch()
        plan.check()
        for (ids, d), (wi, wd) in zip(outs, want2):
            _assert_graph_equal(ids, d, _np(wi), _np(wd))
    # one instance alone, with its own schedule, gives the same lists
    n, D, lm, t = specs[1]
    q = knng.default_params(k=k, leaf_max=lm, tree_passes=2, refine_rounds=3, seed=21, precision=prec,
                            twomeans_iters=t)
    ids1, d1 = knng.knng_build_ex(datas[1], q)
    _assert_graph_equal(want2[1][0], want2[1][1], _np(ids1), _np(d1))
    with pytest.raises(knng.KnngError):   # instances of one D must share the schedule
        knng.knng_build_batched(datas[:2], p, twomeans_iters=[2, 3])


def test_batched_build_host_buffers_and_errors(knng):
    X1 = datagen.gaussian_mixture(1000, 16, 10, seed=1)
    X2 = datagen.gaussian_mixture(1500, 16, 10, seed=2)
    p = knng.default_params(k=8, leaf_max=32, tree_passes=1, refine_rounds=1, seed=3)
    outs = knng.knng_build_batched([X1, X2], p)      # numpy: host buffers through the C ABI
    for X, (ids, d) in zip([X1, X2], outs):
        ids1, d1 = knng.knng_build_ex(_dev(X), p)
        _assert_graph_equal(ids, d, _np(ids1), _np(d1))
    with pytest.raises(knng.KnngError):
        knng.knng_build_batched([X1, X2[:5]], p)      # second instance: n <= k


def test_autotune_picks_a_measured_tile_and_schedule(knng):
    from paper_1701_08475_gb300.autotune import autotune
    datas = [_dev(datagen.gaussian_mixture(6000, 32, 30, seed=1)), _dev(datagen.gaussian_mixture(3000, 64, 30, seed=2))]
    p = knng.default_params(k=10, tree_passes=1, refine_rounds=1, seed=4)
    leafs, iters, report = autotune(datas, p, iters_candidates=(1, 3), pilot_rows=4000, sample_rows=200)
    assert set(report) == {32, 64}
    for i, D in enumerate((32, 64)):
        rows = report[D]
        assert [(r[0], r[1]) for r in rows] == [(64, 1), (64, 3), (128, 1), (128, 3), (256, 1), (256, 3)]
        assert all(r[2] > 0 and 0 <= r[3] <= 1 for r in rows)
        best = max(r[3] for r in rows)
        pick = [r for r in rows if (r[0], r[1]) == (leafs[i], iters[i])][0]
        assert pick[3] >= best - 0.002
        assert pick[2] == min(r[2] for r in rows if r[3] >= best - 0.002)


def test_autotune_leaf_max_picks_a_measured_candidate(knng):
    from paper_1701_08475_gb300.autotune import autotune_leaf_max
    datas = [_dev(datagen.gaussian_mixture(6000, 32, 30, seed=1)), _dev(datagen.gaussian_mixture(3000, 64, 30, seed=2)),
             _dev(datagen.gaussian_mixture(4000, 32, 30, seed=3))]
    p = knng.default_params(k=10, tree_passes=1, refine_rounds=1, seed=4)
    leafs, report = autotune_leaf_max(datas, p, pilot_rows=4000, sample_rows=200)
    assert leafs[0] == leafs[2]                   # one choice per D
    assert set(report) == {32, 64}
    for D, rows in report.items():
        assert [r[0] for r in rows] == [64, 128, 256]
        assert all(r[1] > 0 and 0 <= r[2] <= 1 for r in rows)
        best = max(r[2] for r in rows)
        pick = [r for r in rows if r[0] == leafs[0 if D == 32 else 1]][0]
        assert pick[2] >= best - 0.002


@pytest.mark.parametrize("k,mode", [(16, oracle.FWD_REV), (24, oracle.FWD)])
def test_screening_join_matches_oracle(knng, monkeypatch, k, mode):
    # KNNG_JOIN_SCREEN=1: with a copy that is not exact the join screens pairs
    # on the tensor cores and decides offers on canonical distances
    monkeypatch.setenv("KNNG_JOIN_SCREEN", "1")
    n = 3500
    X = datagen.gaussian_mixture(n, 96, 40, seed=k + 1)
    common = dict(k=k, leaf_max=128, tree_passes=1, refine_rounds=4, seed=5, join_mode=mode)
    knng.stats_reset()
    knng.stats_enable(True, False)
    try:
        ids, d = knng.knng_build_ex(_dev(X), knng.default_params(precision=knng.KNNG_BF16, **common))
    finally:
        knng.stats_enable(False)
    assert knng.stats().get("k5_join_tc_cert", {}).get("launches", 0) > 0
    o_ids, o_d = oracle.build_graph(X, k, 128, passes=1, rounds=4, seed=5, mode=mode)
    _assert_graph_equal(ids, d, o_ids, o_d)


@pytest.mark.parametrize("kind,precision", [("float", "fp16"), ("float", "bf16"), ("integer", "bf16")])
def test_wide_rows_join_matches_oracle(knng, monkeypatch, kind, precision):
    # rows wider than four 64-dim chunks stream through the tensor-core join's
    # chunk ring: exact integers (the exact join) and float data (the
    # screening join, requested) both equal the FP32 build (and the oracle)
    monkeypatch.setenv("KNNG_JOIN_SCREEN", "1")
    n, D, k = 2500, 600, 12
    rng = np.random.default_rng(D + k)
    X = (rng.integers(0, 60, size=(n, D)).astype(np.float32) if kind == "integer"
         else datagen.gaussian_mixture(n, D, 25, seed=11))
    prec = {"bf16": knng.KNNG_BF16, "fp16": knng.KNNG_FP16}[precision]
    common = dict(k=k, leaf_max=64, tree_passes=2, refine_rounds=3, seed=5, join_mode=oracle.FWD_REV)
    knng.stats_reset()
    knng.stats_enable(True, False)
    try:
        ids, d = knng.knng_build_ex(_dev(X), knng.default_params(precision=prec, **common))
    finally:
        knng.stats_enable(False)
    joins = knng.stats()
    assert joins.get("k5_join_tc" if kind == "integer" else "k5_join_tc_cert", {}).get("launches", 0) > 0
    assert joins.get("k5_join", {}).get("launches", 0) == 0
    f_ids, f_d = knng.knng_build_ex(_dev(X), knng.default_params(precision=knng.KNNG_FP32, **common))
    _assert_graph_equal(ids, d, _np(f_ids), _np(f_d))
    if kind == "integer":
        o_ids, o_d = oracle.build_graph(X, k, 64, passes=2, rounds=3, seed=5, mode=oracle.FWD_REV)
        _assert_graph_equal(ids, d, o_ids, o_d)
    # the recorded build takes the same joins on the device
    Xd = _dev(X)
    with knng.BuildPlan(Xd, knng.default_params(precision=prec, **common)) as plan:
        pi, pd = plan.launch()
        plan.check()
        _assert_graph_equal(pi, pd, _np(f_ids), _np(f_d))


# ---------------------------------------------------------------- recorded builds
@pytest.mark.parametrize("precision,kind,mode", [("bf16", "integer", oracle.FWD_REV), ("fp32", "float", oracle.FWD_REV),
                                                 ("bf16", "float", oracle.FWD), ("fp16", "integer", oracle.FWD)])
def test_recorded_build_equals_direct_build(knng, precision, kind, mode):
    # a build recorded into a CUDA graph makes every data-dependent choice on
    # the device; replays equal direct builds, also after the data change kind
    n, D, k = 6000, 64, 12
    X = (datagen.sift_like(n, D=D, n_centres=60, seed=2) if kind == "integer"
         else datagen.gaussian_mixture(n, D, 30, seed=2))
    prec = {"fp32": knng.KNNG_FP32, "bf16": knng.KNNG_BF16, "fp16": knng.KNNG_FP16}[precision]
    p = knng.default_params(k=k, leaf_max=64, tree_passes=2, refine_rounds=3, seed=3, precision=prec, join_mode=mode)
    ids0, d0 = knng.knng_build_ex(_dev(X), p)
    Xd = _dev(X)
    with knng.BuildPlan(Xd, p) as plan:
        for _ in range(2):
            ids, d = plan.launch()
            plan.check()
            _assert_graph_equal(ids, d, _np(ids0), _np(d0))
        X2 = (datagen.gaussian_mixture(n, D, 30, seed=7) if kind == "integer"
              else datagen.sift_like(n, D=D, n_centres=60, seed=7))
        Xd.copy_(torch.from_numpy(X2))
        ids, d = plan.launch()
        plan.check()
        ids2, d2 = knng.knng_build_ex(_dev(X2), p)
        _assert_graph_equal(ids, d, _np(ids2), _np(d2))
        Xd[5, 3] = float("nan")
        plan.launch()
        with pytest.raises(knng.KnngError):
            plan.check()


def test_recorded_build_from_pinned_host_buffers(knng):
    # page-locked host data and outputs: each replay copies the rows in and
    # the lists out inside the graph; the lists equal the device build's
    n, D, k = 5000, 48, 10
    X = datagen.sift_like(n, D=D, n_centres=50, seed=4)
    p = knng.default_params(k=k, leaf_max=64, tree_passes=2, refine_rounds=2, seed=8,
                            precision=knng.KNNG_BF16, join_mode=oracle.FWD_REV)
    ids0, d0 = knng.knng_build_ex(_dev(X), p)
    o_ids, o_d = oracle.build_graph(X, k, 64, passes=2, rounds=2, seed=8, mode=oracle.FWD_REV)
    _assert_graph_equal(ids0, d0, o_ids, o_d)
    Xh = torch.from_numpy(X).pin_memory()
    with knng.BuildPlan(Xh, p) as plan:
        assert not plan.ids.is_cuda and plan.ids.is_pinned() and plan.dists.is_pinned()
        for _ in range(2):
            plan.ids.fill_(-7)
            ids, d = plan.launch()
            plan.check()  # waits for the stream: the lists are in host memory
            _assert_graph_equal(ids, d, o_ids, o_d)
        X2 = datagen.sift_like(n, D=D, n_centres=50, seed=9)
        Xh.copy_(torch.from_numpy(X2))
        ids, d = plan.launch()
        plan.check()
        ids2, d2 = knng.knng_build_ex(_dev(X2), p)
        _assert_graph_equal(ids, d, _np(ids2), _np(d2))
    # pageable host memory cannot be named by a recorded copy
    with pytest.raises(knng.KnngError):
        knng.BuildPlan(torch.from_numpy(X), p)
