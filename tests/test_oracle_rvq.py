"""Pins of the oracle's residue vector quantisation and inverted index
(Sec. 4.1, Eqn. 1; Sec. 4.2, Eqns. 2 and 3, cascaded pruning).

Each pin is fixed by a definition or a closed form, never by the oracle's own
output: brute-force nearest words in float64 on data whose FP32 distances are
exact; cluster means of separated clusters after one Lloyd iteration; the
fixed point of converged Lloyd iterations (every word the mean of its members,
every vector at its nearest word), checked in float64 on dyadic data where the
FP32 arithmetic is exact; the monotone quantisation error of Lloyd's
iterations; the degenerate vocabularies W = n and W = 1; the index as a
stable sort by key; and the seeds against Eqn. 2 evaluated directly in
integers, which catches any slip in the expansion of Eqn. 3.
"""
import numpy as np
import pytest

import oracle


def _sq64(A, B):
    A = A.astype(np.float64)
    B = B.astype(np.float64)
    return ((A[:, None, :] - B[None, :, :]) ** 2).sum(-1)


def test_init_positions_one_per_stratum():
    for N, W in [(10, 10), (1000, 256), (257, 256), (5000, 7)]:
        for stage in (1, 2):
            pos = oracle.rvq_init_positions(N, W, 11, stage)
            lo = np.arange(W, dtype=np.int64) * N // W
            hi = (np.arange(W, dtype=np.int64) + 1) * N // W
            assert ((pos >= lo) & (pos < hi)).all()
    a = oracle.rvq_init_positions(100000, 64, 11, 1)
    assert not np.array_equal(a, oracle.rvq_init_positions(100000, 64, 11, 2))
    assert not np.array_equal(a, oracle.rvq_init_positions(100000, 64, 12, 1))


def test_zero_iterations_give_each_stage_its_drawn_vectors():
    # With no Lloyd iteration each stage's words are its own draws: stage 1 the
    # points at the stage-1 positions; stage 2 the residues (x - w1[c1], c1 the
    # brute-force nearest stage-1 word on integer data) at the stage-2 positions.
    rng = np.random.default_rng(7)
    X = rng.integers(-50, 51, size=(3000, 6)).astype(np.float32)
    W1, W2, seed = 24, 16, 9
    w1, w2 = oracle.rvq_train(X, W1, W2, iters=0, seed=seed)
    p1 = oracle.rvq_init_positions(3000, W1, seed, 1)
    p2 = oracle.rvq_init_positions(3000, W2, seed, 2)
    assert np.array_equal(w1, X[p1])
    c1 = np.argmin(_sq64(X, w1), axis=1)
    assert np.array_equal(w2, (X - w1[c1])[p2])


def test_a_word_without_members_keeps_its_value():
    # Identical points: every draw is the same vector, every vector goes to
    # word 0 (ties to the smaller index), the other words have no member and
    # keep their value, so every word of stage 1 is the point (stage 2: zero).
    X = np.tile(np.array([[3.0, -1.5, 7.25]], np.float32), (500, 1))
    w1, w2 = oracle.rvq_train(X, 8, 4, iters=3, seed=2)
    assert np.array_equal(w1, np.tile(X[:1], (8, 1)))
    assert not w2.any()


def test_assign_is_the_brute_force_argmin_with_ties_to_the_smaller_index():
    rng = np.random.default_rng(1)
    V = rng.integers(0, 4, size=(2000, 5)).astype(np.float32)        # many exact ties
    words = rng.integers(0, 4, size=(40, 5)).astype(np.float32)
    words[7] = words[3]                                                # duplicate words
    codes = oracle.rvq_assign(V, words)
    assert np.array_equal(codes, np.argmin(_sq64(V, words), axis=1))  # argmin takes the first
    assert not (codes == 7).any()


def _clustered(W, M, D, seed):
    """W separated integer clusters of M points each, cluster c in rows c*M .. c*M + M - 1."""
    rng = np.random.default_rng(seed)
    centres = rng.permutation(W)[:, None] * 1000.0 + rng.integers(0, 50, size=(W, D))
    X = centres[:, None, :] + rng.integers(-20, 21, size=(W, M, D))
    return X.reshape(W * M, D).astype(np.float32)


def test_one_iteration_from_separated_clusters_gives_their_means():
    W, M, D = 12, 9, 6
    X = _clustered(W, M, D, 2)
    w1, _ = oracle.rvq_train(X, W, 3, iters=1, seed=5)
    want = X.reshape(W, M, D).astype(np.float64).mean(1).astype(np.float32)   # integer sums: exact
    assert np.array_equal(w1, want)
    w1b, _ = oracle.rvq_train(X, W, 3, iters=6, seed=5)                         # a fixed point
    assert np.array_equal(w1b, want)
    w1z, _ = oracle.rvq_train(X, W, 3, iters=0, seed=5)                         # no iteration: the draws
    assert np.array_equal(w1z, X[oracle.rvq_init_positions(len(X), W, 5, 1)])


def _converged(X, W1, W2, seed):
    for T in range(1, 60):
        a = oracle.rvq_train(X, W1, W2, iters=T, seed=seed)
        b = oracle.rvq_train(X, W1, W2, iters=T + 1, seed=seed)
        if all(np.array_equal(u, v) for u, v in zip(a, b)):
            return a
    raise AssertionError("Lloyd did not settle in 60 iterations")


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_converged_training_is_a_fixed_point_of_both_stages(seed):
    # integer data: stage-1 sums are exact, so the stage-1 words equal the
    # float64 means of their members rounded to FP32 exactly; the residues
    # (FP32 differences, Eqn. 1) are summed exactly here (math.fsum), so the
    # stage-2 words lie within the rounding of a float64 sum of their members
    import math
    rng = np.random.default_rng(seed)
    X = rng.integers(0, 16, size=(256, 4)).astype(np.float32)
    w1, w2 = _converged(X, 8, 6, seed)
    codes, _, _ = oracle.rvq_index(X, w1, w2)
    c1, c2 = codes[:, 0], codes[:, 1]
    d1 = _sq64(X, w1)
    assert (d1[np.arange(256), c1] <= d1.min(1) * (1 + 1e-6) + 1e-9).all()   # nearest stage-1 word
    R = (X - w1[c1]).astype(np.float32)                                       # residues in FP32
    d2 = _sq64(R, w2)
    assert (d2[np.arange(256), c2] <= d2.min(1) * (1 + 1e-6) + 1e-9).all()   # nearest stage-2 word
    for j in range(len(w1)):
        if (c1 == j).any():
            assert np.array_equal(w1[j], X[c1 == j].astype(np.float64).mean(0).astype(np.float32)), j
    for j in range(len(w2)):
        M = R[c2 == j].astype(np.float64)
        if len(M):
            exact = np.array([math.fsum(M[:, t]) / len(M) for t in range(M.shape[1])])
            bound = 2.0 ** -23 * np.abs(exact) + 2.0 ** -50 * np.abs(M).sum(0)
            assert (np.abs(w2[j] - exact) <= bound).all(), j


def test_quantisation_error_never_grows_over_iterations():
    # Lloyd's iterations never raise the quantisation error of a stage
    # (up to the FP32 rounding of the means); stage 2 run as the first stage of
    # a training on the residues sees fixed inputs
    rng = np.random.default_rng(4)
    X = (rng.standard_normal((600, 8)) * 3 + rng.integers(0, 4, size=(600, 1)) * 10).astype(np.float32)
    prev = np.inf
    for T in range(0, 8):
        w1, _ = oracle.rvq_train(X, 16, 1, iters=T, seed=9)
        e = _sq64(X, w1).min(1).sum()
        assert e <= prev * (1 + 1e-6)
        prev = e
    c1 = np.argmin(_sq64(X, w1), axis=1)
    R = (X - w1[c1]).astype(np.float32)
    prev = _sq64(X, w1).min(1).sum()                 # stage 2 refines stage 1's error
    for T in range(0, 8):
        w2, _ = oracle.rvq_train(R, 16, 1, iters=T, seed=9)
        e = _sq64(R, w2).min(1).sum()
        assert e <= prev * (1 + 1e-6)
        prev = e
    # a two-stage training's stage 2 is that Lloyd run on the same residues
    _, w2b = oracle.rvq_train(X, 16, 16, iters=7, seed=9)
    assert _sq64(R, w2b).min(1).sum() <= _sq64(X, w1).min(1).sum()


def test_one_word_per_point_and_a_single_word():
    rng = np.random.default_rng(6)
    X = rng.integers(0, 100, size=(30, 5)).astype(np.float32)
    w1, w2 = oracle.rvq_train(X, 30, 30, iters=4, seed=2)
    assert np.array_equal(w1, X)                     # every point its own word
    assert not w2.any()                              # residues all zero
    w1, w2 = oracle.rvq_train(X, 1, 1, iters=3, seed=2)
    assert np.array_equal(w1[0], X.astype(np.float64).mean(0).astype(np.float32))
    R = X.astype(np.float64) - w1[0].astype(np.float64)
    assert np.allclose(w2[0], (X - w1[0]).astype(np.float64).mean(0), atol=1e-5)
    assert np.abs(R.mean(0)).max() < 1e-3


def test_index_is_a_stable_sort_by_key():
    rng = np.random.default_rng(7)
    X = rng.integers(0, 8, size=(3000, 6)).astype(np.float32)
    w1 = rng.integers(0, 8, size=(10, 6)).astype(np.float32)
    w2 = rng.integers(-2, 3, size=(7, 6)).astype(np.float32)
    codes, off, ids = oracle.rvq_index(X, w1, w2)
    c1 = np.argmin(_sq64(X, w1), axis=1)
    c2 = np.argmin(_sq64(X.astype(np.float64) - w1[c1], w2), axis=1)
    assert np.array_equal(codes[:, 0], c1) and np.array_equal(codes[:, 1], c2)
    key = c1 * 7 + c2
    assert np.array_equal(off, np.concatenate([[0], np.cumsum(np.bincount(key, minlength=70))]))
    assert np.array_equal(ids, np.argsort(key, kind="stable"))


def _seeds_by_eqn2(w1, w2, off, ids, q, p1, s):
    """Eqn. 2 evaluated directly in integers, pruning by term 1 = |q - w1|^2."""
    W2 = len(w2)
    q = q.astype(np.int64)
    t1 = ((q - w1.astype(np.int64)) ** 2).sum(1)
    kept = np.lexsort((np.arange(len(w1)), t1))[:p1]
    cand = []
    for a in kept:
        for b in range(W2):
            d = int(((q - w1[a].astype(np.int64) - w2[b].astype(np.int64)) ** 2).sum())
            cand.append((d, int(a) * W2 + b))
    cand.sort()
    out = []
    for _, key in cand:
        out.extend(ids[off[key]:off[key + 1]].tolist())
    out = out[:s]
    return out + [-1] * (s - len(out))


@pytest.mark.parametrize("p1,s", [(1, 5), (3, 40), (12, 300), (12, 5000)])
def test_seeds_follow_eqn2_with_pruning_by_the_first_term(p1, s):
    rng = np.random.default_rng(8)
    W1, W2, D, n = 12, 9, 6, 2000
    w1 = rng.integers(-8, 9, size=(W1, D)).astype(np.float32)
    w2 = rng.integers(-3, 4, size=(W2, D)).astype(np.float32)
    key = rng.integers(0, W1 * W2, size=n)
    key[key % 5 == 0] = 0                                 # some long lists, some empty ones
    off = np.concatenate([[0], np.cumsum(np.bincount(key, minlength=W1 * W2))]).astype(np.int32)
    ids = np.argsort(key, kind="stable").astype(np.int32)
    Q = rng.integers(-10, 11, size=(25, D)).astype(np.float32)
    S = oracle.rvq_seeds(w1, w2, off, ids, Q, p1, s)
    for r in range(len(Q)):
        assert S[r].tolist() == _seeds_by_eqn2(w1, w2, off, ids, Q[r], p1, s), r


def test_seeds_tie_by_key_when_the_query_norm_absorbs_the_differences():
    # Eqn. 3's first term is evaluated in FP32 with the query's squared norm
    # in it: for q = (2^14, 0) every stage-1 word (0, u) with u^2 < 16 gets
    # term1 = fl(2^28 + u^2) = 2^28 (the spacing of FP32 there is 32), so every
    # key ties and the seeds come by ascending key: point a is word a's only
    # member, so the seeds are 0, 1, ..., W1 - 1, then -1 padding.
    # word a = (0, u_a, a / 4): |w|^2 <= 9 + 49/16 < 16; the third coordinate,
    # which q does not see, keeps words with the same u apart
    u = np.array([3, 0, 2, 1, 3, 2, 0, 1], np.float32)
    w1 = np.stack([np.zeros(8, np.float32), u, np.arange(8, dtype=np.float32) / 4], 1)
    w2 = np.zeros((1, 3), np.float32)
    codes, off, ids = oracle.rvq_index(w1, w1, w2)
    assert np.array_equal(codes[:, 0], np.arange(8))
    Q = np.array([[2.0 ** 14, 0.0, 0.0]], np.float32)
    S = oracle.rvq_seeds(w1, w2, off, ids, Q, 8, 10)
    assert S[0].tolist() == list(range(8)) + [-1, -1]


def test_seeds_on_float_data_follow_the_direct_distance_up_to_rounding():
    rng = np.random.default_rng(9)
    X = rng.standard_normal((3000, 10)).astype(np.float32)
    w1, w2 = oracle.rvq_train(X, 16, 16, iters=4, seed=3)
    codes, off, ids = oracle.rvq_index(X, w1, w2)
    Q = rng.standard_normal((10, 10)).astype(np.float32)
    S = oracle.rvq_seeds(w1, w2, off, ids, Q, 16, 3000)
    assert (np.sort(S, axis=1) == np.arange(3000)).all()   # all lists: every point once
    for r in range(10):
        c = codes[S[r]]
        w = w1[c[:, 0]].astype(np.float64) + w2[c[:, 1]].astype(np.float64)
        d = ((Q[r].astype(np.float64) - w) ** 2).sum(1)
        assert (np.diff(d) >= -1e-4 * (1 + d[1:])).all()
