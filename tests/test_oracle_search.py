"""Pins of the oracle's enhanced hill-climbing search (Sec. 3.2, Alg. 2).

Each pin is fixed by the algorithm's definition on an input where the answer
has a closed form: no iterations leave the seeds ranked by distance; one
iteration over a complete graph visits every point (brute force); on a path
graph the frontier advances one node per iteration.  Expected values come
from float64 numpy, never from the oracle itself.
"""
import numpy as np
import pytest

import oracle


def _d64(X, q):
    diff = X.astype(np.float64) - q.astype(np.float64)
    return np.einsum("ij,ij->i", diff, diff)


def _topk(d, ks):
    order = np.lexsort((np.arange(len(d)), d))
    return order[:ks]


def test_no_iterations_rank_the_seeds():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((300, 16)).astype(np.float32)
    Q = rng.standard_normal((8, 16)).astype(np.float32)
    S = np.stack([rng.choice(300, size=12, replace=False) for _ in range(8)]).astype(np.int32)
    G = np.full((300, 4), -1, np.int32)
    ids, d = oracle.search(X, G, Q, S, 0, 5)
    for r in range(8):
        dd = _d64(X[S[r]], Q[r])
        want = S[r][_topk(dd, 5)]
        assert np.array_equal(ids[r], want)
        assert np.allclose(d[r], np.sort(dd)[:5], rtol=1e-5)


def test_one_iteration_over_a_complete_graph_is_brute_force():
    rng = np.random.default_rng(2)
    n = 120
    X = rng.standard_normal((n, 8)).astype(np.float32)
    G = np.array([[j for j in range(n) if j != i] for i in range(n)], np.int32)
    Q = rng.standard_normal((10, 8)).astype(np.float32)
    S = rng.integers(0, n, size=(10, 1)).astype(np.int32)
    ids, d = oracle.search(X, G, Q, S, 1, 7)
    for r in range(10):
        dd = _d64(X, Q[r])
        assert np.array_equal(ids[r], _topk(dd, 7))
        assert np.allclose(d[r], np.sort(dd)[:7], rtol=1e-5)


@pytest.mark.parametrize("ks", [1, 2, 4])
@pytest.mark.parametrize("t0", [0, 1, 3, 7, 40])
def test_path_graph_frontier_moves_one_node_per_iteration(ks, t0):
    n = 25
    X = np.arange(n, dtype=np.float32)[:, None]
    G = np.array([[i - 1 if i > 0 else -1, i + 1 if i + 1 < n else -1] for i in range(n)], np.int32)
    Q = np.array([[n + 5.0]], np.float32)          # far to the right
    S = np.array([[0]], np.int32)
    ids, d = oracle.search(X, G, Q, S, t0, ks)
    front = min(t0, n - 1)                         # nodes 0 .. front are visited
    want = [front - a if front - a >= 0 else -1 for a in range(ks)]
    assert ids[0].tolist() == want
    for a, i in enumerate(want):
        assert (d[0, a] == (n + 5.0 - i) ** 2) if i >= 0 else np.isinf(d[0, a])


def test_repeated_and_out_of_range_seeds_count_once():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((40, 4)).astype(np.float32)
    G = np.full((40, 2), -1, np.int32)
    Q = rng.standard_normal((1, 4)).astype(np.float32)
    S = np.array([[5, 5, -1, 40, 7, 5]], np.int32)
    ids, d = oracle.search(X, G, Q, S, 3, 4)
    dd = _d64(X[[5, 7]], Q[0])
    want = np.array([5, 7])[np.argsort(dd)]
    assert ids[0, :2].tolist() == want.tolist()
    assert ids[0, 2:].tolist() == [-1, -1] and np.isinf(d[0, 2:]).all()


def test_rows_are_sorted_unique_and_carry_canonical_distances():
    rng = np.random.default_rng(4)
    X = rng.integers(0, 50, size=(400, 12)).astype(np.float32)
    G, _ = oracle.build_graph(X, 8, 40, passes=1, rounds=1, seed=3)
    Q = rng.integers(0, 50, size=(6, 12)).astype(np.float32)
    S = rng.integers(0, 400, size=(6, 4)).astype(np.int32)
    ids, d = oracle.search(X, G, Q, S, 4, 10)
    for r in range(6):
        real = ids[r] >= 0
        assert len(set(ids[r][real].tolist())) == real.sum()
        keys = list(zip(d[r][real].tolist(), ids[r][real].tolist()))
        assert keys == sorted(keys)
        for i, dv in zip(ids[r][real], d[r][real]):
            assert dv == np.float32(_d64(X[i:i + 1], Q[r])[0])   # integer data: exact in FP32


@pytest.mark.parametrize("ks,want", [(2, [2, 0]), (1, [0])])
def test_every_top_entry_is_expanded_not_only_the_first(ks, want):
    # Alg. 2 expands each of the top ks entries per iteration (the change from
    # the original GNNS, which expands only the first).  1-D points, dyadic so
    # every distance is exact: q = 10.5; seeds A = 10 (d 0.25) and B = 13
    # (d 6.25); B's only neighbour C = 10.75 (d 0.0625) beats A, A's only
    # neighbour E = 20 (d 90.25).  With ks = 2 one iteration finds C.
    X = np.array([[10.0], [13.0], [10.75], [20.0]], np.float32)
    G = np.array([[3], [2], [1], [0]], np.int32)
    Q = np.array([[10.5]], np.float32)
    S = np.array([[0, 1]], np.int32)
    ids, d = oracle.search(X, G, Q, S, 1, ks)
    assert ids[0].tolist() == want
    assert d[0].tolist() == [{0: 0.25, 1: 6.25, 2: 0.0625, 3: 90.25}[i] for i in want]
