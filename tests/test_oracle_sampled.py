"""Pins of the oracle's sampled refinement round: nearest-neighbour descent
with sampling (the prior art Sec. 1 cites; Dong, Charikar and Li 2011), in
Jacobi form, with per-entry new/old flags and ms samples per list.

Fixed by the definition, not by the oracle's output: without samples or
without new entries nothing is joined; with an unlimited sample every
new x new and new x old pair of each node's members (its list and its
reverse lists) is joined, which a set-based brute force of the definition
reproduces exactly (lists and flags), and so does it with limited samples
drawn by the (pinned) priority; the sample is the ms new entries of least
priority; lists only improve; rounds from random lists approach the
exact graph.
"""
import numpy as np
import pytest

import oracle


def _random_lists(X, k, seed):
    rng = np.random.default_rng(seed)
    n = len(X)
    ids, d = oracle.new_graph(n, k)
    for i in range(n):
        for j in rng.choice(n, size=k + 2, replace=False):
            if j != i:
                oracle.list_insert(ids[i], d[i], oracle.dist_f32(X[i], X[j]), int(j))
    return ids, d


def test_priority_is_splitmix_of_the_stated_key():
    for seed, r, v, u in [(0, 0, 0, 0), (5, 3, 17, 4), (2**40 + 1, 7, 123456, 99)]:
        h = oracle.splitmix64(oracle.splitmix64(seed ^ r) ^ ((v << 32) | u))
        assert oracle.sample_prio(seed, r, v, u) == (h & ~0xFFFFFFFF) | u     # hash bits above the id
    assert oracle.sample_prio(1, 0, 3, 4) != oracle.sample_prio(1, 1, 3, 4)
    assert oracle.sample_prio(1, 0, 3, 4) != oracle.sample_prio(1, 0, 4, 3)


def test_no_samples_or_no_new_entries_change_nothing():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((60, 5)).astype(np.float32)
    ids, d = _random_lists(X, 6, 2)
    flags = np.ones(ids.shape, np.uint8)
    i2, d2, f2, c = oracle.refine_sampled(X, ids, d, flags, 0, seed=3)
    assert c == 0 and np.array_equal(i2, ids) and np.array_equal(d2, d) and np.array_equal(f2, flags)
    flags = np.zeros(ids.shape, np.uint8)
    i2, d2, f2, c = oracle.refine_sampled(X, ids, d, flags, 6, seed=3)
    assert c == 0 and np.array_equal(i2, ids) and np.array_equal(f2, flags)


def _least(owner, members, ms, seed, r):
    return set(sorted(members, key=lambda u: (oracle.sample_prio(seed, r, owner, u), u))[:ms])


def _brute_round(X, ids, d, flags, ms=10**6, seed=0, r=0):
    """The round from the definition with sets: samples of ms by priority."""
    n, k = ids.shape
    fresh = [set(int(u) for u, f in zip(ids[v], flags[v]) if u >= 0 and f) for v in range(n)]
    new = [_least(v, fresh[v], ms, seed, r) for v in range(n)]
    old = [set(int(u) for u, f in zip(ids[v], flags[v]) if u >= 0 and not f) for v in range(n)]
    rnew = [set() for _ in range(n)]
    rold = [set() for _ in range(n)]
    for v in range(n):
        for u in new[v]:
            rnew[u].add(v)
        for u in old[v]:
            rold[u].add(v)
    rnew = [_least(u, rnew[u], ms, seed, r) for u in range(n)]
    rold = [_least(u, rold[u], ms, seed, r) for u in range(n)]
    offers = [set() for _ in range(n)]
    for v in range(n):
        Nn = new[v] | rnew[v]
        No = (old[v] | rold[v]) - Nn
        for a in Nn:
            for b in Nn | No:
                if a != b:
                    offers[a].add(b)
                    offers[b].add(a)
    out_ids = np.full_like(ids, -1)
    out_d = np.full_like(d, np.inf)
    out_f = np.zeros_like(flags)
    for u in range(n):
        cand = {int(j): float(dj) for j, dj in zip(ids[u], d[u]) if j >= 0}
        cand_old = set(cand)
        for w in offers[u]:
            cand.setdefault(w, oracle.dist_f32(X[u], X[w]))
        best = sorted(cand.items(), key=lambda t: (t[1], t[0]))[:k]
        for t, (j, dj) in enumerate(best):
            out_ids[u, t], out_d[u, t] = j, dj
            out_f[u, t] = 1 if (j not in cand_old or j in fresh[u] - new[u]) else 0
    return out_ids, out_d, out_f


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_unlimited_sample_joins_every_new_pair(seed):
    rng = np.random.default_rng(seed)
    X = rng.integers(0, 30, size=(40, 4)).astype(np.float32)
    ids, d = _random_lists(X, 4, seed)
    flags = (rng.random(ids.shape) < 0.6).astype(np.uint8)
    i2, d2, f2, c = oracle.refine_sampled(X, ids, d, flags, 10**6, seed=seed, round_=2)
    wi, wd, wf = _brute_round(X, ids, d, flags)
    assert np.array_equal(i2, wi)
    assert np.array_equal(d2, wd)
    assert np.array_equal(f2, wf)
    assert c == int(sum(len(set(wi[u][wi[u] >= 0]) - set(ids[u][ids[u] >= 0])) for u in range(len(X))))


@pytest.mark.parametrize("seed,ms", [(3, 1), (4, 2), (5, 3)])
def test_limited_sample_joins_the_sampled_members(seed, ms):
    rng = np.random.default_rng(seed + 10)
    X = rng.integers(0, 30, size=(50, 4)).astype(np.float32)
    ids, d = _random_lists(X, 5, seed)
    flags = (rng.random(ids.shape) < 0.7).astype(np.uint8)
    i2, d2, f2, _ = oracle.refine_sampled(X, ids, d, flags, ms, seed=seed, round_=1)
    wi, wd, wf = _brute_round(X, ids, d, flags, ms, seed, 1)
    assert np.array_equal(i2, wi)
    assert np.array_equal(d2, wd)
    assert np.array_equal(f2, wf)


def test_the_sample_is_the_least_priorities():
    rng = np.random.default_rng(6)
    X = rng.standard_normal((80, 6)).astype(np.float32)
    k, ms, seed, r = 6, 2, 9, 4
    ids, d = _random_lists(X, k, 7)
    flags = np.ones(ids.shape, np.uint8)
    i2, _, f2, _ = oracle.refine_sampled(X, ids, d, flags, ms, seed=seed, round_=r)
    for v in range(len(X)):
        live = [int(u) for u in ids[v] if u >= 0]
        sampled = sorted(live, key=lambda u: (oracle.sample_prio(seed, r, v, u), u))[:ms]
        for t, u in enumerate(i2[v]):
            if u in live:   # an entry that stayed: old exactly when it was sampled
                assert f2[v, t] == (0 if u in sampled else 1), (v, u)


def test_lists_only_improve_and_stay_canonical():
    rng = np.random.default_rng(8)
    X = rng.standard_normal((150, 8)).astype(np.float32)
    ids, d = _random_lists(X, 8, 9)
    flags = np.ones(ids.shape, np.uint8)
    for r in range(5):
        i2, d2, flags, _ = oracle.refine_sampled(X, ids, d, flags, 4, seed=1, round_=r)
        assert (d2[:, -1] <= d[:, -1]).all()
        for u in range(len(X)):
            real = i2[u] >= 0
            assert len(set(i2[u][real].tolist())) == real.sum() and u not in i2[u]
            keys = list(zip(d2[u][real].tolist(), i2[u][real].tolist()))
            assert keys == sorted(keys)
            for j, dj in zip(i2[u][real], d2[u][real]):
                assert dj == np.float32(oracle.dist_f32(X[u], X[j]))
        ids, d = i2, d2


def test_sampled_rounds_approach_the_exact_graph():
    rng = np.random.default_rng(10)
    centres = rng.uniform(-10, 10, size=(8, 6))
    X = (centres[rng.integers(0, 8, 400)] + rng.standard_normal((400, 6))).astype(np.float32)
    k = 8
    ids, d = _random_lists(X, k, 11)
    flags = np.ones(ids.shape, np.uint8)
    gi, gd = oracle.exact_f32(X, k)
    r0 = oracle.recall(ids, d, gi, gd, np.arange(400))[0]
    changes = []
    for r in range(10):
        ids, d, flags, c = oracle.refine_sampled(X, ids, d, flags, k // 2, seed=2, round_=r)
        changes.append(c)
    r1 = oracle.recall(ids, d, gi, gd, np.arange(400))[0]
    assert r0 < 0.2 and r1 > 0.9, (r0, r1)
    assert changes[-1] < changes[0]


def test_sampled_build_is_the_passes_then_sampled_rounds():
    rng = np.random.default_rng(12)
    X = rng.integers(0, 40, size=(700, 8)).astype(np.float32)
    k, ms, seed = 8, 3, 21
    ids, d = oracle.build_graph_sampled(X, k, 32, passes=2, rounds=3, iters=3, ms=ms, seed=seed)
    wi, wd = oracle.build_graph(X, k, 32, passes=2, rounds=0, iters=3, seed=seed)
    flags = np.ones(wi.shape, np.uint8)
    for r in range(3):
        wi, wd, flags, _ = oracle.refine_sampled(X, wi, wd, flags, ms, seed=seed, round_=r)
    assert np.array_equal(ids, wi) and np.array_equal(d, wd)
    i0, _ = oracle.build_graph_sampled(X, k, 32, passes=2, rounds=0, iters=3, ms=ms, seed=seed)
    b0, _ = oracle.build_graph(X, k, 32, passes=2, rounds=0, iters=3, seed=seed)
    assert np.array_equal(i0, b0)
