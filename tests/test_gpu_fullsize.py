"""GPU parity at the workloads' full sizes, in the launch configuration that
bench.py times, on sampled outputs and on properties that hold at any size.

Per workload: the low-precision graph equals the FP32 graph bit for bit (the
certified re-rank, or exact mode); every row satisfies the graph conventions;
the stored distances of sampled rows equal the oracle's canonical FP32
distance of the same pairs bit for bit; recall@k against exact lists of
sampled rows stays above the level the build reaches (a regression guard,
not a claim about the method); and leaf lists of sampled leaves of a
GPU-made partition equal the oracle's leaf stage on the same leaves.
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


def _check_rows(ids, d):
    """Graph conventions on every row: k real entries, no self loop, unique
    ids, sorted by (d, id)."""
    ids, d = _np(ids), _np(d)
    n, k = ids.shape
    assert (ids >= 0).all() and (ids < n).all()
    assert not np.any(ids == np.arange(n)[:, None])
    s = np.sort(ids, axis=1)
    assert not np.any(s[:, 1:] == s[:, :-1])
    assert np.all(d[:, 1:] >= d[:, :-1])
    tie = d[:, 1:] == d[:, :-1]
    assert not np.any(tie & (ids[:, 1:] < ids[:, :-1]))


def _check_sampled_distances(X, ids, d, rows):
    ids, d = _np(ids), _np(d)
    for i in rows:
        for j, dij in zip(ids[i], d[i]):
            assert np.float32(oracle.dist_f32(X[i], X[j])).view(np.uint32) == np.float32(dij).view(np.uint32)


def _recall(knng, Xd, ids, d, k, n_rows):
    smp = torch.from_numpy(datagen.sample_rows(Xd.shape[0], n_rows, seed=11)).cuda()
    gi, gd = knng.knng_exact(Xd, k, smp)
    return knng.knng_recall(ids, d, gi, gd, smp)[0]


def _check_leaves(knng, X, Xd, k, leaf_max, seed, n_leaves=24):
    """Leaf stage on the GPU's own partition: sampled leaves against the
    oracle's leaf stage run on just those leaves."""
    perm, off = knng.knng_partition(Xd, leaf_max, seed=seed)
    perm, off = _np(perm), _np(off)
    n = X.shape[0]
    ids = torch.full((n, k), -1, dtype=torch.int32, device="cuda")
    d = torch.full((n, k), float("inf"), dtype=torch.float32, device="cuda")
    knng.knng_leaf_update(Xd, k, _dev(perm), _dev(off), ids, d)
    ids, d = _np(ids), _np(d)
    rng = np.random.default_rng(seed)
    for l in rng.choice(len(off) - 1, size=n_leaves, replace=False):
        a, b = int(off[l]), int(off[l + 1])
        pts = np.sort(perm[a:b])
        Xs = X[pts]
        o_ids, o_d = oracle.leaf_update(Xs, k, np.arange(b - a, dtype=np.int32), np.array([0, b - a]))
        got = ids[pts]
        mapped = np.where(o_ids >= 0, pts[np.maximum(o_ids, 0)], -1)
        assert np.array_equal(got, mapped), "leaf %d ids" % l
        assert np.array_equal(d[pts].view(np.uint32), o_d.view(np.uint32)), "leaf %d distances" % l


def _full_build(knng, name, precision, recall_floor, check_leaves=True):
    w = datagen.WORKLOADS[name]
    X = datagen.make(name)
    Xd = _dev(X)
    k = w["k"]
    common = dict(k=k, leaf_max=w["leaf_max"], tree_passes=w["passes"], refine_rounds=w["rounds"], seed=w["seed"],
                  join_mode=knng.KNNG_JOIN_FWD_REV)
    lp_ids, lp_d = knng.knng_build_ex(Xd, knng.default_params(precision=precision, **common))
    f_ids, f_d = knng.knng_build_ex(Xd, knng.default_params(precision=knng.KNNG_FP32, **common))
    assert torch.equal(lp_ids, f_ids) and torch.equal(lp_d, f_d), "low-precision graph differs from FP32"
    _check_rows(f_ids, f_d)
    rows = datagen.sample_rows(X.shape[0], 300, seed=7)
    _check_sampled_distances(X, f_ids, f_d, rows)
    rec = _recall(knng, Xd, f_ids, f_d, k, 2000)
    assert rec >= recall_floor, rec
    if check_leaves:
        _check_leaves(knng, X, Xd, k, w["leaf_max"], w["seed"])
    return rec


def test_sift_like_1m_d128_bf16(knng):
    _full_build(knng, "sift-like-1m-d128", knng.KNNG_BF16, 0.98)   # reaches 0.992


def _holders(ids, n):
    """For every id t, the nodes whose list holds t (CSR: order, start, end)."""
    k = ids.shape[1]
    tgt = ids.ravel().astype(np.int64)
    src = np.repeat(np.arange(n, dtype=np.int64), k)
    keep = tgt >= 0
    tgt, src = tgt[keep], src[keep]
    order = np.argsort(tgt, kind="stable")
    tgt, src = tgt[order], src[order]
    ids_ = np.arange(n)
    return src, np.searchsorted(tgt, ids_), np.searchsorted(tgt, ids_, side="right")


def _check_round_on_sampled_nodes(X, ids0, d0, ids1, d1, rows):
    """One refinement round (Jacobi, forward and reverse lists) on sampled
    nodes against its definition, with the oracle's reverse lists, canonical
    distances and list insertion: node v's new list is its old list offered
    every member u != v of every node i whose members (G_old[i] and R[i])
    hold v."""
    n, k = ids0.shape
    rid, rd = oracle.reverse_lists(ids0, d0)
    g_src, g_lo, g_hi = _holders(ids0, n)   # i with v in G_old[i]
    r_src, r_lo, r_hi = _holders(rid, n)    # i with v in R[i]
    for v in rows:
        joins = set(g_src[g_lo[v]:g_hi[v]].tolist()) | set(r_src[r_lo[v]:r_hi[v]].tolist())
        cand = set()
        for i in joins:
            m = set(ids0[i][ids0[i] >= 0].tolist()) | set(rid[i][rid[i] >= 0].tolist())
            assert v in m
            cand |= m
        cand.discard(int(v))
        e_ids, e_d = ids0[v].copy(), d0[v].copy()
        for u in sorted(cand):
            oracle.list_insert(e_ids, e_d, oracle.dist_f32(X[v], X[u]), u)
        assert np.array_equal(ids1[v], e_ids), "node %d ids" % v
        assert np.array_equal(d1[v].view(np.uint32), e_d.view(np.uint32)), "node %d distances" % v


def test_sift_like_1m_rounds_on_sampled_nodes(knng):
    # the first round (every member new) and the last one (old pairs and leaf
    # mates skipped, nodes without a new member not joined) of the bench's
    # build, each from the graph the build reached before it
    name = "sift-like-1m-d128"
    w = datagen.WORKLOADS[name]
    X = datagen.make(name)
    Xd = _dev(X)
    graphs = {}
    for r in (0, 1, w["rounds"] - 1, w["rounds"]):
        p = knng.default_params(k=w["k"], leaf_max=w["leaf_max"], tree_passes=w["passes"], refine_rounds=r,
                                seed=w["seed"], precision=knng.KNNG_BF16, join_mode=knng.KNNG_JOIN_FWD_REV)
        ids, d = knng.knng_build_ex(Xd, p)
        graphs[r] = (_np(ids), _np(d))
    rows = datagen.sample_rows(X.shape[0], 150, seed=13)
    for r in (1, w["rounds"]):
        _check_round_on_sampled_nodes(X, *graphs[r - 1], *graphs[r], rows)


def test_gist_like_1m_d960_fp16(knng):
    _full_build(knng, "gist-like-1m-d960", knng.KNNG_FP16, 0.90, check_leaves=False)   # reaches 0.926


def test_unit_10m_d96_bf16(knng):
    _full_build(knng, "unit-10m-d96", knng.KNNG_BF16, 0.53, check_leaves=False)   # reaches 0.558


def test_batched_64_instances(knng):
    w = datagen.BATCHED
    datas = datagen.batched_mixtures(n_inst=w["n_inst"], seed=w["seed"])
    dev = [_dev(x) for x in datas]
    p = knng.default_params(k=w["k"], leaf_max=128, tree_passes=w["passes"], refine_rounds=w["rounds"],
                            seed=w["seed"], precision=knng.KNNG_BF16)
    outs = knng.knng_build_batched(dev, p)
    for ids, d in outs:
        _check_rows(ids, d)
    # sampled instances equal their own builds
    for i in (0, 17, 41, 63):
        ids1, d1 = knng.knng_build_ex(dev[i], p)
        assert torch.equal(outs[i][0], ids1) and torch.equal(outs[i][1], d1), "instance %d" % i
        rows = datagen.sample_rows(datas[i].shape[0], 50, seed=i)
        _check_sampled_distances(datas[i], outs[i][0], outs[i][1], rows)
