"""Measured choice of each instance's leaf tile shape and split schedule for batched builds.

Two parameters of Sec. 3.1's tree trade time for recall and set how the GPU
tiles the work: the cluster bound ("no bigger than a threshold", leaf_max)
fixes the leaf kernel's tile shape (clusters of up to 128 points fill one
128-row tensor-core tile, larger ones two) and the number of pairs per pass;
the Lloyd iterations per two-means split (twomeans_iters) fix the split's
schedule (one projection, selection and centroid sweep per iteration and
level).  For every dimension D present, the tuner builds a pilot (the first
rows of the largest instance of that D) once per candidate pair with the
caller's other parameters, times each build with CUDA events, measures its
recall@k on sampled rows against exact lists, and keeps the fastest candidate
whose recall is within `recall_slack` of the best.  Every build and
measurement goes through the library's own entry points.
"""
import numpy as np

from . import _lib as L

__all__ = ["autotune", "autotune_leaf_max", "pick"]


def _timed_build(pilot, q, repeats):
    import torch
    ids, d = L.knng_build_ex(pilot, q)  # warm
    times = []
    for _ in range(repeats):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        ids, d = L.knng_build_ex(pilot, q)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return ids, d, float(np.median(times))


def pick(rows, recall_slack):
    """The fastest of rows (leaf_max, twomeans_iters, ms, recall) whose recall
    is within recall_slack of the best; the first of equally fast ones."""
    best = max(r[3] for r in rows)
    ok = [r for r in rows if r[3] >= best - recall_slack]
    return min(ok, key=lambda r: r[2])


def autotune(datas, params, leaf_candidates=(64, 128, 256), iters_candidates=(2, 3, 4), pilot_rows=20000,
             sample_rows=500, recall_slack=0.002, repeats=2):
    """Returns (leaf_max per instance, twomeans_iters per instance, report
    {D: [(leaf_max, twomeans_iters, ms, recall), ...]}).

    datas: device tensors (n_i x D_i, float32); params: the build's Params
    (its leaf_max and twomeans_iters are the ones tuned)."""
    import torch

    k = params.k
    leafs = [c for c in leaf_candidates if 2 * (k + 1) <= c <= 256]
    if not leafs:
        raise ValueError("no candidate leaf_max >= 2(k+1) = %d" % (2 * (k + 1)))
    iters = [t for t in iters_candidates if 0 <= t <= 64] or [params.twomeans_iters]
    by_dim = {}
    for i, x in enumerate(datas):
        by_dim.setdefault(int(x.shape[1]), []).append(i)
    choice, report = {}, {}
    for D, idx in by_dim.items():
        big = max(idx, key=lambda i: datas[i].shape[0])
        pilot = datas[big][: min(pilot_rows, datas[big].shape[0])].contiguous()
        n = pilot.shape[0]
        rng = np.random.default_rng(D)
        smp = torch.from_numpy(np.sort(rng.choice(n, size=min(sample_rows, n), replace=False)).astype(np.int32))
        smp = smp.to(pilot.device)
        gi, gd = L.knng_exact(pilot, k, smp)
        rows = []
        for c in leafs:
            for t in iters:
                q = L.Params()
                for f, _ in L.Params._fields_:
                    setattr(q, f, getattr(params, f))
                q.leaf_max = c
                q.twomeans_iters = t
                ids, d, ms = _timed_build(pilot, q, repeats)
                rec = L.knng_recall(ids, d, gi, gd, smp)[0]
                rows.append((c, t, ms, float(rec)))
        chosen = pick(rows, recall_slack)
        choice[D] = (chosen[0], chosen[1])
        report[D] = rows
    return ([choice[int(x.shape[1])][0] for x in datas], [choice[int(x.shape[1])][1] for x in datas], report)


def autotune_leaf_max(datas, params, candidates=(64, 128, 256), pilot_rows=20000, sample_rows=500,
                      recall_slack=0.002, repeats=2):
    """The cluster bound alone (the caller's twomeans_iters kept): (leaf_max
    per instance, report {D: [(leaf_max, ms, recall), ...]})."""
    leafs, _, report = autotune(datas, params, leaf_candidates=candidates,
                                iters_candidates=(params.twomeans_iters,), pilot_rows=pilot_rows,
                                sample_rows=sample_rows, recall_slack=recall_slack, repeats=repeats)
    return leafs, {D: [(c, ms, rec) for c, _, ms, rec in rows] for D, rows in report.items()}
