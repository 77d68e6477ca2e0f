"""Measured choice of each instance's cluster bound (leaf_max) for batched builds.

The cluster bound of Sec. 3.1 ("no bigger than a threshold") trades time for
recall: larger leaves compare more pairs per pass.  For every dimension D
present, the tuner builds a pilot (the first rows of the largest instance of
that D) once per candidate bound with the caller's other parameters, times
each build with CUDA events and measures its recall@k on sampled rows against
exact lists, then keeps the fastest candidate whose recall is within
`recall_slack` of the best.  Every build and measurement goes through the
library's own entry points.
"""
import numpy as np

from . import _lib as L

__all__ = ["autotune_leaf_max"]


def autotune_leaf_max(datas, params, candidates=(64, 128, 256), pilot_rows=20000, sample_rows=500,
                      recall_slack=0.002, repeats=2):
    """Returns (leaf_max per instance, report {D: [(leaf_max, ms, recall), ...]}).

    datas: device tensors (n_i x D_i, float32); params: the build's Params
    (its leaf_max is ignored)."""
    import torch

    k = params.k
    cands = [c for c in candidates if c >= 2 * (k + 1) and c <= 256]
    if not cands:
        raise ValueError("no candidate leaf_max >= 2(k+1) = %d" % (2 * (k + 1)))
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
        for c in cands:
            q = L.Params()
            for f, _ in L.Params._fields_:
                setattr(q, f, getattr(params, f))
            q.leaf_max = c
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
            rec = L.knng_recall(ids, d, gi, gd, smp)[0]
            rows.append((c, float(np.median(times)), float(rec)))
        best = max(r[2] for r in rows)
        ok = [r for r in rows if r[2] >= best - recall_slack]
        choice[D] = min(ok, key=lambda r: r[1])[0]
        report[D] = rows
    return [choice[int(x.shape[1])] for x in datas], report
