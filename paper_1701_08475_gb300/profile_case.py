"""Run one stage of the build on a workload, with few kernel launches before
it, so that a profiler can capture that stage's kernels.

  python -m paper_1701_08475_gb300.profile_case STAGE [--workload NAME] [--n N] [--repeat R]

STAGE:
  build   the whole build (passes + rounds) of the workload
  sampled the whole build with the sampled refinement round (ms = k / 2)
  split   one tree pass's partition (the K1 kernels)
  leaf    the leaf stage on a random balanced partition made on the host
  refine  one refinement round on a random graph made on the host
  exact   exact lists of 1024 sampled rows
  search  build the graph (BF16) and the RVQ index (2 x 256 words, 8
          iterations on a 100,000-row prefix), then seed and search 10,000
          queries near the data (t0 = 12, ks = 20, 32 seeds, probe1 = 16)
"""
import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import datagen  # noqa: E402
import paper_1701_08475_gb300 as knng  # noqa: E402


def random_graph(n, k, seed):
    """Random neighbour lists with empty distances filled in by a pack-free
    path: ids only; distances +inf so every offer is taken."""
    rng = np.random.default_rng(seed)
    ids = rng.integers(0, n - 1, size=(n, k), dtype=np.int64)
    ids += ids >= np.arange(n)[:, None]          # no self loops
    ids = np.sort(ids, axis=1)
    dup = np.zeros_like(ids, dtype=bool)
    dup[:, 1:] = ids[:, 1:] == ids[:, :-1]
    ids[dup] = -1
    order = np.argsort(ids < 0, axis=1, kind="stable")  # empty slots last
    ids = np.take_along_axis(ids, order, axis=1).astype(np.int32)
    return ids


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("stage", choices=["build", "sampled", "split", "leaf", "refine", "exact", "search"])
    ap.add_argument("--workload", default="sift-like-1m-d128")
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "fp16", "fp8"])
    a = ap.parse_args()
    import torch

    w = datagen.WORKLOADS[a.workload]
    X = datagen.make(a.workload, a.n)
    n, D = X.shape
    k = w["k"]
    Xd = torch.from_numpy(X).cuda()
    if a.stage == "search":
        p = knng.default_params(k=k, leaf_max=w["leaf_max"], tree_passes=w["passes"], refine_rounds=w["rounds"],
                                seed=w["seed"], precision=knng.KNNG_BF16)
        G, _ = knng.knng_build_ex(Xd, p)
        w1, w2 = knng.knng_rvq_train(Xd[:min(n, 100000)], 256, 256, 8, seed=5)
        _, off, lids = knng.knng_rvq_index(Xd, w1, w2)
        rng = np.random.default_rng(17)
        Q = np.clip(np.rint(X[rng.integers(0, n, 10000)] + rng.normal(0, 4.0, size=(10000, D))), X.min(),
                    X.max()).astype(np.float32)
        Qd = torch.from_numpy(Q).cuda()
    for _ in range(a.repeat):
        if a.stage == "search":
            S = knng.knng_rvq_seeds(w1, w2, off, lids, Qd, 16, 32)
            knng.knng_search(Xd, G, Qd, S, 12, 20)
        elif a.stage in ("build", "sampled"):
            p = knng.default_params(k=k, leaf_max=w["leaf_max"], tree_passes=w["passes"], refine_rounds=w["rounds"],
                                    seed=w["seed"], precision={"fp32": 0, "bf16": 1, "fp16": 2, "fp8": 3}[a.precision])
            if a.stage == "sampled":
                p.join_mode = knng.KNNG_JOIN_SAMPLED
                p.sample = k // 2
            knng.knng_build_ex(Xd, p)
        elif a.stage == "split":
            knng.knng_partition(Xd, w["leaf_max"], seed=w["seed"])
        elif a.stage == "leaf":
            L = knng.knng_tree_depth(n, w["leaf_max"])
            off = np.linspace(0, n, (1 << L) + 1).astype(np.int64)
            perm = np.random.default_rng(0).permutation(n).astype(np.int32)
            for s, e in zip(off[:-1], off[1:]):
                perm[s:e].sort()
            ids = torch.full((n, k), -1, dtype=torch.int32, device="cuda")
            d = torch.full((n, k), float("inf"), dtype=torch.float32, device="cuda")
            knng.knng_leaf_update(Xd, k, torch.from_numpy(perm).cuda(), torch.from_numpy(off).cuda(), ids, d)
        elif a.stage == "refine":
            ids_h = random_graph(n, k, 1)
            ids = torch.from_numpy(ids_h).cuda()
            # canonical distances of the random lists come from the exact kernel's
            # definition; here every slot is re-offered, so +inf is enough
            d = torch.full((n, k), float("inf"), dtype=torch.float32, device="cuda")
            d[ids < 0] = float("inf")
            p = knng.default_params(k=k, refine_rounds=1, join_mode=knng.KNNG_JOIN_FWD_REV)
            knng.knng_refine(Xd, ids, d, p)
        elif a.stage == "exact":
            smp = torch.from_numpy(datagen.sample_rows(n, 1024, seed=1)).cuda()
            knng.knng_exact(Xd, k, smp)
    torch.cuda.synchronize()
    print("ok", a.stage, n, D)


if __name__ == "__main__":
    main()
