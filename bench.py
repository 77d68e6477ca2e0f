"""Benchmark: kNN-graph build throughput (points/s) with recall@k against exact.

One step = one whole build (tree passes of Alg. 1, Sec. 3.1, then the
refinement rounds) of the workload's n points, inputs resident in HBM.
Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   # the CPU oracle on a bounded sample

N > 1 (under torchrun): every rank builds its own instance (weak scaling,
no collective on the data path); the step time is the max over ranks.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import datagen  # noqa: E402

DEFAULT_WORKLOAD = "sift-like-1m-d128"
REF_SAMPLE_N = 10_000      # oracle sample size per reference-arm step (~8 s)
CPU_BASELINE_N = 20_000    # oracle sample size of the cpu_baseline entry (~16 s)
RECALL_SAMPLE = 10_000


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-search", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16", "fp16"])
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_config(name):
    w = dict(datagen.WORKLOADS[name])
    return dict(workload=name, n=w["n"], D=w["D"], k=w["k"], leaf_max=w["leaf_max"], tree_passes=w["passes"],
                refine_rounds=w["rounds"], join_mode="fwd_rev", twomeans_iters=4, precision="fp32",
                generator=w["gen"], seed=w["seed"])


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == len(self.FIELDS):
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        if not self.rows:
            return None
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(self.rows), "reasons": reasons}


# ---------------------------------------------------------------- roofline
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


KERNEL_SOURCES = {"k1_": "split.cu", "k2_leaf_fp32": "leaf.cu", "k2_": "leaf_tc.cu", "k4_": "join.cu",
                  "k5_join_tc": "join_tc.cu", "k5_": "join.cu", "k6_": "join.cu", "k7_": "exact.cu",
                  "k0_": "leaf_tc.cu"}
ALU_KERNELS = ("k5_join", "k2_leaf_fp32", "k7_exact")
TENSOR_KERNELS = ("k2_leaf_bf16", "k2_leaf_fp16")


def kernel_source_hash(kernel):
    for pre, f in KERNEL_SOURCES.items():
        if kernel.startswith(pre):
            path = os.path.join(ROOT, "paper_1701_08475_gb300", "csrc", f)
            with open(path, "rb") as fh:
                return hashlib.sha256(fh.read()).hexdigest()[:16]
    return None


def profiled_traffic(kernel, workload):
    """DRAM bytes per algorithmic byte from the committed ncu summary of this
    kernel, or None when there is none or the kernel source changed since."""
    import glob
    path = os.path.join(ROOT, "profiles", "%s_%s.md" % (kernel, workload))
    if not os.path.exists(path):   # a capture of a smaller case of the same recipe
        cands = sorted(glob.glob(os.path.join(ROOT, "profiles", "%s_*.md" % kernel)))
        if not cands:
            return None
        path = cands[0]
    vals = {}
    with open(path) as f:
        for line in f:
            if line.startswith("- ") and ":" in line:
                k_, v = line[2:].split(":", 1)
                vals[k_.strip()] = v.strip().strip("`")
    if vals.get("source_sha256_16") != kernel_source_hash(kernel):
        return None
    try:
        return float(vals["dram_bytes_per_alg_byte"])
    except (KeyError, ValueError):
        return None


def roofline(stats, clocks, workload, steps, name=None):
    """Roofline of kernel `name` (default: the one with the most device time)."""
    peaks, kind = measured_peaks()
    if name is None:
        name = max(stats.items(), key=lambda kv: kv[1]["ms"])[0]
    st = stats[name]
    avg_ms = st["ms"] / st["launches"]
    per_launch_bytes = st["bytes"] / st["launches"]
    if name in ALU_KERNELS:
        # FP32 issue-slot roofline: one FSUB + one FFMA per pair and dim
        # (flops counted 3 per pair-dim: sub 1, fma 2 -> 2 issue slots)
        sm_mhz = (clocks or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
        ops = st["flops"] / st["launches"] * 2.0 / 3.0
        achieved = ops / (avg_ms * 1e-3) / 1e12
        peak = 152 * 128 * sm_mhz * 1e6 / 1e12
        out = {"kernel": name, "bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3),
               "unit": "Top/s", "frac": round(achieved / peak, 4),
               "peak_source": "derived: 152 SMs x 128 FP32 lanes x median SM clock %.0f MHz" % sm_mhz}
    elif name in TENSOR_KERNELS:
        # dense 16-bit tensor rate; timed inside a long step: the sustained peak
        achieved = st["flops"] / st["launches"] / (avg_ms * 1e-3) / 1e12
        peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1900.0)))
        out = {"kernel": name, "bound": "tensor", "achieved": round(achieved, 2), "peak": peak, "unit": "TFLOP/s",
               "frac": round(achieved / peak, 4), "peak_source": "%s bf16_tflops_sustained" % kind}
    else:
        achieved = per_launch_bytes / (avg_ms * 1e-3) / 1e9
        peak = float(peaks["hbm_gbs"])
        out = {"kernel": name, "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
               "frac": round(achieved / peak, 4), "peak_source": "%s hbm_gbs" % kind}
    ratio = profiled_traffic(name, workload)
    out["traffic"] = None if ratio is None else round(ratio * per_launch_bytes)
    out["alg_bytes_per_launch"] = round(per_launch_bytes)
    out["avg_launch_ms"] = round(avg_ms, 4)
    out["launches_per_step"] = st["launches"] / steps
    out["share_of_step"] = None
    return out


def distance_error(X, ids, dists, rows):
    """max |d - d64| / d64 over the stored entries of sampled rows, d64 the
    squared distance in FP64 (numpy, on the host)."""
    ids_h = ids[rows].cpu().numpy() if hasattr(ids, "cpu") else ids[rows]
    d_h = dists[rows].cpu().numpy() if hasattr(dists, "cpu") else dists[rows]
    worst, count = 0.0, 0
    for r, i in enumerate(rows):
        real = ids_h[r] >= 0
        if not real.any():
            continue
        diff = X[ids_h[r][real]].astype(np.float64) - X[i].astype(np.float64)
        d64 = np.einsum("ij,ij->i", diff, diff)
        pos = d64 > 0
        if pos.any():
            worst = max(worst, float(np.max(np.abs(d_h[r][real][pos] - d64[pos]) / d64[pos])))
        count += int(real.sum())
    return {"max_rel": worst, "entries": count, "rows": int(len(rows)),
            "against": "FP64 squared l2 of the stored pairs (numpy)"}


# ---------------------------------------------------------------- CPU oracle
def oracle_build_seconds(cfg, n_s):
    import oracle
    X = datagen.make(cfg["workload"], n_s)
    t = time.perf_counter()
    oracle.build_graph(X, cfg["k"], cfg["leaf_max"], passes=cfg["tree_passes"], rounds=cfg["refine_rounds"],
                       iters=cfg["twomeans_iters"], mode=oracle.FWD_REV, seed=cfg["seed"])
    return time.perf_counter() - t


def cpu_baseline(cfg):
    n_s = CPU_BASELINE_N
    sec = oracle_build_seconds(cfg, n_s)
    return {"value": round(n_s / sec, 1), "unit": "points/s", "cores": 1, "kind": "oracle",
            "sample": "whole build (same k, leaf_max, passes, rounds, iters) of the first recipe draw at "
                      "n=%d instead of %d points; %.1f s single-threaded" % (n_s, cfg["n"], sec),
            "host_cpus": os.cpu_count()}


def run_reference(args, cfg):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    n_s = REF_SAMPLE_N
    for _ in range(args.warmup):
        oracle_build_seconds(cfg, n_s)
    total = 0.0
    for _ in range(args.steps):
        total += oracle_build_seconds(cfg, n_s)
    value = n_s * args.steps / total
    line = {"impl": "reference", "metric": "kNN-graph build points/s at recall@k vs exact", "value": round(value, 1),
            "unit": "points/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total / args.steps * 1e3, 2), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": round(value, 1), "unit": "points/s", "cores": 1, "kind": "oracle",
                             "sample": "each step: whole build of n=%d points of the recipe (same parameters)" % n_s},
            "e2e": {"value": round(value, 1), "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
PRECISIONS = {"fp32": 0, "bf16": 1, "fp16": 2}


def search_measure(knng, X, Xd, G, dev, stream, m=10000, t0=12, ks=20, n_seeds=32, n_check=200):
    """The enhanced hill-climbing search (Alg. 2) over the built graph: m
    queries (input points moved by N(0, 4^2) noise, rounded and clipped for
    integer data), timed with CUDA events; recall against float64 brute force
    on n_check of them.  Seeds: random (the paper's baseline); random plus one
    point of the query's own cluster; and the inverted index of Sec. 4 (its
    training, indexing and seeding timed too)."""
    import torch
    n, D = X.shape
    rng = np.random.default_rng(17)
    base = rng.integers(0, n, size=m)
    Q = X[base].astype(np.float64) + rng.normal(0.0, 4.0, size=(m, D))
    if np.array_equal(X, np.rint(X)):
        Q = np.clip(np.rint(Q), X.min(), X.max())
    Q = Q.astype(np.float32)
    S_rand = rng.integers(0, n, size=(m, n_seeds)).astype(np.int32)
    S_near = S_rand.copy()
    S_near[:, 0] = G[:, -1].cpu().numpy()[base]
    Qd = torch.from_numpy(Q).to(dev)
    check = np.sort(rng.choice(m, size=n_check, replace=False))
    # ||x - q||^2 - ||q||^2 = ||x||^2 - 2 x.q, one float64 GEMM for all checked queries
    Xd64 = Xd.double()
    Qc = Qd[torch.from_numpy(check).to(dev)].double()
    part = (Xd64 * Xd64).sum(1, keepdim=True) - 2.0 * (Xd64 @ Qc.T)
    truth = torch.topk(part, ks, dim=0, largest=False).indices.T.cpu().numpy()
    del Xd64, part
    out = {"queries": m, "t0": t0, "ks": ks, "seeds_per_query": n_seeds,
           "queries_from": "input points moved by N(0, 4^2) noise", "truth": "float64 brute force, %d queries" % n_check}

    def timed(fn, reps=3):
        with torch.cuda.stream(stream):
            r = fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                r = fn()
            e1.record(stream)
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1) / reps

    # the inverted index of Sec. 4: vocabularies from a 100,000-row prefix,
    # the whole input indexed, seeds from the lists (Eqns. 2-3)
    n_train, W, iters, probe1 = min(n, 100000), 256, 8, 16
    (w1, w2), train_ms = timed(lambda: knng.knng_rvq_train(Xd[:n_train], W, W, iters, seed=5, stream=stream), 1)
    (_, off, lids), index_ms = timed(lambda: knng.knng_rvq_index(Xd, w1, w2, stream=stream), 1)
    S_ivf, seeds_ms = timed(lambda: knng.knng_rvq_seeds(w1, w2, off, lids, Qd, probe1, n_seeds, stream=stream))
    out["index"] = {"train_rows": n_train, "W1": W, "W2": W, "iters": iters, "probe1": probe1,
                    "train_ms": round(train_ms, 3), "index_ms": round(index_ms, 3), "seeds_ms": round(seeds_ms, 3),
                    "nonempty_lists": int((off[1:] > off[:-1]).sum().item())}
    # per-kernel device time of one training, indexing and seeding (events
    # around every launch: a separate, slower run)
    knng.stats_reset()
    knng.stats_enable(True, timing=True)
    with torch.cuda.stream(stream):
        knng.knng_rvq_train(Xd[:n_train], W, W, iters, seed=5, stream=stream)
        knng.knng_rvq_index(Xd, w1, w2, stream=stream)
        knng.knng_rvq_seeds(w1, w2, off, lids, Qd, probe1, n_seeds, stream=stream)
        knng.knng_search(Xd, G, Qd, S_ivf, t0, ks, stream=stream)
    torch.cuda.synchronize()
    knng.stats_enable(False)
    st = knng.stats()
    out["index"]["kernels_ms"] = {k: round(v["ms"], 3) for k, v in sorted(st.items(), key=lambda kv: -kv[1]["ms"])
                                  if v["ms"] >= 0.05}
    for name, S in (("random_seeds", S_rand), ("near_seed", S_near), ("ivf_seeds", S_ivf)):
        Sd = torch.from_numpy(S).to(dev) if isinstance(S, np.ndarray) else S
        with torch.cuda.stream(stream):
            knng.knng_search(Xd, G, Qd, Sd, t0, ks, stream=stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                ids, _d = knng.knng_search(Xd, G, Qd, Sd, t0, ks, stream=stream)
            e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 3
        got = ids.cpu().numpy()[check]
        r1 = float(np.mean([got[i, 0] == truth[i][0] for i in range(n_check)]))
        rk = float(np.mean([len(set(got[i].tolist()) & set(truth[i].tolist())) / ks for i in range(n_check)]))
        out[name] = {"queries_per_s": round(m / (ms * 1e-3), 1), "ms": round(ms, 3), "recall_at_1": round(r1, 4),
                     "recall_at_ks": round(rk, 4)}
        if name == "ivf_seeds":   # seeds and search together
            out[name]["queries_per_s_with_seeds"] = round(m / ((ms + seeds_ms) * 1e-3), 1)
    return out


def run_ours(args, cfg):
    import torch
    import paper_1701_08475_gb300 as knng

    from paper_1701_08475_gb300 import replicas

    rank, world, local = replicas.rank_env()
    torch.cuda.set_device(local)
    replicas.init("nccl")
    dev = torch.device("cuda", local)
    knng.load()

    X = datagen.make(cfg["workload"])
    if world > 1:   # independent replica per rank: a different draw
        X = np.ascontiguousarray(X[replicas.replica_rows(X.shape[0], rank)])
    n, D = X.shape
    Xd = torch.from_numpy(X).to(dev)
    stream = torch.cuda.Stream(dev)

    def params(prec):
        return knng.default_params(k=cfg["k"], leaf_max=cfg["leaf_max"], tree_passes=cfg["tree_passes"],
                                   refine_rounds=cfg["refine_rounds"], join_mode=knng.KNNG_JOIN_FWD_REV,
                                   twomeans_iters=cfg["twomeans_iters"], seed=cfg["seed"],
                                   precision=PRECISIONS[prec])

    barrier = replicas.barrier

    def max_over_ranks(v):
        return replicas.max_over_ranks(v, dev)

    def timed(prec, sample_clocks):
        """steps whole builds on one stream, CUDA events, after warm-up."""
        p = params(prec)
        ids = torch.empty((n, cfg["k"]), dtype=torch.int32, device=dev)
        dists = torch.empty((n, cfg["k"]), dtype=torch.float32, device=dev)
        with torch.cuda.stream(stream):
            for _ in range(max(3, args.warmup)):
                knng.knng_build_ex(Xd, p, stream=stream, out=(ids, dists))
        torch.cuda.synchronize()

        def run(stats):
            """steps builds between two events; with per-kernel event timing
            when `stats` (that run only feeds the breakdown and rooflines)."""
            knng.stats_reset()
            knng.stats_enable(True, timing=True) if stats else knng.stats_enable(True, timing=False)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            barrier()
            torch.cuda.synchronize()
            with torch.cuda.stream(stream):
                ev0.record(stream)
                for _ in range(args.steps):
                    knng.knng_build_ex(Xd, p, stream=stream, out=(ids, dists))
                ev1.record(stream)
            torch.cuda.synchronize()
            knng.stats_enable(False)
            barrier()
            return max_over_ranks(ev0.elapsed_time(ev1)), knng.stats()

        clocks = ClockSampler(local) if sample_clocks else None
        if clocks:
            clocks.start()
        ms, counted = run(False)     # the timed number: launches counted, no per-kernel events
        clk = clocks.stop() if clocks else None
        ms_k, st = run(True)
        for name_, v in st.items():  # launches of the timed run
            v["launches_timed_run"] = counted.get(name_, {}).get("launches", 0)
        return ms, st, clk, ids, dists, ms_k

    ms_direct, st, _, ids, dists, ms_k = timed(args.precision, False)
    launches_direct = sum(v["launches_timed_run"] for v in st.values())

    # recall of the last graph on sampled rows, against exact lists
    smp = datagen.sample_rows(n, RECALL_SAMPLE, seed=3)
    smp_d = torch.from_numpy(smp).to(dev)
    gi, gd = knng.knng_exact(Xd, cfg["k"], smp_d)
    rec_ids, rec_tie = knng.knng_recall(ids, dists, gi, gd, smp_d)
    dist_err = distance_error(X, ids, dists, smp[:2000])

    # the plain FP32 form of the same build, timed the same way
    def replayed(prec, sample_clocks):
        """The build recorded once into a CUDA graph (knng_plan_create, outside
        the timed region) and replayed once per step (knng_plan_launch)."""
        plan = knng.BuildPlan(Xd, params(prec), stream=stream)
        with torch.cuda.stream(stream):
            for _ in range(max(3, args.warmup)):
                plan.launch()
        torch.cuda.synchronize()
        plan.check()
        clocks = ClockSampler(local) if sample_clocks else None
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        with torch.cuda.stream(stream):
            g0.record(stream)
            for _ in range(args.steps):
                plan.launch()
            g1.record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop() if clocks else None
        plan.check()
        out = (max_over_ranks(g0.elapsed_time(g1)), plan.kernels, plan.ids.clone(), plan.dists.clone(), clk)
        plan.close()
        return out

    fp32 = None
    if args.precision != "fp32":
        ms32, _, ids32, d32, _ = replayed("fp32", False)
        r32 = knng.knng_recall(ids32, d32, gi, gd, smp_d)
        fp32 = {"value": round(replicas.aggregate(n, args.steps, ms32 * 1e-3, world), 1),
                "ms_per_step": round(ms32 / args.steps, 3),
                "recall_ids": round(r32[0], 5),
                "graph_identical": bool(torch.equal(ids32, ids) and torch.equal(d32, dists))}

    ms, kernels, gids, gd_, clk = replayed(args.precision, True)
    value = replicas.aggregate(n, args.steps, ms * 1e-3, world)
    launches = kernels * args.steps
    graph_same = bool(torch.equal(gids, ids) and torch.equal(gd_, dists))
    direct = {"value": round(replicas.aggregate(n, args.steps, ms_direct * 1e-3, world), 1),
              "ms_per_step": round(ms_direct / args.steps, 3), "gpu_launches": int(launches_direct),
              "graph_identical": graph_same,
              "how": "knng_build_ex per step (the host launches every kernel and reads offer counts back)"}

    # end to end: host buffers through the C ABI, copies inside the timed region
    p = params(args.precision)
    Xh = torch.from_numpy(X).pin_memory()
    oi = torch.empty((n, cfg["k"]), dtype=torch.int32).pin_memory()
    od = torch.empty((n, cfg["k"]), dtype=torch.float32).pin_memory()
    knng.knng_build_ex(Xh, p, stream=stream, out=(oi, od))   # warm
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        knng.knng_build_ex(Xh, p, stream=stream, out=(oi, od))
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": round(replicas.aggregate(n, args.e2e_steps, e2e_s, world), 1), "unit": "points/s",
           "h2d_bytes_per_step": int(X.nbytes), "d2h_bytes_per_step": int(oi.numel() * 4 + od.numel() * 4),
           "steps": args.e2e_steps, "timer": "host wall clock around synchronous C-ABI calls"}
    same = bool(torch.equal(oi, ids.cpu()) and torch.equal(od, dists.cpu()))

    if rank != 0:
        replicas.finish()
        return
    roof = roofline(st, clk, cfg["workload"], args.steps)
    roof["share_of_step"] = round(st[roof["kernel"]]["ms"] / ms_k, 4)
    # the same figures for the other kernels above 2 % of the step
    others = []
    for name_, v in sorted(st.items(), key=lambda kv: -kv[1]["ms"]):
        if name_ == roof["kernel"] or v["ms"] < 0.02 * ms_k or v["launches"] == 0 or v["ms"] <= 0:
            continue
        r_ = roofline(st, clk, cfg["workload"], args.steps, name_)
        r_["share_of_step"] = round(v["ms"] / ms_k, 4)
        others.append({key: r_[key] for key in ("kernel", "bound", "achieved", "peak", "unit", "frac",
                                                 "share_of_step", "traffic")})
    cfg_out = dict(cfg)
    cfg_out["precision"] = args.precision
    cfg_out["l2"] = "inputs larger than L2: X is %.0f MB (L2 129 MB)" % (X.nbytes / 1e6)
    line = {
        "metric": "kNN-graph build points/s at recall@k vs exact", "value": round(value, 1), "unit": "points/s",
        "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": round(ms / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else args.precision + "+f32", "data": "synthetic",
        "config": cfg_out,
        "recall_at_k": {"ids": round(rec_ids, 5), "tie": round(rec_tie, 5), "sample_rows": int(len(smp)),
                        "exact": "knng_exact canonical FP32"},
        "timed": "CUDA-graph replays of the recorded build (knng_plan_launch), inputs resident in HBM",
        "direct_form": direct,
        "fp32_form": fp32,
        "roofline": roof, "roofline_other_kernels": others, "distance_error": dist_err, "e2e": e2e, "e2e_graph_equals_device_graph": same, "gpu_launches": int(launches),
        "clocks": clk,
        "kernels": {k_: {"ms_per_step": round(v["ms"] / args.steps, 3), "launches_per_step": v["launches"] / args.steps}
                    for k_, v in sorted(st.items(), key=lambda kv: -kv[1]["ms"])[:10]},
        "kernel_breakdown_run": {"ms_per_step": round(ms_k / args.steps, 3),
                                 "note": "a second run of the same steps with CUDA events around every launch; "
                                         "the per-kernel times, shares and rooflines come from it"},
    }
    if world == 1 and not args.no_search:
        line["search"] = search_measure(knng, X, Xd, ids, dev, stream)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg)
    print(json.dumps(line), flush=True)
    replicas.finish()


def run_batched(args):
    """The batched workload: 64 independent instances in one knng_build_batched
    call per step, leaf_max per D from the autotuner (time not counted)."""
    import torch
    import paper_1701_08475_gb300 as knng
    from paper_1701_08475_gb300.autotune import autotune_leaf_max

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    w = datagen.BATCHED
    datas = datagen.batched_mixtures(n_inst=w["n_inst"], seed=w["seed"] + rank)
    n_tot = sum(x.shape[0] for x in datas)
    dev = [torch.from_numpy(x).cuda() for x in datas]
    prec = PRECISIONS[args.precision]
    p = knng.default_params(k=w["k"], leaf_max=128, tree_passes=w["passes"], refine_rounds=w["rounds"],
                            join_mode=knng.KNNG_JOIN_FWD_REV, seed=w["seed"], precision=prec)
    leafs, report = autotune_leaf_max(dev, p)
    stream = torch.cuda.Stream()

    def timed(q):
        with torch.cuda.stream(stream):
            for _ in range(max(3, args.warmup)):
                outs = knng.knng_build_batched(dev, q, leaf_maxes=leafs, stream=stream)
        torch.cuda.synchronize()
        knng.stats_reset()
        knng.stats_enable(True, timing=False)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(args.steps):
                outs = knng.knng_build_batched(dev, q, leaf_maxes=leafs, stream=stream)
            e1.record(stream)
        torch.cuda.synchronize()
        launches = sum(v["launches"] for v in knng.stats().values())
        knng.stats_enable(False)
        return e0.elapsed_time(e1), outs, launches

    ms, outs, launches = timed(p)
    # recall on 200 sampled rows of every instance
    hit = tot = 0
    for x, (ids, d) in zip(dev, outs):
        smp = torch.from_numpy(datagen.sample_rows(x.shape[0], 200, seed=5)).cuda()
        gi, gd = knng.knng_exact(x, w["k"], smp)
        r = knng.knng_recall(ids, d, gi, gd, smp)[0]
        hit += r * len(smp)
        tot += len(smp)
    q32 = knng.default_params(k=w["k"], leaf_max=128, tree_passes=w["passes"], refine_rounds=w["rounds"],
                              join_mode=knng.KNNG_JOIN_FWD_REV, seed=w["seed"], precision=knng.KNNG_FP32)
    ms32, outs32, _ = timed(q32)
    same = all(torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]) for a, b in zip(outs, outs32))
    line = {
        "metric": "kNN-graph build points/s at recall@k vs exact", "value": round(n_tot * args.steps / (ms * 1e-3), 1),
        "unit": "points/s", "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup),
        "ms_per_step": round(ms / args.steps, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else args.precision + "+f32", "data": "synthetic",
        "config": {"workload": w["name"], "instances": len(datas), "points": int(n_tot), "k": w["k"],
                   "tree_passes": w["passes"], "refine_rounds": w["rounds"], "precision": args.precision,
                   "leaf_max_by_D": {str(x.shape[1]): l for x, l in zip(datas, leafs)},
                   "autotune": {str(D): rows for D, rows in report.items()}},
        "recall_at_k": {"ids": round(hit / tot, 5), "sample_rows": int(tot)},
        "fp32_form": {"value": round(n_tot * args.steps / (ms32 * 1e-3), 1), "ms_per_step": round(ms32 / args.steps, 3),
                      "graph_identical": bool(same)},
        "gpu_launches": int(launches),
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.workload == datagen.BATCHED["name"]:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the batched workload has no reference arm; "
                              "the oracle arm runs the single-instance workloads"}))
            return
        run_batched(args)
        return
    cfg = workload_config(args.workload)
    if args.impl == "reference":
        run_reference(args, cfg)
    else:
        run_ours(args, cfg)


if __name__ == "__main__":
    main()
