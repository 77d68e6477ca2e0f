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
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-search", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the other workloads' measurements")
    ap.add_argument("--config-steps", type=int, default=2, help="timed steps per form of the other workloads")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16", "fp16", "fp8"])
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_config(name, precision="fp32"):
    w = dict(datagen.WORKLOADS[name])
    X_mb = w["n"] * w["D"] * 4 / 1e6
    return dict(workload=name, n=w["n"], D=w["D"], k=w["k"], leaf_max=w["leaf_max"], tree_passes=w["passes"],
                refine_rounds=w["rounds"], join_mode="fwd_rev", twomeans_iters=4, precision=precision,
                generator=w["gen"], seed=w["seed"],
                l2="inputs larger than L2: X is %.0f MB (L2 129 MB)" % X_mb if X_mb > 129 else
                   "X is %.1f MB, smaller than L2 (129 MB): a latency case" % X_mb)


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


# the sources whose change makes a kernel's committed counters stale: its own
# file, and for the tensor-core join also join.cu, which sets the order in
# which it takes the nodes (and so its DRAM traffic)
KERNEL_SOURCES = {"k1_": ("split.cu",), "k2_leaf_fp32": ("leaf.cu",), "k2_": ("leaf_tc.cu",), "k4_": ("join.cu",),
                  "k5_join_tc": ("join_tc.cu", "join.cu"), "k5_": ("join.cu",), "k6_": ("join.cu",),
                  "k7_": ("exact.cu",), "k0_": ("leaf_tc.cu",)}
ALU_KERNELS = ("k5_join", "k2_leaf_fp32", "k7_exact")
TENSOR_KERNELS = ("k2_leaf_bf16", "k2_leaf_fp16", "k2_leaf_fp8")


def kernel_source_hash(kernel):
    for pre, files in KERNEL_SOURCES.items():
        if kernel.startswith(pre):
            h = hashlib.sha256()
            for f in files:
                with open(os.path.join(ROOT, "paper_1701_08475_gb300", "csrc", f), "rb") as fh:
                    h.update(fh.read())
            return h.hexdigest()[:16]
    return None


def profiled_traffic(kernel, workload):
    """DRAM bytes per algorithmic byte from the committed ncu summary of this
    kernel, or None when there is none or the kernel source changed since."""
    import glob
    path = os.path.join(ROOT, "profiles", "%s_%s.md" % (kernel, workload))
    if not os.path.exists(path):
        # a capture of a smaller case of the same recipe: the kernel's exact
        # name, then the recipe's name (the workload's up to its size)
        recipe = workload.split("-")[0]
        cands = sorted(glob.glob(os.path.join(ROOT, "profiles", "%s_%s-*.md" % (kernel, recipe))))
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
        # dense tensor rate; timed inside a long step: the sustained peak.
        # FP16 runs at the BF16 rate; FP8 at twice it (the nominal 4.5 / 2.25
        # PFLOP/s ratio applied to the measured BF16 figure)
        achieved = st["flops"] / st["launches"] / (avg_ms * 1e-3) / 1e12
        ratio = 2.0 if name == "k2_leaf_fp8" else 1.0
        peak = ratio * float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1900.0)))
        out = {"kernel": name, "bound": "tensor", "achieved": round(achieved, 2), "peak": peak, "unit": "TFLOP/s",
               "frac": round(achieved / peak, 4),
               "peak_source": "%s bf16_tflops_sustained%s" % (kind, " x 2 (nominal FP8 / BF16)" if ratio != 1 else "")}
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


def kernel_roofline_ms(name, st, clocks, peaks):
    """Roofline time of all of a kernel's launches, in ms: the larger of its
    algorithmic bytes at the measured HBM bandwidth and its arithmetic at the
    peak of its kind (tensor kernels: the sustained dense rate, FP8 at twice
    BF16; the FP32 kernels: the derived FFMA issue rate, two issue slots per
    pair and dim as in roofline()).  Returns (ms, bound)."""
    t_mem = st["bytes"] / (float(peaks["hbm_gbs"]) * 1e9)
    t_cmp, kind = 0.0, "hbm"
    if name in TENSOR_KERNELS:
        ratio = 2.0 if name == "k2_leaf_fp8" else 1.0
        peak = ratio * float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1900.0))) * 1e12
        t_cmp, kind = st["flops"] / peak, "tensor"
    elif name in ALU_KERNELS:
        sm_mhz = (clocks or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
        t_cmp, kind = st["flops"] * 2.0 / 3.0 / (152 * 128 * sm_mhz * 1e6), "alu"
    if t_cmp > t_mem:
        return t_cmp * 1e3, kind
    return t_mem * 1e3, "hbm"


def whole_build_roofline(stats, clocks, builds, ms_per_step):
    """The whole build against its roofline: the sum over kernels of each
    kernel's roofline time (kernel_roofline_ms) per build, divided by the
    measured time of one build.  `stats` covers `builds` builds."""
    peaks, kind = measured_peaks()
    by = {"hbm": 0.0, "tensor": 0.0, "alu": 0.0}
    for name, st in stats.items():
        if st["launches"] == 0:
            continue
        t, bound = kernel_roofline_ms(name, st, clocks, peaks)
        by[bound] += t / builds
    ideal = sum(by.values())
    return {"roofline_ms_per_step": round(ideal, 3), "ms_per_step": round(ms_per_step, 3),
            "frac": round(ideal / ms_per_step, 4) if ms_per_step > 0 else None,
            "roofline_ms_by_bound": {b: round(v, 3) for b, v in by.items()},
            "peak_source": "%s peaks" % kind,
            "how": "sum over kernels of max(algorithmic bytes / HBM peak, arithmetic / peak of its kind) per "
                   "build, divided by the timed step"}


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
def oracle_build_seconds(cfg, n_s, X=None):
    import oracle
    if X is None:
        X = datagen.make(cfg["workload"], n_s)
    t = time.perf_counter()
    oracle.build_graph(X, cfg["k"], cfg["leaf_max"], passes=cfg["tree_passes"], rounds=cfg["refine_rounds"],
                       iters=cfg["twomeans_iters"], mode=oracle.FWD_REV, seed=cfg["seed"])
    return time.perf_counter() - t


def oracle_all_cores(cfg, n_s, cores=None):
    """The single-threaded oracle run as `cores` independent builds at once
    (one host thread each; the C code runs without the GIL), each on its own
    draw of the recipe: whole-host throughput of the oracle as it stands."""
    from concurrent.futures import ThreadPoolExecutor
    import oracle
    cores = cores or os.cpu_count() or 1
    oracle.build()
    draws = [datagen.make(cfg["workload"], n_s) if i == 0 else None for i in range(cores)]
    # other draws: the same recipe at another seed (the generators take the seed)
    w = datagen.WORKLOADS[cfg["workload"]]
    for i in range(1, cores):
        draws[i] = datagen.make_seeded(cfg["workload"], n_s, w["seed"] + 1000 * i)
    t = time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(lambda X: oracle_build_seconds(cfg, n_s, X), draws))
    sec = time.perf_counter() - t
    return cores * n_s / sec, sec, cores


def cpu_baseline(cfg, n_s=None):
    n_s = n_s or CPU_BASELINE_N
    sec = oracle_build_seconds(cfg, n_s)
    multi, msec, cores = oracle_all_cores(cfg, n_s)
    return {"value": round(n_s / sec, 1), "unit": "points/s", "cores": 1, "kind": "oracle",
            "sample": "whole build (same k, leaf_max, passes, rounds, iters) of the first recipe draw at "
                      "n=%d instead of %d points; %.1f s single-threaded" % (n_s, cfg["n"], sec),
            "host_cpus": os.cpu_count(),
            "all_cores": {"value": round(multi, 1), "unit": "points/s", "cores": cores,
                          "sample": "%d independent whole builds of n=%d draws of the recipe at once, one host "
                                    "thread each; %.1f s wall" % (cores, n_s, msec)}}


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
PRECISIONS = {"fp32": 0, "bf16": 1, "fp16": 2, "fp8": 3}


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
        # every call is synchronous (host work around each): five calls
        # timed one by one, the median kept, so that one host stall does not
        # set the figure
        times = []
        with torch.cuda.stream(stream):
            knng.knng_search(Xd, G, Qd, Sd, t0, ks, stream=stream)
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ids, _d = knng.knng_search(Xd, G, Qd, Sd, t0, ks, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
        ms = float(np.median(times))
        got = ids.cpu().numpy()[check]
        r1 = float(np.mean([got[i, 0] == truth[i][0] for i in range(n_check)]))
        rk = float(np.mean([len(set(got[i].tolist()) & set(truth[i].tolist())) / ks for i in range(n_check)]))
        out[name] = {"queries_per_s": round(m / (ms * 1e-3), 1), "ms": round(ms, 3), "recall_at_1": round(r1, 4),
                     "recall_at_ks": round(rk, 4)}
        if name == "ivf_seeds":   # seeds and search together
            out[name]["queries_per_s_with_seeds"] = round(m / ((ms + seeds_ms) * 1e-3), 1)
    return out


def event_time(stream, fn, reps):
    """CUDA-event time (ms) of `reps` calls of fn on `stream` (after the caller's warm-up)."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def sampled_measure(knng, Xd, cfg, base_params, gi, gd, smp_d, stream, steps, full):
    """The sampled refinement round (nearest-neighbour descent with sampling,
    the prior art Sec. 1 cites) in place of the full local join: the same
    build with ms = k/2 and k/4 samples per list, direct knng_build_ex calls
    timed with CUDA events; `full` = the full round's direct form."""
    import torch
    n, k = Xd.shape[0], cfg["k"]
    out = {"full_fwd_rev": full, "how": "knng_build_ex per step, join_mode KNNG_JOIN_SAMPLED, same passes, rounds, "
                                        "seed and precision as the headline"}
    ids = torch.empty((n, k), dtype=torch.int32, device=Xd.device)
    dists = torch.empty((n, k), dtype=torch.float32, device=Xd.device)
    for ms in sorted({max(1, k // 2), max(1, k // 4)}, reverse=True):
        p = knng.default_params(**{f: getattr(base_params, f) for f, _ in base_params._fields_})
        p.join_mode = knng.KNNG_JOIN_SAMPLED
        p.sample = ms
        with torch.cuda.stream(stream):
            knng.knng_build_ex(Xd, p, stream=stream, out=(ids, dists))
        ms_t = event_time(stream, lambda: knng.knng_build_ex(Xd, p, stream=stream, out=(ids, dists)), steps)
        r_ids, r_tie = knng.knng_recall(ids, dists, gi, gd, smp_d)
        out["ms_%d" % ms] = {"value": round(n * steps / (ms_t * 1e-3), 1), "ms_per_step": round(ms_t / steps, 3),
                             "recall_ids": round(r_ids, 5), "recall_tie": round(r_tie, 5)}
    return out


# Every other workload of the scope table, measured in the same run: its
# forms (low precision first), event-timed steps, and the oracle's sample
# size for its single-threaded CPU baseline.
OTHER_CONFIGS = [
    ("gmm-10k-d32", ["fp32"], 10_000),
    ("gist-like-1m-d960", ["fp16", "fp32"], 1_500),
    ("unit-10m-d96", ["fp8", "bf16", "fp32"], 10_000),
]


def measure_config(knng, name, forms, cpu_n, steps, dev, stream, recall_rows=2000):
    """One workload: for each form, `steps` direct builds timed with CUDA
    events after one warm-up, a further build with events around every launch
    (per-kernel times, the dominant kernel's roofline, the certificate's
    fallback rows), recall@k against exact lists on sampled rows and the
    distance error against FP64; the graphs of the forms compared; the oracle
    timed single-threaded on a bounded draw of the same recipe."""
    import torch
    cfg = workload_config(name, forms[0])
    t0 = time.perf_counter()
    X = datagen.make(name)
    gen_s = time.perf_counter() - t0
    n, D = X.shape
    k = cfg["k"]
    Xd = torch.from_numpy(X).to(dev)
    smp = datagen.sample_rows(n, recall_rows, seed=3)
    smp_d = torch.from_numpy(smp).to(dev)
    gi, gd = knng.knng_exact(Xd, k, smp_d)
    out = {"n": n, "D": D, "k": k, "leaf_max": cfg["leaf_max"], "tree_passes": cfg["tree_passes"],
           "refine_rounds": cfg["refine_rounds"], "generator": cfg["generator"], "seed": cfg["seed"],
           "l2": cfg["l2"], "steps": steps, "forms": {}, "datagen_s": round(gen_s, 1)}
    first = None
    for prec in forms:
        p = knng.default_params(k=k, leaf_max=cfg["leaf_max"], tree_passes=cfg["tree_passes"],
                                refine_rounds=cfg["refine_rounds"], join_mode=knng.KNNG_JOIN_FWD_REV,
                                twomeans_iters=cfg["twomeans_iters"], seed=cfg["seed"], precision=PRECISIONS[prec])
        ids = torch.empty((n, k), dtype=torch.int32, device=dev)
        dists = torch.empty((n, k), dtype=torch.float32, device=dev)
        with torch.cuda.stream(stream):
            knng.knng_build_ex(Xd, p, stream=stream, out=(ids, dists))
        ms_direct = event_time(stream, lambda: knng.knng_build_ex(Xd, p, stream=stream, out=(ids, dists)), steps)
        # the timed number: replays of the build recorded into a CUDA graph
        # (as the headline), so that no host work sits between the kernels
        plan = knng.BuildPlan(Xd, p, stream=stream)
        with torch.cuda.stream(stream):
            plan.launch()
        plan.check()
        ms = event_time(stream, plan.launch, steps)
        plan.check()
        replay_same = bool(torch.equal(plan.ids, ids) and torch.equal(plan.dists, dists))
        plan.close()
        knng.stats_reset()
        knng.stats_enable(True, timing=True)
        ms_k = event_time(stream, lambda: knng.knng_build_ex(Xd, p, stream=stream, out=(ids, dists)), 1)
        knng.stats_enable(False)
        st = knng.stats()
        roof = roofline(st, None, name, 1)
        roof["share_of_step"] = round(st[roof["kernel"]]["ms"] / ms_k, 4)
        leaf = [v for key, v in st.items() if key.startswith("k2_leaf_") and key != "k2_leaf_fp32"]
        r_ids, r_tie = knng.knng_recall(ids, dists, gi, gd, smp_d)
        form = {"value": round(n * steps / (ms * 1e-3), 1), "unit": "points/s", "ms_per_step": round(ms / steps, 3),
                "timed": "CUDA-graph replays of the recorded build", "replay_equals_direct": replay_same,
                "direct_ms_per_step": round(ms_direct / steps, 3),
                "recall_ids": round(r_ids, 5), "recall_tie": round(r_tie, 5), "recall_rows": int(len(smp)),
                "distance_error": distance_error(X, ids, dists, smp[:500]),
                "roofline": roof,
                "whole_build_roofline": whole_build_roofline(st, None, 1, ms / steps),
                "kernels_ms": {key: round(v["ms"], 3) for key, v in sorted(st.items(), key=lambda kv: -kv[1]["ms"])[:6]}}
        if leaf:
            form["certificate_fallback_rows"] = {"rows": int(leaf[0]["items"]), "of": n * cfg["tree_passes"],
                                                 "rate": round(leaf[0]["items"] / (n * cfg["tree_passes"]), 4)}
        out["forms"][prec] = form
        if first is None:
            first = (ids, dists)
        else:
            form["graph_identical_to_%s" % forms[0]] = bool(torch.equal(first[0], ids) and torch.equal(first[1], dists))
    sec = oracle_build_seconds(cfg, cpu_n)
    out["cpu_baseline"] = {"value": round(cpu_n / sec, 1), "unit": "points/s", "cores": 1, "kind": "oracle",
                           "sample": "whole build (same parameters) of an n=%d draw of the recipe; %.1f s" % (cpu_n, sec)}
    del Xd, first
    torch.cuda.empty_cache()
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

    sampled = None
    if world == 1:
        sampled = sampled_measure(knng, Xd, cfg, params(args.precision), gi, gd, smp_d, stream, args.steps,
                                  {"value": direct["value"], "ms_per_step": direct["ms_per_step"],
                                   "recall_ids": round(rec_ids, 5), "recall_tie": round(rec_tie, 5)})

    # end to end: page-locked host buffers through the C ABI, copies inside
    # the timed region.  Two calls a user makes: the recorded build over the
    # host buffers (knng_plan_create once, outside the timed region; every
    # replay copies the rows in and the lists out inside its graph, and
    # knng_plan_check waits for them), and knng_build_ex on the same buffers.
    p = params(args.precision)
    Xh = torch.from_numpy(X).pin_memory()

    def host_steps(step):
        barrier()
        step_s = []
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            t1 = time.perf_counter()
            step()
            step_s.append(time.perf_counter() - t1)
        return max_over_ranks(time.perf_counter() - t0), step_s

    oi = torch.empty((n, cfg["k"]), dtype=torch.int32).pin_memory()
    od = torch.empty((n, cfg["k"]), dtype=torch.float32).pin_memory()
    for _ in range(2):   # warm: the workspace pool grows to the host-buffer call's size
        knng.knng_build_ex(Xh, p, stream=stream, out=(oi, od))
    direct_s, direct_steps = host_steps(lambda: knng.knng_build_ex(Xh, p, stream=stream, out=(oi, od)))
    same_direct = bool(torch.equal(oi, ids.cpu()) and torch.equal(od, dists.cpu()))
    torch.cuda.synchronize()
    hplan = knng.BuildPlan(Xh, p, stream=stream)
    for _ in range(2):
        hplan.launch()
        hplan.check()

    def plan_step():
        hplan.launch()
        hplan.check()  # waits for the stream: the lists are in host memory

    e2e_s, step_s = host_steps(plan_step)
    same = bool(torch.equal(hplan.ids, ids.cpu()) and torch.equal(hplan.dists, dists.cpu())) and same_direct
    e2e = {"value": round(replicas.aggregate(n, args.e2e_steps, e2e_s, world), 1), "unit": "points/s",
           "h2d_bytes_per_step": int(X.nbytes), "d2h_bytes_per_step": int(oi.numel() * 4 + od.numel() * 4),
           "steps": args.e2e_steps, "step_ms": [round(t * 1e3, 2) for t in step_s],
           "timer": "host wall clock around each replay and the wait for it",
           "how": "knng_plan_launch + knng_plan_check of a build recorded over page-locked host buffers",
           "direct": {"value": round(replicas.aggregate(n, args.e2e_steps, direct_s, world), 1),
                      "step_ms": [round(t * 1e3, 2) for t in direct_steps],
                      "how": "knng_build_ex on the same host buffers (synchronous)"}}
    hplan.close()

    if rank != 0:
        replicas.finish()
        return
    roof = roofline(st, clk, cfg["workload"], args.steps)
    whole = whole_build_roofline(st, clk, args.steps, ms / args.steps)
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
        "roofline": roof, "roofline_other_kernels": others, "whole_build_roofline": whole,
        "distance_error": dist_err, "e2e": e2e, "e2e_graph_equals_device_graph": same, "gpu_launches": int(launches),
        "clocks": clk,
        "kernels": {k_: {"ms_per_step": round(v["ms"] / args.steps, 3), "launches_per_step": v["launches"] / args.steps}
                    for k_, v in sorted(st.items(), key=lambda kv: -kv[1]["ms"])[:10]},
        "kernel_breakdown_run": {"ms_per_step": round(ms_k / args.steps, 3),
                                 "note": "a second run of the same steps with CUDA events around every launch; "
                                         "the per-kernel times, shares and rooflines come from it"},
    }
    if sampled is not None:
        line["sampled"] = sampled
    if world == 1 and not args.no_search:
        line["search"] = search_measure(knng, X, Xd, ids, dev, stream)
    if world == 1 and not args.no_configs:
        del Xd, Xh
        torch.cuda.empty_cache()
        configs = {}
        for name, forms, cpu_n in OTHER_CONFIGS:
            configs[name] = measure_config(knng, name, forms, cpu_n, args.config_steps, dev, stream)
        configs[datagen.BATCHED["name"]] = batched_measure(knng, args.config_steps, 1, "bf16")
        line["configs"] = configs
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cfg)
    print(json.dumps(line), flush=True)
    replicas.finish()


def batched_measure(knng, steps, warmup, precision, local=0):
    """The batched workload: 64 independent instances recorded once into a
    CUDA graph (knng_plan_create_batched) and replayed once per step, each D
    group's leaf tile shape (leaf_max) and split schedule (twomeans_iters)
    from the autotuner (its time not counted); the low-precision form against
    FP32, graphs compared; direct knng_build_batched calls timed beside."""
    import torch
    from paper_1701_08475_gb300.autotune import autotune

    w = datagen.BATCHED
    datas = datagen.batched_mixtures(n_inst=w["n_inst"], seed=w["seed"] + local)
    n_tot = sum(x.shape[0] for x in datas)
    dev = [torch.from_numpy(x).cuda() for x in datas]
    prec = PRECISIONS[precision]
    p = knng.default_params(k=w["k"], leaf_max=128, tree_passes=w["passes"], refine_rounds=w["rounds"],
                            join_mode=knng.KNNG_JOIN_FWD_REV, seed=w["seed"], precision=prec)
    leafs, iters, report = autotune(dev, p)
    stream = torch.cuda.Stream()

    def replayed(q):
        plan = knng.BatchedPlan(dev, q, leaf_maxes=leafs, twomeans_iters=iters, stream=stream)
        with torch.cuda.stream(stream):
            for _ in range(max(1, warmup)):
                plan.launch()
        plan.check()
        ms = event_time(stream, plan.launch, steps)
        plan.check()
        outs = [(a.clone(), b.clone()) for a, b in plan.outs]
        kernels = plan.kernels
        plan.close()
        return ms, outs, kernels

    def direct(q):
        with torch.cuda.stream(stream):
            outs = knng.knng_build_batched(dev, q, leaf_maxes=leafs, twomeans_iters=iters, stream=stream)
        knng.stats_reset()
        knng.stats_enable(True, timing=False)
        ms = event_time(stream, lambda: knng.knng_build_batched(dev, q, leaf_maxes=leafs, twomeans_iters=iters,
                                                                 stream=stream), steps)
        launches = sum(v["launches"] for v in knng.stats().values())
        knng.stats_enable(False)
        return ms, launches

    ms, outs, kernels = replayed(p)
    ms_d, launches_d = direct(p)
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
    ms32, outs32, _ = replayed(q32)
    same = all(torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]) for a, b in zip(outs, outs32))
    return {
        "value": round(n_tot * steps / (ms * 1e-3), 1), "unit": "points/s", "steps": steps,
        "ms_per_step": round(ms / steps, 3),
        "dtype": "f32" if precision == "fp32" else precision + "+f32",
        "config": {"workload": w["name"], "instances": len(datas), "points": int(n_tot), "k": w["k"],
                   "tree_passes": w["passes"], "refine_rounds": w["rounds"], "precision": precision,
                   "leaf_max_by_D": {str(x.shape[1]): l for x, l in zip(datas, leafs)},
                   "twomeans_iters_by_D": {str(x.shape[1]): t for x, t in zip(datas, iters)},
                   "autotune": {str(D): rows for D, rows in report.items()}},
        "recall_at_k": {"ids": round(hit / tot, 5), "sample_rows": int(tot)},
        "fp32_form": {"value": round(n_tot * steps / (ms32 * 1e-3), 1), "ms_per_step": round(ms32 / steps, 3),
                      "graph_identical": bool(same)},
        "direct_form": {"value": round(n_tot * steps / (ms_d * 1e-3), 1), "ms_per_step": round(ms_d / steps, 3),
                        "gpu_launches": int(launches_d), "how": "knng_build_batched per step"},
        "gpu_launches": int(kernels * steps),
        "timed": "CUDA-graph replays of the recorded batched build (knng_plan_create_batched, knng_plan_launch)",
    }


def run_batched(args):
    import torch
    import paper_1701_08475_gb300 as knng

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    knng.load()
    m = batched_measure(knng, args.steps, args.warmup, args.precision, local=rank)
    line = {"metric": "kNN-graph build points/s at recall@k vs exact", "value": m["value"], "unit": "points/s",
            "n_gpus": 1, "steps": args.steps, "warmup": max(1, args.warmup), "ms_per_step": m["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": m["dtype"],
            "data": "synthetic", "config": m["config"], "recall_at_k": m["recall_at_k"],
            "fp32_form": m["fp32_form"], "gpu_launches": m["gpu_launches"]}
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
    cfg = workload_config(args.workload, args.precision)
    if args.impl == "reference":
        run_reference(args, cfg)
    else:
        run_ours(args, cfg)


if __name__ == "__main__":
    main()
