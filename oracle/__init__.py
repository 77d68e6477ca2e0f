"""CPU oracle for kNN-graph construction (arXiv 1701.08475, Sec. 3.1, Alg. 1),
the graph search (Sec. 3.2, Alg. 2) and its residue-quantisation inverted index
(Sec. 4).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The oracle shares no code
with the CUDA library in ``paper_1701_08475_gb300`` and never loads it.

The arithmetic lives in ``knng_oracle.c`` (plain C, single thread); this module
compiles it with gcc on first use and marshals numpy arrays through ctypes.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "knng_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

FWD = 0
FWD_REV = 1


def build(force=False):
    """Compile the oracle with gcc (-O2, no floating-point contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    P = ctypes.c_void_p
    i64, i32, u64 = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64
    sig = {
        "orc_splitmix64": (u64, [u64]),
        "orc_pass_seed": (u64, [u64, i32]),
        "orc_init_positions": (None, [u64, i32, i64, i64, P, P]),
        "orc_dist_f32": (ctypes.c_float, [P, P, i32]),
        "orc_dist_f64": (ctypes.c_double, [P, P, i32]),
        "orc_list_insert": (None, [P, P, i32, ctypes.c_float, ctypes.c_int32]),
        "orc_exact_f32": (i32, [P, i64, i32, i32, P, i64, P, P]),
        "orc_exact_f64": (i32, [P, i64, i32, i32, P, i64, P, P]),
        "orc_tree_depth": (i32, [i64, i32]),
        "orc_partition": (i32, [P, i64, i32, i32, i32, u64, i32, P, P]),
        "orc_leaf_update": (i32, [P, i64, i32, i32, P, P, i64, P, P]),
        "orc_reverse_lists": (i32, [i64, i32, P, P, P, P]),
        "orc_refine_round": (i32, [P, i64, i32, i32, i32, P, P]),
        "orc_build": (i32, [P, i64, i32, i32, i32, i32, i32, i32, i32, u64, P, P]),
        "orc_recall": (i32, [P, P, P, P, P, i64, i32, P, P]),
        "orc_search": (i32, [P, i64, i32, P, i32, P, i64, P, i32, i32, i32, P, P]),
        "orc_sample_prio": (u64, [u64, i32, i64, ctypes.c_int32]),
        "orc_build_sampled": (i32, [P, i64, i32, i32, i32, i32, i32, i32, i32, u64, P, P]),
        "orc_refine_sampled": (i64, [P, i64, i32, i32, i32, u64, i32, P, P, P]),
        "orc_rvq_init_positions": (None, [i64, i32, u64, i32, P]),
        "orc_rvq_assign": (i32, [P, i64, i32, P, i32, P]),
        "orc_rvq_train": (i32, [P, i64, i32, i32, i32, i32, u64, P, P]),
        "orc_rvq_index": (i32, [P, i64, i32, P, i32, P, i32, P, P, P]),
        "orc_rvq_seeds": (i32, [P, i32, P, i32, i32, P, P, P, i64, i32, i32, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
        return _lib


def compile_variant(src_text, out_path):
    """Compile a variant of the oracle source (used by the tests that plant
    mistakes in the oracle to show that the pins catch them)."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                    "-fPIC", "-shared", "-o", out_path, src, "-lm"], check=True)
    return _bind(ctypes.CDLL(out_path))


def source_text():
    with open(_SRC) as f:
        return f.read()


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def splitmix64(z):
    return int(_load().orc_splitmix64(ctypes.c_uint64(z & (2**64 - 1))))


def pass_seed(seed, p):
    return int(_load().orc_pass_seed(seed & (2**64 - 1), p))


def init_positions(pass_seed_, level, seg, m):
    h = ctypes.c_int64()
    h2 = ctypes.c_int64()
    _load().orc_init_positions(pass_seed_ & (2**64 - 1), level, seg, m,
                               ctypes.byref(h), ctypes.byref(h2))
    return h.value, h2.value


def dist_f32(x, y):
    x, y = _f32(x), _f32(y)
    return float(_load().orc_dist_f32(_p(x), _p(y), x.shape[-1]))


def dist_f64(x, y):
    x, y = _f32(x), _f32(y)
    return float(_load().orc_dist_f64(_p(x), _p(y), x.shape[-1]))


def new_graph(n, k):
    """An empty graph: every slot (id -1, d +inf)."""
    return np.full((n, k), -1, np.int32), np.full((n, k), np.inf, np.float32)


def list_insert(ids_row, d_row, cd, cid):
    """Offer (cd, cid) to one sorted unique list, in place."""
    assert ids_row.flags.c_contiguous and d_row.flags.c_contiguous
    _load().orc_list_insert(_p(ids_row), _p(d_row), ids_row.shape[0],
                            ctypes.c_float(cd), int(cid))


def exact_f32(X, k, sample=None):
    X = _f32(X)
    n, D = X.shape
    s = n if sample is None else len(sample)
    sample = None if sample is None else _i32(sample)
    ids = np.empty((s, k), np.int32)
    d = np.empty((s, k), np.float32)
    _load().orc_exact_f32(_p(X), n, D, k, _p(sample), s, _p(ids), _p(d))
    return ids, d


def exact_f64(X, k, sample=None):
    X = _f32(X)
    n, D = X.shape
    s = n if sample is None else len(sample)
    sample = None if sample is None else _i32(sample)
    ids = np.empty((s, k), np.int32)
    d = np.empty((s, k), np.float64)
    _load().orc_exact_f64(_p(X), n, D, k, _p(sample), s, _p(ids), _p(d))
    return ids, d


def tree_depth(n, leaf_max):
    return int(_load().orc_tree_depth(n, leaf_max))


def partition(X, leaf_max, iters=4, seed=0, pass_=0):
    """(perm, leaf_offsets) of one tree pass."""
    X = _f32(X)
    n, D = X.shape
    L = tree_depth(n, leaf_max)
    perm = np.empty(n, np.int32)
    off = np.empty((1 << L) + 1, np.int64)
    r = _load().orc_partition(_p(X), n, D, leaf_max, iters, seed & (2**64 - 1),
                              pass_, _p(perm), _p(off))
    if r < 0:
        raise ValueError("orc_partition: bad arguments")
    return perm, off


def leaf_update(X, k, perm, leaf_offsets, ids=None, dists=None):
    """Apply the leaf stage of one partition to (ids, dists); returns new arrays."""
    X = _f32(X)
    n, D = X.shape
    if ids is None:
        ids, dists = new_graph(n, k)
    ids = np.array(ids, np.int32, order="C", copy=True)
    dists = np.array(dists, np.float32, order="C", copy=True)
    perm = _i32(perm)
    off = np.ascontiguousarray(leaf_offsets, dtype=np.int64)
    _load().orc_leaf_update(_p(X), n, D, k, _p(perm), _p(off), len(off) - 1,
                            _p(ids), _p(dists))
    return ids, dists


def reverse_lists(ids, dists):
    ids = _i32(ids)
    dists = _f32(dists)
    n, k = ids.shape
    rid = np.empty_like(ids)
    rd = np.empty_like(dists)
    _load().orc_reverse_lists(n, k, _p(ids), _p(dists), _p(rid), _p(rd))
    return rid, rd


def refine_round(X, ids, dists, mode=FWD_REV):
    X = _f32(X)
    n, D = X.shape
    ids = np.array(ids, np.int32, order="C", copy=True)
    dists = np.array(dists, np.float32, order="C", copy=True)
    k = ids.shape[1]
    if _load().orc_refine_round(_p(X), n, D, k, mode, _p(ids), _p(dists)) != 0:
        raise MemoryError("orc_refine_round")
    return ids, dists


def sample_prio(seed, round_, v, u):
    """Sampling priority h(v, u) of the sampled refinement round."""
    return int(_load().orc_sample_prio(seed & (2**64 - 1), round_, v, u))


def refine_sampled(X, ids, dists, flags, ms, seed=0, round_=0):
    """One sampled refinement round (nearest-neighbour descent with sampling,
    ms samples per list): (ids, dists, flags, entries that entered a list).
    flags: n x k uint8, 1 = new."""
    X = _f32(X)
    n, D = X.shape
    ids = np.array(ids, np.int32, order="C", copy=True)
    dists = np.array(dists, np.float32, order="C", copy=True)
    flags = np.array(flags, np.uint8, order="C", copy=True)
    k = ids.shape[1]
    r = _load().orc_refine_sampled(_p(X), n, D, k, ms, seed & (2**64 - 1), round_, _p(ids), _p(dists), _p(flags))
    if r < 0:
        raise ValueError("orc_refine_sampled failed: %d" % r)
    return ids, dists, flags, int(r)


def build_graph(X, k, leaf_max, passes=1, rounds=0, iters=4, mode=FWD_REV, seed=0):
    """The whole build: passes of Alg. 1, then refinement rounds."""
    X = _f32(X)
    n, D = X.shape
    ids = np.empty((n, k), np.int32)
    d = np.empty((n, k), np.float32)
    r = _load().orc_build(_p(X), n, D, k, leaf_max, passes, rounds, iters, mode,
                          seed & (2**64 - 1), _p(ids), _p(d))
    if r != 0:
        raise ValueError("orc_build: bad arguments")
    return ids, d


def build_graph_sampled(X, k, leaf_max, passes=1, rounds=0, iters=4, ms=None, seed=0):
    """The whole build with sampled refinement rounds (ms samples per list,
    default k // 2), every entry flagged new before the first round."""
    X = _f32(X)
    n, D = X.shape
    ms = k // 2 if ms is None else ms
    ids = np.empty((n, k), np.int32)
    d = np.empty((n, k), np.float32)
    r = _load().orc_build_sampled(_p(X), n, D, k, leaf_max, passes, rounds, iters, ms, seed & (2**64 - 1),
                                  _p(ids), _p(d))
    if r != 0:
        raise ValueError("orc_build_sampled: bad arguments")
    return ids, d


def recall(ids, dists, gt_ids, gt_d, sample):
    ids, dists = _i32(ids), _f32(dists)
    gt_ids, gt_d, sample = _i32(gt_ids), _f32(gt_d), _i32(sample)
    k = ids.shape[1]
    ri = ctypes.c_double()
    rt = ctypes.c_double()
    _load().orc_recall(_p(ids), _p(dists), _p(gt_ids), _p(gt_d), _p(sample),
                       len(sample), k, ctypes.byref(ri), ctypes.byref(rt))
    return ri.value, rt.value


def search(X, G, Q, S, t0, ks):
    """Enhanced hill-climbing search (Sec. 3.2, Alg. 2) of queries Q (m x D)
    over the graph G (n x k ids, -1 empty) from seeds S (m x s ids), t0
    iterations, ks results per query: (ids m x ks, dists m x ks)."""
    X, Q = _f32(X), _f32(Q)
    G, S = _i32(G), _i32(S)
    n, D = X.shape
    m = Q.shape[0]
    ids = np.empty((m, ks), np.int32)
    d = np.empty((m, ks), np.float32)
    rc = _load().orc_search(_p(X), n, D, _p(G), G.shape[1], _p(Q), m, _p(S), S.shape[1], t0, ks, _p(ids), _p(d))
    if rc != 0:
        raise ValueError("orc_search failed: %d" % rc)
    return ids, d


def rvq_init_positions(N, W, seed, stage):
    """Initial word positions of one stage (one SplitMix64 draw per stratum)."""
    pos = np.empty(W, np.int64)
    _load().orc_rvq_init_positions(N, W, seed & (2**64 - 1), stage, _p(pos))
    return pos


def rvq_assign(V, words):
    """Nearest word of every row of V (canonical FP32, ties to the smaller index)."""
    V, words = _f32(V), _f32(words)
    codes = np.empty(V.shape[0], np.int32)
    if _load().orc_rvq_assign(_p(V), V.shape[0], V.shape[1], _p(words), words.shape[0], _p(codes)) != 0:
        raise ValueError("orc_rvq_assign: bad arguments")
    return codes


def rvq_train(X, W1=256, W2=256, iters=10, seed=0):
    """Two-stage residue vector quantisation vocabularies (Sec. 4.1, Eqn. 1):
    (w1 W1 x D, w2 W2 x D), Lloyd's k-means per stage."""
    X = _f32(X)
    n, D = X.shape
    w1 = np.empty((W1, D), np.float32)
    w2 = np.empty((W2, D), np.float32)
    rc = _load().orc_rvq_train(_p(X), n, D, W1, W2, iters, seed & (2**64 - 1), _p(w1), _p(w2))
    if rc != 0:
        raise ValueError("orc_rvq_train failed: %d" % rc)
    return w1, w2


def rvq_index(X, w1, w2):
    """Codes (n x 2: c1, c2) and the inverted lists (offsets W1*W2 + 1, ids n)
    keyed by c1 * W2 + c2 (Sec. 4.2)."""
    X, w1, w2 = _f32(X), _f32(w1), _f32(w2)
    n, D = X.shape
    W1, W2 = w1.shape[0], w2.shape[0]
    codes = np.empty((n, 2), np.int32)
    off = np.empty(W1 * W2 + 1, np.int32)
    ids = np.empty(n, np.int32)
    rc = _load().orc_rvq_index(_p(X), n, D, _p(w1), W1, _p(w2), W2, _p(codes), _p(off), _p(ids))
    if rc != 0:
        raise ValueError("orc_rvq_index failed: %d" % rc)
    return codes, off, ids


def rvq_seeds(w1, w2, offsets, ids, Q, probe1, s):
    """Seeds of Alg. 2 from the inverted index (Sec. 4.2, Eqns. 2 and 3):
    m x s ids, -1 padded."""
    w1, w2, Q = _f32(w1), _f32(w2), _f32(Q)
    offsets, ids = _i32(offsets), _i32(ids)
    W1, D = w1.shape
    W2 = w2.shape[0]
    m = Q.shape[0]
    S = np.empty((m, s), np.int32)
    rc = _load().orc_rvq_seeds(_p(w1), W1, _p(w2), W2, D, _p(offsets), _p(ids), _p(Q), m, probe1, s, _p(S))
    if rc != 0:
        raise ValueError("orc_rvq_seeds failed: %d" % rc)
    return S
