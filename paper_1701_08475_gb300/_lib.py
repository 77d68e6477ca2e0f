"""ctypes binding of libknng.so (the C ABI of include/knng.h).

Argument marshalling only: tensors and arrays become pointers and sizes,
outputs are allocated like the input (same device; numpy in, numpy out), and
errors become KnngError.  If the CUDA library is missing the import of a
function fails loudly; there is no fallback.
"""
import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libknng.so")
_lock = threading.Lock()
_lib = None

KNNG_JOIN_FWD = 0
KNNG_JOIN_FWD_REV = 1
KNNG_JOIN_SAMPLED = 2
KNNG_FP32 = 0
KNNG_BF16 = 1
KNNG_FP16 = 2
KNNG_FP8 = 3

_CODES = {-1: "KNNG_EINVAL", -2: "KNNG_ENOMEM", -3: "KNNG_ECUDA", -4: "KNNG_ETIMEOUT"}


class KnngError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (_CODES.get(code, "error"), code, msg))
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("leaf_max", ctypes.c_int), ("tree_passes", ctypes.c_int),
                ("refine_rounds", ctypes.c_int), ("join_mode", ctypes.c_int), ("precision", ctypes.c_int),
                ("twomeans_iters", ctypes.c_int), ("seed", ctypes.c_uint64), ("sample", ctypes.c_int)]


class Instance(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("n", ctypes.c_int64), ("D", ctypes.c_int), ("leaf_max", ctypes.c_int),
                ("out_ids", ctypes.c_void_p), ("out_dists", ctypes.c_void_p), ("twomeans_iters", ctypes.c_int)]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_uint64), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("flops", ctypes.c_double), ("items", ctypes.c_double)]


def library_path():
    return _LIB_PATH


def load():
    """Load libknng.so (built by __graft_entry__.build() or build.py)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise ImportError("libknng.so is not built (run __graft_entry__.build()); no fallback exists")
        lib = ctypes.CDLL(_LIB_PATH)
        P, i64, i32, u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint64
        PP = ctypes.POINTER(Params)
        sig = {
            "knng_default_params": (None, [PP]),
            "knng_build": (i32, [P, i64, i32, i32, i32, i32, u64, P, P]),
            "knng_build_ex": (i32, [P, i64, i32, PP, P, P, P]),
            "knng_build_batched": (i32, [i32, ctypes.POINTER(Instance), PP, P]),
            "knng_plan_create": (i32, [P, i64, i32, PP, P, P, P, ctypes.POINTER(ctypes.c_void_p)]),
            "knng_plan_create_batched": (i32, [i32, ctypes.POINTER(Instance), PP, P, ctypes.POINTER(ctypes.c_void_p)]),
            "knng_plan_launch": (i32, [P, P]),
            "knng_plan_kernels": (i64, [P]),
            "knng_plan_check": (i32, [P, P]),
            "knng_plan_destroy": (None, [P]),
            "knng_refine": (i32, [P, i64, i32, PP, P, P, P]),
            "knng_partition": (i32, [P, i64, i32, i32, i32, u64, i32, P, P, P]),
            "knng_tree_depth": (i32, [i64, i32]),
            "knng_leaf_update": (i32, [P, i64, i32, i32, P, P, i64, P, P, P]),
            "knng_leaf_dhat": (i32, [P, i64, i32, i32, P, P, P, P, P, P]),
            "knng_exact": (i32, [P, i64, i32, i32, P, i64, P, P, P]),
            "knng_search": (i32, [P, i64, i32, P, i32, P, i64, P, i32, i32, i32, P, P, P]),
            "knng_rvq_train": (i32, [P, i64, i32, i32, i32, i32, u64, P, P, P]),
            "knng_rvq_index": (i32, [P, i64, i32, P, i32, P, i32, P, P, P, P]),
            "knng_rvq_seeds": (i32, [P, i32, P, i32, i32, P, P, i64, P, i64, i32, i32, P, P]),
            "knng_exact_noalloc": (i32, [P, i64, i32, i32, P, i64, P, P, P]),
            "knng_recall": (i32, [P, P, P, P, P, i64, i32, P, P, P]),
            "knng_last_error": (ctypes.c_char_p, []),
            "knng_workspace_bytes": (ctypes.c_size_t, [i64, i32, PP]),
            "knng_stats_enable": (i32, [i32, i32]),
            "knng_stats_reset": (None, []),
            "knng_stats_count": (i32, []),
            "knng_stats_get": (i32, [i32, ctypes.POINTER(KernelStat)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _check(code):
    if code != 0:
        raise KnngError(code, load().knng_last_error().decode())


# ---------------------------------------------------------------- marshalling
def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    if x is None:
        return None
    if _is_torch(x):
        return ctypes.c_void_p(x.data_ptr())
    return x.ctypes.data_as(ctypes.c_void_p)


def _contig(x, dtype_name):
    """x as a C-contiguous array of the named dtype (torch stays torch)."""
    if _is_torch(x):
        import torch
        dt = {"float32": torch.float32, "int32": torch.int32, "int64": torch.int64}[dtype_name]
        if x.dtype != dt:
            raise TypeError("expected %s, got %s" % (dt, x.dtype))
        return x.contiguous()
    a = np.ascontiguousarray(x)
    if a.dtype != np.dtype(dtype_name):
        raise TypeError("expected %s, got %s" % (dtype_name, a.dtype))
    return a


def _empty_like_input(x, shape, dtype_name):
    if _is_torch(x):
        import torch
        dt = {"float32": torch.float32, "int32": torch.int32, "int64": torch.int64}[dtype_name]
        return torch.empty(shape, dtype=dt, device=x.device, pin_memory=False)
    return np.empty(shape, dtype=dtype_name)


class _DeviceCtx:
    """Make x's CUDA device current and pick its current stream."""

    def __init__(self, x, stream):
        self.x, self.stream, self.ctx = x, stream, None

    def __enter__(self):
        s = self.stream
        if _is_torch(self.x) and self.x.is_cuda:
            import torch
            self.ctx = torch.cuda.device(self.x.device)
            self.ctx.__enter__()
            if s is None:
                s = torch.cuda.current_stream(self.x.device).cuda_stream
        elif s is not None and hasattr(s, "cuda_stream"):
            s = s.cuda_stream
        if s is not None and hasattr(s, "cuda_stream"):
            s = s.cuda_stream
        return ctypes.c_void_p(s) if s else None

    def __exit__(self, *a):
        if self.ctx is not None:
            self.ctx.__exit__(*a)


def default_params(**kw):
    p = Params()
    load().knng_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


# ---------------------------------------------------------------- entry points
def knng_build(data, k, leaf_max, rounds=1, seed=0):
    """Alg. 1 with `rounds` tree passes, FP32, no refinement; returns (ids, dists)."""
    data = _contig(data, "float32")
    n, D = data.shape
    ids = _empty_like_input(data, (n, k), "int32")
    d = _empty_like_input(data, (n, k), "float32")
    with _DeviceCtx(data, None):
        if _is_torch(data) and data.is_cuda:
            import torch
            torch.cuda.current_stream(data.device).synchronize()   # knng_build runs on the default stream
        _check(load().knng_build(_ptr(data), n, D, k, leaf_max, rounds, seed & (2**64 - 1), _ptr(ids), _ptr(d)))
    return ids, d


def knng_build_ex(data, params, stream=None, out=None):
    """The whole build with explicit params; returns (ids, dists)."""
    data = _contig(data, "float32")
    n, D = data.shape
    k = params.k
    if out is None:
        ids = _empty_like_input(data, (n, k), "int32")
        d = _empty_like_input(data, (n, k), "float32")
    else:
        ids, d = out
    with _DeviceCtx(data, stream) as s:
        _check(load().knng_build_ex(_ptr(data), n, D, ctypes.byref(params), _ptr(ids), _ptr(d), s))
    return ids, d


def _instances(datas, k, leaf_maxes, iters=None):
    outs = [(_empty_like_input(x, (x.shape[0], k), "int32"), _empty_like_input(x, (x.shape[0], k), "float32"))
            for x in datas]
    arr = (Instance * len(datas))()
    for i, (x, (ids, d)) in enumerate(zip(datas, outs)):
        arr[i].data = _ptr(x).value
        arr[i].n = x.shape[0]
        arr[i].D = x.shape[1]
        arr[i].leaf_max = int(leaf_maxes[i])
        arr[i].out_ids = _ptr(ids).value
        arr[i].out_dists = _ptr(d).value
        arr[i].twomeans_iters = int(iters[i]) if iters is not None else 0
    return arr, outs


def knng_build_batched(datas, params, leaf_maxes=None, stream=None, twomeans_iters=None):
    """Independent graphs of several inputs in one build; returns a list of
    (ids, dists), ids local to each input.  leaf_maxes, twomeans_iters: per
    input (0: params')."""
    datas = [_contig(x, "float32") for x in datas]
    arr, outs = _instances(datas, params.k, leaf_maxes or [0] * len(datas), twomeans_iters)
    with _DeviceCtx(datas[0], stream) as s:
        _check(load().knng_build_batched(len(datas), arr, ctypes.byref(params), s))
    return outs


class BuildPlan:
    """A build recorded once into a CUDA graph (knng_plan_*): `launch()`
    replays it on `data` into (ids, dists); `check()` waits and raises on a
    device-reported error.  Torch tensors on the device, or page-locked
    host tensors (`pin_memory()`): then every replay copies `data` in and the
    lists out, and the outputs made here are page-locked too."""

    def __init__(self, data, params, stream=None, out=None):
        import torch
        self.data = _contig(data, "float32")
        n, D = self.data.shape
        if out is not None:
            self.ids, self.dists = out
        else:
            pin = not self.data.is_cuda
            self.ids = torch.empty((n, params.k), dtype=torch.int32, device=self.data.device, pin_memory=pin)
            self.dists = torch.empty((n, params.k), dtype=torch.float32, device=self.data.device, pin_memory=pin)
        self._plan = ctypes.c_void_p()
        self._stream = stream
        with _DeviceCtx(self.data, stream) as s:
            _check(load().knng_plan_create(_ptr(self.data), n, D, ctypes.byref(params), _ptr(self.ids),
                                           _ptr(self.dists), s, ctypes.byref(self._plan)))

    @property
    def kernels(self):
        """Kernel launches per replay."""
        return int(load().knng_plan_kernels(self._plan))

    def launch(self, stream=None):
        with _DeviceCtx(self.data, stream if stream is not None else self._stream) as s:
            _check(load().knng_plan_launch(self._plan, s))
        return self.ids, self.dists

    def check(self, stream=None):
        with _DeviceCtx(self.data, stream if stream is not None else self._stream) as s:
            _check(load().knng_plan_check(self._plan, s))

    def close(self):
        if self._plan:
            load().knng_plan_destroy(self._plan)
            self._plan = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class BatchedPlan(BuildPlan):
    """knng_build_batched recorded once into a CUDA graph
    (knng_plan_create_batched): `launch()` replays it on the instances'
    tensors into `outs` (a list of (ids, dists)).  Device tensors only."""

    def __init__(self, datas, params, leaf_maxes=None, stream=None, twomeans_iters=None):
        self.datas = [_contig(x, "float32") for x in datas]
        self.data = self.datas[0]
        arr, self.outs = _instances(self.datas, params.k, leaf_maxes or [0] * len(self.datas), twomeans_iters)
        self._plan = ctypes.c_void_p()
        self._stream = stream
        with _DeviceCtx(self.data, stream) as s:
            _check(load().knng_plan_create_batched(len(self.datas), arr, ctypes.byref(params), s,
                                                   ctypes.byref(self._plan)))

    def launch(self, stream=None):
        with _DeviceCtx(self.data, stream if stream is not None else self._stream) as s:
            _check(load().knng_plan_launch(self._plan, s))
        return self.outs


def knng_refine(data, ids, dists, params, stream=None):
    """Refinement rounds on (ids, dists), in place; returns them."""
    data = _contig(data, "float32")
    n, D = data.shape
    assert ids.shape == (n, params.k) and dists.shape == (n, params.k)
    ids = _contig(ids, "int32")
    dists = _contig(dists, "float32")
    with _DeviceCtx(data, stream) as s:
        _check(load().knng_refine(_ptr(data), n, D, ctypes.byref(params), _ptr(ids), _ptr(dists), s))
    return ids, dists


def knng_tree_depth(n, leaf_max):
    return int(load().knng_tree_depth(n, leaf_max))


def knng_partition(data, leaf_max, twomeans_iters=4, seed=0, pass_=0, stream=None):
    """(perm, leaf_offsets) of tree pass `pass_`."""
    data = _contig(data, "float32")
    n, D = data.shape
    L = knng_tree_depth(n, leaf_max)
    if L < 0:
        raise KnngError(-1, "bad leaf_max")
    perm = _empty_like_input(data, (n,), "int32")
    off = _empty_like_input(data, ((1 << L) + 1,), "int64")
    with _DeviceCtx(data, stream) as s:
        _check(load().knng_partition(_ptr(data), n, D, leaf_max, twomeans_iters, seed & (2**64 - 1), pass_,
                                     _ptr(perm), _ptr(off), s))
    return perm, off


def knng_leaf_update(data, k, perm, leaf_offsets, ids, dists, stream=None):
    """Leaf stage of Alg. 1 on a given partition, in place on (ids, dists)."""
    data = _contig(data, "float32")
    n, D = data.shape
    perm = _contig(perm, "int32")
    leaf_offsets = _contig(leaf_offsets, "int64")
    ids = _contig(ids, "int32")
    dists = _contig(dists, "float32")
    with _DeviceCtx(data, stream) as s:
        _check(load().knng_leaf_update(_ptr(data), n, D, k, _ptr(perm), _ptr(leaf_offsets), len(leaf_offsets) - 1,
                                       _ptr(ids), _ptr(dists), s))
    return ids, dists


def knng_leaf_dhat(data, precision, stream=None):
    """Parity hook of the low-precision leaf stage for one cluster (m <= 256
    points): (d^ m x m, q m x D, scales m, squared norms m, error bounds m)."""
    data = _contig(data, "float32")
    m, D = data.shape
    outs = (_empty_like_input(data, (m, m), "float32"), _empty_like_input(data, (m, D), "float32"),
            _empty_like_input(data, (m,), "float32"), _empty_like_input(data, (m,), "float32"),
            _empty_like_input(data, (m,), "float32"))
    with _DeviceCtx(data, stream) as s:
        _check(load().knng_leaf_dhat(_ptr(data), m, D, precision, *[_ptr(o) for o in outs], s))
    return outs


def knng_search(data, graph_ids, queries, seeds, t0, ks, stream=None):
    """Enhanced hill-climbing search (Sec. 3.2, Alg. 2) of `queries` (m x D)
    over the graph `graph_ids` (n x k ids) from `seeds` (m x s ids), t0
    iterations: (ids, dists), m x ks each."""
    data = _contig(data, "float32")
    graph_ids = _contig(graph_ids, "int32")
    queries = _contig(queries, "float32")
    seeds = _contig(seeds, "int32")
    n, D = data.shape
    m = queries.shape[0]
    ids = _empty_like_input(data, (m, ks), "int32")
    d = _empty_like_input(data, (m, ks), "float32")
    with _DeviceCtx(data, stream) as s:
        _check(load().knng_search(_ptr(data), n, D, _ptr(graph_ids), graph_ids.shape[1], _ptr(queries), m,
                                  _ptr(seeds), seeds.shape[1], t0, ks, _ptr(ids), _ptr(d), s))
    return ids, d


def knng_rvq_train(data, W1=256, W2=256, iters=10, seed=0, stream=None):
    """Two-stage residue vector quantisation vocabularies (Sec. 4.1, Eqn. 1),
    Lloyd's k-means per stage: (words1 W1 x D, words2 W2 x D)."""
    data = _contig(data, "float32")
    n, D = data.shape
    w1 = _empty_like_input(data, (W1, D), "float32")
    w2 = _empty_like_input(data, (W2, D), "float32")
    with _DeviceCtx(data, stream) as s:
        _check(load().knng_rvq_train(_ptr(data), n, D, W1, W2, iters, seed & (2**64 - 1), _ptr(w1), _ptr(w2), s))
    return w1, w2


def knng_rvq_index(data, words1, words2, stream=None):
    """The inverted index of Sec. 4.2: (codes n x 2, list_offsets W1*W2 + 1,
    list_ids n), lists keyed by c1 * W2 + c2, ids ascending."""
    data = _contig(data, "float32")
    words1 = _contig(words1, "float32")
    words2 = _contig(words2, "float32")
    n, D = data.shape
    W1, W2 = words1.shape[0], words2.shape[0]
    codes = _empty_like_input(data, (n, 2), "int32")
    off = _empty_like_input(data, (W1 * W2 + 1,), "int32")
    ids = _empty_like_input(data, (n,), "int32")
    with _DeviceCtx(data, stream) as s:
        _check(load().knng_rvq_index(_ptr(data), n, D, _ptr(words1), W1, _ptr(words2), W2, _ptr(codes), _ptr(off),
                                     _ptr(ids), s))
    return codes, off, ids


def knng_rvq_seeds(words1, words2, list_offsets, list_ids, queries, probe1, s, stream=None):
    """Seeds of Alg. 2 from the inverted index (Sec. 4.2, Eqns. 2 and 3, the
    cascaded pruning keeping probe1 stage-1 words): m x s ids, -1 padded."""
    words1 = _contig(words1, "float32")
    words2 = _contig(words2, "float32")
    list_offsets = _contig(list_offsets, "int32")
    list_ids = _contig(list_ids, "int32")
    queries = _contig(queries, "float32")
    W1, D = words1.shape
    W2 = words2.shape[0]
    m = queries.shape[0]
    out = _empty_like_input(queries, (m, s), "int32")
    with _DeviceCtx(queries, stream) as st:
        _check(load().knng_rvq_seeds(_ptr(words1), W1, _ptr(words2), W2, D, _ptr(list_offsets), _ptr(list_ids),
                                     list_ids.shape[0], _ptr(queries), m, probe1, s, _ptr(out), st))
    return out


def knng_exact(data, k, sample=None, stream=None):
    """Exact k-NN lists of the sampled rows (all rows if sample is None)."""
    data = _contig(data, "float32")
    n, D = data.shape
    if sample is not None:
        sample = _contig(sample, "int32")
    s_rows = n if sample is None else len(sample)
    ids = _empty_like_input(data, (s_rows, k), "int32")
    d = _empty_like_input(data, (s_rows, k), "float32")
    with _DeviceCtx(data, stream) as s:
        _check(load().knng_exact(_ptr(data), n, D, k, _ptr(sample), s_rows, _ptr(ids), _ptr(d), s))
    return ids, d


def knng_exact_noalloc(data, k, sample, out=None, stream=None):
    """knng_exact that allocates no device memory inside the library: for
    callers that cannot allocate at that point (a memory manager owns the
    device's memory, or an allocation's implicit synchronisation is not
    allowed).  Device tensors only; len(sample) * k <= 262144.  Pass `out`
    (two preallocated device tensors of shape (len(sample), k)) to avoid any
    allocation on this side too."""
    data = _contig(data, "float32")
    sample = _contig(sample, "int32")
    n, D = data.shape
    s_rows = len(sample)
    if out is None:
        ids = _empty_like_input(data, (s_rows, k), "int32")
        d = _empty_like_input(data, (s_rows, k), "float32")
    else:
        ids, d = out
    with _DeviceCtx(data, stream) as s:
        _check(load().knng_exact_noalloc(_ptr(data), n, D, k, _ptr(sample), s_rows, _ptr(ids), _ptr(d), s))
    return ids, d


def knng_recall(ids, dists, gt_ids, gt_dists, sample, stream=None):
    """(recall by id set, tie-tolerant recall) of a graph on sampled rows."""
    ids = _contig(ids, "int32")
    dists = _contig(dists, "float32")
    gt_ids = _contig(gt_ids, "int32")
    gt_dists = _contig(gt_dists, "float32")
    sample = _contig(sample, "int32")
    k = ids.shape[1]
    ri = ctypes.c_double()
    rt = ctypes.c_double()
    with _DeviceCtx(ids, stream) as s:
        _check(load().knng_recall(_ptr(ids), _ptr(dists), _ptr(gt_ids), _ptr(gt_dists), _ptr(sample), len(sample), k,
                                  ctypes.byref(ri), ctypes.byref(rt), s))
    return ri.value, rt.value


def knng_workspace_bytes(n, D, params):
    return int(load().knng_workspace_bytes(n, D, ctypes.byref(params)))


def stats_enable(on=True, timing=False):
    load().knng_stats_enable(1 if on else 0, 1 if timing else 0)


def stats_reset():
    load().knng_stats_reset()


def stats():
    """{kernel name: dict(launches, ms, bytes, flops)} summed since the last reset."""
    lib = load()
    out = {}
    st = KernelStat()
    for i in range(lib.knng_stats_count()):
        if lib.knng_stats_get(i, ctypes.byref(st)) == 0:
            out[st.name.decode()] = dict(launches=int(st.launches), ms=float(st.ms), bytes=float(st.bytes),
                                         flops=float(st.flops), items=float(st.items))
    return out
