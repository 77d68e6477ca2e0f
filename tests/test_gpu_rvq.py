"""GPU parity of the residue-quantisation inverted index (Sec. 4.1, Eqn. 1;
Sec. 4.2, Eqns. 2 and 3): vocabularies, codes, lists and seeds from the CUDA
path equal the oracle's bit for bit on the same inputs.  Float and integer
data, dimensions below, at and across the 64-dim chunk, vocabularies of 1 to
256 words, counts that leave ragged assignment and sort tiles, zero
iterations, probe counts from 1 to the 8192-key limit, seed counts from 1 to
beyond the listed points; at the sift-like 1M size, vocabularies trained on a
20,000-row prefix, the codes of all rows (the oracle's assignment run in
threads over row chunks), the lists, and the seeds of sampled queries."""
import concurrent.futures as cf

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


def _data(kind, n, D, seed):
    if kind == "float":
        return datagen.gaussian_mixture(n, D, 40, seed=seed)
    return datagen.sift_like(n, D=D, n_centres=60, seed=seed)


TRAIN_CASES = [
    ("float", 5000, 8, 16, 16, 5),
    ("integer", 6001, 33, 7, 13, 4),
    ("float", 4097, 64, 256, 256, 3),
    ("integer", 20000, 128, 256, 256, 4),
    ("float", 3000, 130, 32, 8, 2),
    ("integer", 2500, 20, 1, 1, 3),
    ("float", 300, 12, 256, 200, 2),
    ("integer", 4000, 16, 64, 64, 0),
]


@pytest.mark.parametrize("kind,n,D,W1,W2,iters", TRAIN_CASES)
def test_train_matches_oracle(knng, kind, n, D, W1, W2, iters):
    X = _data(kind, n, D, 31 + n)
    w1, w2 = knng.knng_rvq_train(_dev(X), W1, W2, iters, seed=77)
    o1, o2 = oracle.rvq_train(X, W1, W2, iters, seed=77)
    assert np.array_equal(_np(w1).view(np.uint32), o1.view(np.uint32))
    assert np.array_equal(_np(w2).view(np.uint32), o2.view(np.uint32))


@pytest.mark.parametrize("kind,n,D,W1,W2", [("float", 7000, 24, 32, 16), ("integer", 9001, 128, 256, 256),
                                            ("float", 2049, 70, 5, 256), ("integer", 100, 8, 256, 3)])
def test_index_matches_oracle(knng, kind, n, D, W1, W2):
    X = _data(kind, n, D, 41 + n)
    o1, o2 = oracle.rvq_train(X, W1 if W1 <= n else n, W2, 3, seed=5) if W1 <= n else (None, None)
    if o1 is None:   # more words than points: vocabularies of other points of the same recipe
        Y = _data(kind, 4 * W1, D, 43)
        o1, o2 = oracle.rvq_train(Y, W1, W2, 2, seed=5)
    codes, off, ids = knng.knng_rvq_index(_dev(X), _dev(o1), _dev(o2))
    oc, oo, oi = oracle.rvq_index(X, o1, o2)
    assert np.array_equal(_np(codes), oc)
    assert np.array_equal(_np(off), oo)
    assert np.array_equal(_np(ids), oi)


@pytest.mark.parametrize("probe1,s", [(1, 1), (1, 50), (4, 200), (16, 33), (32, 1000), (256, 5), (8, 100000)])
def test_seeds_match_oracle(knng, probe1, s):
    n, D = 12000, 40
    X = _data("integer", n, D, 51)
    W1 = 256 if probe1 > 32 else 64
    W2 = 32 if probe1 > 32 else 256
    o1, o2 = oracle.rvq_train(X, W1, W2, 2, seed=9)
    _, off, ids = oracle.rvq_index(X, o1, o2)
    Q = _data("integer", 300, D, 52)
    S = knng.knng_rvq_seeds(_dev(o1), _dev(o2), _dev(off), _dev(ids), _dev(Q), probe1, s)
    assert np.array_equal(_np(S), oracle.rvq_seeds(o1, o2, off, ids, Q, probe1, s))


def test_seeds_on_float_data_and_host_buffers(knng):
    X = _data("float", 5000, 48, 61)
    o1, o2 = oracle.rvq_train(X, 40, 50, 3, seed=2)
    _, off, ids = oracle.rvq_index(X, o1, o2)
    Q = _data("float", 257, 48, 62)
    S = knng.knng_rvq_seeds(o1, o2, off, ids, Q, 12, 64)          # host buffers
    assert np.array_equal(_np(S), oracle.rvq_seeds(o1, o2, off, ids, Q, 12, 64))
    w1, w2 = knng.knng_rvq_train(X, 40, 50, 3, seed=2)            # host buffers
    assert np.array_equal(_np(w1), o1) and np.array_equal(_np(w2), o2)


def test_bad_offsets_are_rejected(knng):
    w = np.zeros((4, 8), np.float32)
    off = np.array([0, 3, 2] + [5] * 14, np.int32)                # decreasing
    ids = np.arange(5, dtype=np.int32)
    with pytest.raises(knng.KnngError):
        knng.knng_rvq_seeds(_dev(w), _dev(w), _dev(off), _dev(ids), _dev(np.zeros((2, 8), np.float32)), 2, 3)
    off = np.array([0] * 16 + [9], np.int32)                      # beyond the 5 ids
    with pytest.raises(knng.KnngError):
        knng.knng_rvq_seeds(_dev(w), _dev(w), _dev(off), _dev(ids), _dev(np.zeros((2, 8), np.float32)), 2, 3)


def _oracle_codes_threaded(X, o1, o2, chunk=32768):
    """The oracle's assignment (both stages) over row chunks in threads (the
    C calls release the interpreter lock); residues as the oracle forms them,
    FP32 differences."""
    rows = [(a, min(len(X), a + chunk)) for a in range(0, len(X), chunk)]
    with cf.ThreadPoolExecutor(max_workers=16) as ex:
        c1 = np.concatenate(list(ex.map(lambda r: oracle.rvq_assign(X[r[0]:r[1]], o1), rows)))
        R = (X - o1[c1]).astype(np.float32)
        c2 = np.concatenate(list(ex.map(lambda r: oracle.rvq_assign(R[r[0]:r[1]], o2), rows)))
    return c1, c2


def test_sift_like_1m(knng):
    w = datagen.WORKLOADS["sift-like-1m-d128"]
    X = datagen.make("sift-like-1m-d128")
    n = X.shape[0]
    Xd = _dev(X)
    ntrain = 20000
    w1, w2 = knng.knng_rvq_train(Xd[:ntrain], 256, 256, 4, seed=w["seed"])
    o1, o2 = oracle.rvq_train(X[:ntrain], 256, 256, 4, seed=w["seed"])
    assert np.array_equal(_np(w1), o1) and np.array_equal(_np(w2), o2)
    codes, off, ids = knng.knng_rvq_index(Xd, w1, w2)
    codes, off, ids = _np(codes), _np(off), _np(ids)
    c1, c2 = _oracle_codes_threaded(X, o1, o2)
    assert np.array_equal(codes[:, 0], c1) and np.array_equal(codes[:, 1], c2)
    key = c1.astype(np.int64) * 256 + c2
    assert np.array_equal(off, np.concatenate([[0], np.cumsum(np.bincount(key, minlength=65536))]))
    assert np.array_equal(ids, np.argsort(key, kind="stable"))
    rng = np.random.default_rng(3)
    Q = np.clip(np.rint(X[rng.integers(0, n, 64)] + rng.normal(0, 4.0, size=(64, 128))), 0, 255).astype(np.float32)
    S = knng.knng_rvq_seeds(w1, w2, _dev(off), _dev(ids), _dev(Q), 16, 64)
    assert np.array_equal(_np(S), oracle.rvq_seeds(o1, o2, off, ids, Q, 16, 64))
