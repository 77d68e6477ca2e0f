"""GPU parity of the sampled refinement round (nearest-neighbour descent with
sampling, the prior art Sec. 1 cites): lists and distances equal the
oracle's bit for bit, round by round from a given graph and for whole builds
in the plain (FP32 join) and exact (tensor-core join) forms."""
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


@pytest.mark.parametrize("k,ms,rounds", [(8, 1, 1), (8, 4, 3), (20, 10, 4), (32, 7, 2)])
def test_rounds_from_a_graph_match_oracle(knng, k, ms, rounds):
    X = datagen.sift_like(4000, D=24, n_centres=30, seed=k)
    gi, gd = oracle.build_graph(X, k, 2 * (k + 1) + 8, passes=1, rounds=0, seed=3)
    p = knng.default_params(k=k, refine_rounds=rounds, join_mode=knng.KNNG_JOIN_SAMPLED, sample=ms, seed=11)
    ids, d = _dev(gi), _dev(gd)
    knng.knng_refine(_dev(X), ids, d, p)
    wi, wd, flags = gi, gd, np.ones(gi.shape, np.uint8)
    for r in range(rounds):
        wi, wd, flags, _ = oracle.refine_sampled(X, wi, wd, flags, ms, seed=11, round_=r)
    assert np.array_equal(ids.cpu().numpy(), wi)
    assert np.array_equal(d.cpu().numpy(), wd)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("kind", ["integer", "float"])
def test_whole_build_matches_oracle(knng, precision, kind):
    n, D, k = 6000, 32, 12
    X = datagen.sift_like(n, D=D, n_centres=40, seed=5) if kind == "integer" else \
        datagen.gaussian_mixture(n, D, 40, seed=5)
    prec = {"fp32": knng.KNNG_FP32, "bf16": knng.KNNG_BF16}[precision]
    p = knng.default_params(k=k, leaf_max=48, tree_passes=2, refine_rounds=3, join_mode=knng.KNNG_JOIN_SAMPLED,
                            sample=6, seed=7, twomeans_iters=3, precision=prec)
    ids, d = knng.knng_build_ex(_dev(X), p)
    wi, wd = oracle.build_graph_sampled(X, k, 48, passes=2, rounds=3, iters=3, ms=6, seed=7)
    assert np.array_equal(ids.cpu().numpy(), wi)
    assert np.array_equal(d.cpu().numpy(), wd)
