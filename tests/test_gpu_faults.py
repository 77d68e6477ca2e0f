"""Failure detection on the host (no device fault is ever made).

KNNG_FAULT=alloc makes the library's workspace allocation fail as if the
device were out of memory; KNNG_FAULT=launch makes the runtime refuse one
kernel launch on the host (a block larger than any GPU allows).  Each call
must return its error code (KNNG_ENOMEM, KNNG_ECUDA) instead of a graph, and
the next call, without the variable, must work and give the usual result.
The device-side checks (status word, bounded waits) are covered where their
inputs arise: non-finite data and bad ids in the parity tests.
"""
import os

import numpy as np
import pytest

import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ENOMEM, ECUDA = -2, -3


@pytest.fixture(scope="module")
def knng():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1701_08475_gb300 as m
    m.load()
    return m


@pytest.fixture
def fault():
    def set_(mode):
        if mode is None:
            os.environ.pop("KNNG_FAULT", None)
        else:
            os.environ["KNNG_FAULT"] = mode
    yield set_
    os.environ.pop("KNNG_FAULT", None)


def _params(knng):
    return knng.default_params(k=8, leaf_max=40, tree_passes=2, refine_rounds=2,
                               join_mode=knng.KNNG_JOIN_FWD_REV, twomeans_iters=3, seed=11)


@pytest.mark.parametrize("mode,code", [("alloc", ENOMEM), ("launch", ECUDA)])
def test_build_reports_injected_fault_and_recovers(knng, fault, mode, code):
    X = torch.from_numpy(datagen.sift_like(3000, D=24, n_centres=20, seed=7)).cuda()
    want = knng.knng_build_ex(X, _params(knng))
    fault(mode)
    with pytest.raises(knng.KnngError) as e:
        knng.knng_build_ex(X, _params(knng))
    assert e.value.code == code
    fault(None)
    got = knng.knng_build_ex(X, _params(knng))
    torch.cuda.synchronize()
    assert torch.equal(got[0], want[0]) and torch.equal(got[1], want[1])


@pytest.mark.parametrize("mode,code", [("alloc", ENOMEM), ("launch", ECUDA)])
def test_exact_reports_injected_fault_and_recovers(knng, fault, mode, code):
    X = torch.from_numpy(datagen.gaussian_mixture(4000, 20, 10, seed=3)).cuda()
    smp = torch.from_numpy(datagen.sample_rows(4000, 100, seed=1)).cuda()
    want = knng.knng_exact(X, 10, smp)
    fault(mode)
    with pytest.raises(knng.KnngError) as e:
        knng.knng_exact(X, 10, smp)
    assert e.value.code == code
    fault(None)
    got = knng.knng_exact(X, 10, smp)
    assert torch.equal(got[0], want[0]) and torch.equal(got[1], want[1])


def test_noalloc_reports_a_refused_launch(knng, fault):
    """The entry point without allocation checks for a refused launch before
    it trusts its status word (the outputs would hold stale lists)."""
    X = torch.from_numpy(datagen.gaussian_mixture(3000, 16, 10, seed=5)).cuda()
    smp = torch.from_numpy(datagen.sample_rows(3000, 50, seed=2)).cuda()
    want = knng.knng_exact(X, 12, smp)
    fault("launch")
    with pytest.raises(knng.KnngError) as e:
        knng.knng_exact_noalloc(X, 12, smp)
    assert e.value.code == ECUDA
    fault(None)
    got = knng.knng_exact_noalloc(X, 12, smp)
    torch.cuda.synchronize()
    assert torch.equal(got[0], want[0])
    assert np.array_equal(got[1].cpu().numpy().view(np.int32), want[1].cpu().numpy().view(np.int32))
