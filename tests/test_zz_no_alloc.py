"""knng_exact_noalloc: exact lists with no device allocation in the library,
for callers that cannot allocate at that point (a memory manager owns the
device's memory, or an allocation's implicit synchronisation is not allowed).

Checked through the C ABI against knng_exact on two calls in a row (the
second with other rows, so that leftovers of the first call would show), at
the tolerance the other parity tests use: ids and distance bits identical.
This file is collected last so that a failure here stops a -x run only after
every other test has run.
"""
import numpy as np
import pytest

import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def knng():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1701_08475_gb300 as m
    m.load()
    return m


def test_noalloc_matches_exact_on_two_calls(knng):
    X = datagen.gaussian_mixture(5000, 37, 30, seed=41)
    Xd = torch.from_numpy(X).cuda()
    k = 20
    for seed, s in ((1, 300), (2, 1000)):
        smp = torch.from_numpy(datagen.sample_rows(5000, s, seed=seed)).cuda()
        out = (torch.empty((s, k), dtype=torch.int32, device="cuda"),
               torch.empty((s, k), dtype=torch.float32, device="cuda"))
        got_ids, got_d = knng.knng_exact_noalloc(Xd, k, smp, out=out)
        want_ids, want_d = knng.knng_exact(Xd, k, smp)
        torch.cuda.synchronize()
        assert torch.equal(got_ids, want_ids)
        assert torch.equal(got_d.view(torch.int32), want_d.view(torch.int32))


def test_noalloc_rejects_requests_beyond_its_scratch(knng):
    X = torch.from_numpy(datagen.gaussian_mixture(40000, 8, 10, seed=2)).cuda()
    smp = torch.arange(20000, dtype=torch.int32, device="cuda")
    with pytest.raises(knng.KnngError) as e:
        knng.knng_exact_noalloc(X, 16, smp)     # 20000 * 16 > 262144 entries
    assert e.value.code == -1 and "262144" in str(e.value)
    with pytest.raises(knng.KnngError):
        knng.knng_exact_noalloc(X.cpu(), 16, smp[:10].cpu())   # host pointers are refused
