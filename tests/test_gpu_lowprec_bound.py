"""The low-precision leaf stage against its error bound, on the GB300.

The leaf certificate (and the pruned re-rank built on it) is exact only if
the tensor cores' approximate distances d^ stay within the bound
    |d^ - d~| <= c (||x~_i|| + ||x~_j||)^2 + 2^-23 |d^|
of the exact distance d~ = ||x~_i - x~_j||^2 of the quantised rows, with
c = (16 Dp + 8) 2^-24 for the 16-bit forms (four times the textbook bound of
an FP32 dot product, the summation order of the tensor cores being
unspecified) plus D 2^-13 for FP8 (an assumed accumulator of at least 14
significant bits).  The parity hook knng_leaf_dhat returns the kernel's d^,
its quantised copy, scales, norms and error bounds for one cluster; here d~
is taken in FP64 from the quantised values, the FP8 quantiser is checked
against the E4M3 format written out from its definition (1 sign, 4 exponent
bits of bias 7, 3 fraction bits, no infinities, S.1111.111 = NaN), and the
error bounds e >= ||x - x~|| are checked in FP64.  The largest observed error
in units of the assumed bound is printed: the margin the assumption has.
"""
import numpy as np
import pytest

import datagen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -24


def e4m3_values():
    """The 254 finite E4M3 values (both signs, +-0 once each), from the format's definition."""
    vals = []
    for e in range(16):
        for f in range(8):
            if e == 15 and f == 7:
                continue  # NaN
            v = (f / 8.0) * 2.0 ** -6 if e == 0 else (1.0 + f / 8.0) * 2.0 ** (e - 7)
            vals.append((v, f))
    return vals


def e4m3_round(t):
    """Round-to-nearest-even onto the E4M3 grid, saturating at +-448 (float64 in, float64 out)."""
    grid = np.array([v for v, _ in e4m3_values()])
    frac = np.array([f for _, f in e4m3_values()])
    a = np.minimum(np.abs(t), 448.0)
    idx = np.searchsorted(grid, a)
    lo = grid[np.clip(idx - 1, 0, len(grid) - 1)]
    hi = grid[np.clip(idx, 0, len(grid) - 1)]
    flo = frac[np.clip(idx - 1, 0, len(grid) - 1)]
    pick_hi = (hi - a < a - lo) | ((hi - a == a - lo) & (flo % 2 == 1))
    r = np.where(a <= lo, lo, np.where(pick_hi, hi, lo))
    r = np.where(a >= hi, hi, r)
    return np.sign(t) * r


def cases():
    rng = np.random.default_rng(5)
    out = {
        "gauss-128x96": rng.standard_normal((128, 96)).astype(np.float32),
        "unit-256x96": datagen.unit_mixture(256, 96, 4, seed=3),
        "offset-128x128": (100.0 + rng.standard_normal((128, 128))).astype(np.float32),
        "gist-200x960": datagen.gist_like(200, 960, 3, seed=4),
        "range-100x64": (rng.standard_normal((100, 64)) * 10.0 ** rng.uniform(-3, 3, (100, 64))).astype(np.float32),
        "signed-int-97x40": rng.integers(-250, 250, size=(97, 40)).astype(np.float32),
    }
    return out


CASES = cases()


@pytest.fixture(scope="module")
def knng():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1701_08475_gb300 as m
    m.load()
    return m


@pytest.mark.parametrize("precision", ["bf16", "fp16", "fp8"])
@pytest.mark.parametrize("name", list(CASES))
def test_leaf_dhat_within_the_certificate_bound(knng, precision, name):
    X = CASES[name]
    m, D = X.shape
    prec = {"bf16": knng.KNNG_BF16, "fp16": knng.KNNG_FP16, "fp8": knng.KNNG_FP8}[precision]
    dh, q, sc, nrm, err = knng.knng_leaf_dhat(X, prec)
    q64, s64 = q.astype(np.float64), sc.astype(np.float64)
    xt = q64 * s64[:, None]                       # x~ = s q, exact in FP64
    if precision == "fp8":
        # the quantiser: s = max|x| / 448 in FP32, q = E4M3(x / s) nearest even, saturated
        amax = np.abs(X).max(axis=1)
        s_want = np.where(amax >= 1e-30, (amax / np.float32(448.0)).astype(np.float32), np.float32(1.0))
        assert np.array_equal(sc, s_want)
        t = (X / s_want[:, None]).astype(np.float32).astype(np.float64)
        assert np.array_equal(q64, e4m3_round(t))
        Dp = (D + 127) // 128 * 128
    else:
        # the 16-bit copy is x rounded to nearest even
        want = torch.from_numpy(X).to(torch.bfloat16 if precision == "bf16" else torch.float16).float().numpy()
        assert np.array_equal(q, want)
        assert np.all(sc == 1.0)
        Dp = (D + 63) // 64 * 64
    # error bounds e >= ||x - x~|| and not far above it
    true_e = np.sqrt(((X.astype(np.float64) - xt) ** 2).sum(1))
    assert np.all(err.astype(np.float64) >= true_e)
    assert np.all(err.astype(np.float64) <= true_e * (1 + 1e-4) + 1e-30)
    # squared norms of x~ as the kernel uses them
    n64 = (xt * xt).sum(1)
    assert np.all(np.abs(nrm.astype(np.float64) - n64) <= (Dp + 8) * U * n64 + 1e-38)
    # d^ against the exact d~ of the quantised rows
    diff = xt[:, None, :] - xt[None, :, :]
    dt = np.einsum("ijk,ijk->ij", diff, diff)
    nr = np.sqrt(n64)
    scale2 = (nr[:, None] + nr[None, :]) ** 2
    c = (16.0 * Dp + 8.0) * U + (Dp * 2.0 ** -13 if precision == "fp8" else 0.0)
    bound = c * scale2 + 2.0 ** -23 * np.abs(dh.astype(np.float64))
    e = np.abs(dh.astype(np.float64) - dt)
    worst = float(np.max(e / np.maximum(bound, 1e-300)))
    textbook = float(np.max(e / np.maximum((Dp + 2) * U * scale2, 1e-300)))
    print("%s %s: max |d^ - d~| = %.3g of the assumed bound, %.3g of the textbook FP32 bound"
          % (name, precision, worst, textbook))
    assert worst <= 1.0


@pytest.mark.parametrize("kind,n,D,k,lm", [("float", 5000, 32, 10, 64), ("float", 3000, 200, 16, 100),
                                           ("signed", 2000, 64, 12, 60), ("integer", 4000, 128, 20, 128),
                                           ("unit", 6000, 96, 16, 128), ("float", 3000, 320, 10, 160),
                                           ("float", 4000, 96, 12, 200)])
def test_fp8_build_equals_fp32(knng, kind, n, D, k, lm):
    """The FP8 leaf stage (per-row scales, pruned exact re-rank) returns the
    FP32 form's graph bit for bit, leaves of one and two 128-row tiles."""
    rng = np.random.default_rng(n + D)
    X = {"float": lambda: datagen.gaussian_mixture(n, D, 30, seed=n + D),
         "signed": lambda: rng.integers(-250, 250, size=(n, D)).astype(np.float32),
         "integer": lambda: datagen.sift_like(n, D=D, n_centres=max(2, n // 80), seed=n + D),
         "unit": lambda: datagen.unit_mixture(n, D, 60, seed=n + D)}[kind]()
    common = dict(k=k, leaf_max=lm, tree_passes=2, refine_rounds=1, seed=9,
                  join_mode=knng.KNNG_JOIN_FWD_REV if 2 * k <= 64 else knng.KNNG_JOIN_FWD)
    Xd = torch.from_numpy(X).cuda()
    a_ids, a_d = knng.knng_build_ex(Xd, knng.default_params(precision=knng.KNNG_FP8, **common))
    f_ids, f_d = knng.knng_build_ex(Xd, knng.default_params(precision=knng.KNNG_FP32, **common))
    torch.cuda.synchronize()
    assert torch.equal(a_ids, f_ids)
    assert torch.equal(a_d.view(torch.int32), f_d.view(torch.int32))
