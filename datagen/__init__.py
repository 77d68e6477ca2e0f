"""Seeded synthetic inputs shaped like the workloads of arXiv 1701.08475, Sec. 5.

This module only draws inputs.  It holds none of the graph-construction
arithmetic, so both the CUDA path and the CPU oracle can use it.

The paper evaluates on SIFT1M (128-d, integer values 0..255) and GIST1M
(960-d, non-negative) (Sec. 5).  Those datasets are not available here; the
generators below produce stand-ins with the same dimensionality, value range
and clustered structure.  No item of either dataset is reproduced.
"""
import numpy as np

__all__ = ["gaussian_mixture", "sift_like", "gist_like", "unit_mixture", "batched_mixtures",
           "WORKLOADS", "BATCHED", "make", "make_seeded", "sample_rows"]


def gaussian_mixture(n, D, n_centres, seed, lo=-10.0, hi=10.0, sigma=1.0):
    """Isotropic Gaussian mixture: centres ~ U[lo, hi]^D, point = centre + N(0, sigma^2)."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(lo, hi, size=(n_centres, D)).astype(np.float32)
    lab = rng.integers(0, n_centres, size=n)
    X = rng.standard_normal(size=(n, D), dtype=np.float32)
    X *= np.float32(sigma)
    X += centres[lab]
    return np.ascontiguousarray(X, dtype=np.float32)


def _chunks(n, chunk, fill):
    """Runs fill(a, b, rng) over the row ranges [a, b) of `chunk` rows in
    parallel threads; chunk c draws from its own stream, seeded by the
    caller's seed material and c, so the result does not depend on the
    number of threads (numpy's generators release the GIL in bulk draws)."""
    from concurrent.futures import ThreadPoolExecutor
    import os
    starts = list(range(0, n, chunk))
    if len(starts) <= 1:
        for c, a in enumerate(starts):
            fill(a, min(n, a + chunk), c)
        return
    with ThreadPoolExecutor(max_workers=min(len(starts), os.cpu_count() or 4, 32)) as ex:
        list(ex.map(lambda ca: fill(ca[1], min(n, ca[1] + chunk), ca[0]), enumerate(starts)))


def sift_like(n, D=128, n_centres=1000, seed=0, zero_frac=0.3, spread=25.0, latent_dim=16, noise=4.0,
              chunk=1 << 18):
    """Non-negative integers 0..255 stored as FP32, clustered, low intrinsic dimension.

    Centres ~ U[0, 120]^D, each with its own set of zero coordinates
    (Bernoulli(zero_frac)).  A point varies around its centre inside the
    centre's own latent_dim-dimensional subspace (a random D x latent_dim basis
    scaled so every coordinate has standard deviation `spread`), plus
    N(0, noise^2) in every coordinate; the centre's zero coordinates stay
    zero; then clip to [0, 255] and round.  (Descriptors like SIFT's have a
    low intrinsic dimension; isotropic 128-d noise would make every point of a
    cluster nearly equidistant, which no real descriptor set does.)
    With latent_dim=None the variation is isotropic N(0, spread^2) instead.
    """
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.0, 120.0, size=(n_centres, D)).astype(np.float32)
    keep = (rng.random(size=(n_centres, D)) >= zero_frac).astype(np.float32)
    lab = rng.integers(0, n_centres, size=n)
    if latent_dim:
        basis = rng.standard_normal(size=(n_centres, latent_dim, D), dtype=np.float32)
        basis *= np.float32(spread / np.sqrt(latent_dim))
    X = np.empty((n, D), np.float32)

    def fill(a, b, c):
        r = np.random.default_rng([seed, c + 1])
        lb = lab[a:b]
        if latent_dim:
            z = r.standard_normal(size=(b - a, latent_dim), dtype=np.float32)
            v = r.standard_normal(size=(b - a, D), dtype=np.float32) * np.float32(noise)
            order = np.argsort(lb, kind="stable")
            bounds = np.searchsorted(lb[order], np.arange(n_centres + 1))
            for ci in range(n_centres):
                rows = order[bounds[ci]:bounds[ci + 1]]
                if len(rows):
                    v[rows] += z[rows] @ basis[ci]
        else:
            v = r.standard_normal(size=(b - a, D), dtype=np.float32) * np.float32(spread)
        v += centres[lb]
        v *= keep[lb]
        np.clip(v, 0.0, 255.0, out=v)
        np.rint(v, out=v)
        X[a:b] = v

    _chunks(n, chunk, fill)
    return X


def gist_like(n, D=960, n_centres=1000, seed=0, block=32, alpha=0.3, conc=50.0, chunk=1 << 15):
    """Values in [0, 1], non-negative, L1-normalised per `block`-dim block.

    Each centre has a Dirichlet(alpha) profile per block; a point draws
    Gamma(conc * profile) per coordinate around its centre and L1-normalises
    every block.
    """
    assert D % block == 0
    rng = np.random.default_rng(seed)
    prof = rng.gamma(alpha, size=(n_centres, D)).astype(np.float32) + np.float32(1e-3)
    prof = prof.reshape(n_centres, D // block, block)
    prof /= prof.sum(axis=2, keepdims=True)
    prof = prof.reshape(n_centres, D)
    lab = rng.integers(0, n_centres, size=n)
    X = np.empty((n, D), np.float32)

    def fill(a, b, c):
        r = np.random.default_rng([seed, c + 1])
        v = r.gamma(conc * prof[lab[a:b]] + np.float32(1e-3)).astype(np.float32)
        v = v.reshape(b - a, D // block, block)
        v /= np.maximum(v.sum(axis=2, keepdims=True), np.float32(1e-30))
        X[a:b] = v.reshape(b - a, D)

    _chunks(n, chunk, fill)
    return X


def unit_mixture(n, D=96, n_centres=10000, seed=0, sigma=0.1, chunk=1 << 18):
    """Unit-normalised mixture: centres ~ N(0, I) normalised; point = centre + N(0, sigma^2), normalised."""
    rng = np.random.default_rng(seed)
    cen = rng.standard_normal(size=(n_centres, D), dtype=np.float32)
    cen /= np.linalg.norm(cen, axis=1, keepdims=True)
    lab = rng.integers(0, n_centres, size=n)
    X = np.empty((n, D), np.float32)

    def fill(a, b, c):
        r = np.random.default_rng([seed, c + 1])
        v = r.standard_normal(size=(b - a, D), dtype=np.float32)
        v *= np.float32(sigma)
        v += cen[lab[a:b]]
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        X[a:b] = v

    _chunks(n, chunk, fill)
    return X


# The batched workload: 64 independent Gaussian mixtures of 2,000 - 200,000
# points, D in {64, 128, 256}, k = 16, leaf_max chosen per D by the autotuner.
BATCHED = dict(name="batched-64-gmm", n_inst=64, seed=1238, k=16, passes=3, rounds=4)

# Workload recipes: sizes and build parameters of the graph workloads.
WORKLOADS = {
    "gmm-10k-d32": dict(gen="gaussian_mixture", n=10_000, D=32, n_centres=50, seed=1235,
                        k=10, leaf_max=64, passes=1, rounds=2),
    "sift-like-1m-d128": dict(gen="sift_like", n=1_000_000, D=128, n_centres=1000, seed=1236,
                              k=20, leaf_max=128, passes=3, rounds=4),
    "gist-like-1m-d960": dict(gen="gist_like", n=1_000_000, D=960, n_centres=1000, seed=1237,
                              k=20, leaf_max=256, passes=3, rounds=4),
    "unit-10m-d96": dict(gen="unit_mixture", n=10_000_000, D=96, n_centres=10000, seed=1239,
                         k=16, leaf_max=128, passes=3, rounds=4),
}


def batched_mixtures(n_inst=64, seed=1238, n_lo=2000, n_hi=200000, dims=(64, 128, 256), c_lo=20, c_hi=500):
    """Independent instances for a batched build: n ~ U[n_lo, n_hi], D drawn
    from `dims`, each an isotropic Gaussian mixture (centres U[-10, 10],
    sigma 1) with U[c_lo, c_hi] centres.  Returns a list of (n x D) arrays."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_inst):
        n = int(rng.integers(n_lo, n_hi + 1))
        D = int(dims[int(rng.integers(0, len(dims)))])
        c = int(rng.integers(c_lo, c_hi + 1))
        out.append(gaussian_mixture(n, D, c, seed=seed * 1000 + i))
    return out


def make(name, n=None):
    """Draw the input of workload `name` (optionally only its first `n` rows' recipe at size n)."""
    return make_seeded(name, n, WORKLOADS[name]["seed"])


def make_seeded(name, n=None, seed=None):
    """The recipe of workload `name` at size n (default: its own) and another seed (default: its own)."""
    w = dict(WORKLOADS[name])
    n = w["n"] if n is None else n
    seed = w["seed"] if seed is None else seed
    g = w["gen"]
    if g == "gaussian_mixture":
        return gaussian_mixture(n, w["D"], w["n_centres"], seed)
    if g == "sift_like":
        return sift_like(n, w["D"], w["n_centres"], seed)
    if g == "gist_like":
        return gist_like(n, w["D"], w["n_centres"], seed)
    if g == "unit_mixture":
        return unit_mixture(n, w["D"], w["n_centres"], seed)
    raise KeyError(g)


def sample_rows(n, s, seed):
    """A sorted seeded sample of s distinct row indices (all rows if s >= n)."""
    if s >= n:
        return np.arange(n, dtype=np.int32)
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=s, replace=False)).astype(np.int32)
