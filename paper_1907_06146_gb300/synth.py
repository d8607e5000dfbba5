"""Seeded synthetic inputs for the NSSG build and search.

This module holds no arithmetic of the method itself: it only draws base vectors,
queries and navigating-node ids.  Both the CUDA path and the CPU oracle consume
what it produces, so it is the one piece of code the two share.

The paper evaluates on SIFT1M, GIST1M and Deep100M (Sec. 5.1, Table 2), none of
which ship with this project.  The generators below stand in for them with the
same shapes, sizes and value ranges:

* ``small``      -- 10,000 x 32 float32, a mixture of 16 isotropic Gaussians
                    (centres ~ N(0, 4I), unit spread); 1,000 queries.  Sized
                    like the SIFT10K pre-experiment of Sec. 4.1.
* ``sift_like``  -- 1,000,000 x 128 float32 holding integers 0..255: 1,000
                    overlapping anisotropic Gaussians in a shared basis (power-law
                    spectrum, local intrinsic dimension about 13), rounded and
                    clipped, shifted so that about 30% of all coordinates are zero;
                    10,000 queries.  Shaped like SIFT1M (Table 2: d = 128, LID 12.9).
* ``gist_like``  -- 1,000,000 x 960 float32 in [0, 1]: 500 overlapping anisotropic
                    Gaussians built like sift_like's (a flatter spectrum, centres spread
                    half as widely as the points: local intrinsic dimension 2.3 times
                    sift_like's) passed through a softplus and divided by the global
                    maximum; 1,000 queries.  Shaped like GIST1M (Table 2: d = 960,
                    LID 29.1).
* ``deep_like``  -- N x 96 float32: 2,000 overlapping anisotropic Gaussians built
                    like sift_like's (no rounding, a steeper spectrum: local
                    intrinsic dimension 0.79 of sift_like's), rows L2-normalised.  Shaped like
                    Deep100M (Table 2: d = 96, LID 10.2) at a smaller N.

All draws use numpy's PCG64 with a fixed seed, so a configuration is fully
determined by its name, its sizes and its seed.
"""
from __future__ import annotations

import dataclasses

import numpy as np

SEED_SMALL = 190706141
SEED_SIFT = 190706142
SEED_GIST = 190706143
SEED_BATCH = 190706144
SEED_DEEP = 190706145


@dataclasses.dataclass
class Workload:
    name: str
    base: np.ndarray      # float32 [n][d], C-contiguous
    queries: np.ndarray   # float32 [nq][d], C-contiguous
    K: int                # kNN-graph degree
    L: int                # candidate pool size (paper's l)
    R: int                # maximum out-degree (paper's r)
    alpha: float          # minimum angle in degrees
    n_nav: int            # navigating nodes (paper's s, or m in Sec. 5.3)
    info: dict

    @property
    def n(self) -> int:
        return self.base.shape[0]

    @property
    def d(self) -> int:
        return self.base.shape[1]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def batched_specs(count: int = 64, n_min: int = 10_000, n_max: int = 500_000,
                  seed: int = SEED_BATCH) -> list:
    """Shapes of the many-index batch: n log-uniform in [n_min, n_max], d from
    {64, 96, 128, 256}, L from {100, 200}; K = 100, R = 32, alpha = 60 for all.  Index i's
    data come from batched_index(spec, seed + 1 + i)."""
    rng = _rng(seed)
    specs = []
    for i in range(count):
        n = int(round(np.exp(rng.uniform(np.log(n_min), np.log(n_max)))))
        d = int(rng.choice([64, 96, 128, 256]))
        L = int(rng.choice([100, 200]))
        specs.append({"index": i, "n": n, "d": d, "K": 100, "L": L, "R": 32, "alpha": 60.0,
                      "seed": seed + 1 + i})
    return specs


def batched_index(spec: dict, nq: int = 0) -> Workload:
    """One index of the batch: the 16-centre isotropic mixture of `small` at its shape."""
    w = small(n=spec["n"], d=spec["d"], nq=nq, n_centres=16, seed=spec["seed"])
    return Workload("batched", w.base, w.queries, K=spec["K"], L=spec["L"], R=spec["R"],
                    alpha=spec["alpha"], n_nav=10, info=dict(spec))


def small(n: int = 10_000, d: int = 32, nq: int = 1_000, n_centres: int = 16,
          seed: int = SEED_SMALL) -> Workload:
    """Isotropic Gaussian mixture: centres ~ N(0, 4I), points = centre + N(0, I)."""
    rng = _rng(seed)
    centres = rng.normal(0.0, 2.0, size=(n_centres, d))
    lab = rng.integers(0, n_centres, size=n)
    base = centres[lab] + rng.normal(0.0, 1.0, size=(n, d))
    qlab = rng.integers(0, n_centres, size=nq)
    queries = centres[qlab] + rng.normal(0.0, 1.0, size=(nq, d))
    return Workload("small", np.ascontiguousarray(base, dtype=np.float32),
                    np.ascontiguousarray(queries, dtype=np.float32),
                    K=20, L=100, R=32, alpha=60.0, n_nav=3,
                    info={"seed": seed, "n_centres": n_centres})


def _random_orthonormal(rng: np.random.Generator, d: int) -> np.ndarray:
    a = rng.normal(size=(d, d))
    q, r = np.linalg.qr(a)
    return q * np.sign(np.diag(r))[None, :]


def _aniso_mixture(rng: np.random.Generator, m: int, d: int, n_clusters: int, gamma: float,
                   top: float, jitter: float, chunk: int, centre_scale: float = 1.0) -> np.ndarray:
    """m float32 rows of a mixture of anisotropic Gaussians sharing one random orthonormal
    basis Q.  Along Q's k-th axis the centres spread with standard deviation centre_scale *
    top * k^-gamma and each cluster's own spread is top * k^-gamma times a per-cluster
    log-normal factor (sigma = jitter), so the clusters overlap into one continuous cloud
    whose local intrinsic dimension falls as gamma grows."""
    Q = _random_orthonormal(rng, d)
    k = np.arange(1, d + 1, dtype=np.float64)
    spec = top * k ** (-gamma)
    centres = (rng.normal(size=(n_clusters, d)) * (centre_scale * spec)) @ Q.T
    spreads = spec * np.exp(rng.normal(0.0, jitter, size=(n_clusters, d)))
    lab = rng.integers(0, n_clusters, size=m)
    y = np.empty((m, d), dtype=np.float32)
    for s in range(0, m, chunk):
        e = min(m, s + chunk)
        w = rng.normal(size=(e - s, d)) * spreads[lab[s:e]]
        y[s:e] = centres[lab[s:e]] + w @ Q.T
    return y


def sift_like(n: int = 1_000_000, d: int = 128, nq: int = 10_000, n_clusters: int = 1_000,
              zero_frac: float = 0.30, seed: int = SEED_SIFT, gamma: float = 1.0,
              top: float = 70.0, jitter: float = 0.3, chunk: int = 131_072) -> Workload:
    """Integer-valued (0..255) mixture of anisotropic Gaussians with ~30% zeros.

    All clusters share one random orthonormal basis Q.  Along its k-th axis the cluster
    centres spread with standard deviation top * k^-gamma and each cluster's own spread is
    top * k^-gamma times a per-cluster log-normal factor (sigma = jitter), so the clusters
    overlap into one continuous, anisotropic cloud whose local intrinsic dimension is
    about 13 for the defaults (SIFT1M: 12.9, Table 2).  A common shift is bisected so that
    the rounded, clipped data hold the requested fraction of zeros."""
    rng = _rng(seed)
    y = _aniso_mixture(rng, n + nq, d, n_clusters, gamma, top, jitter, chunk)
    flat = y.reshape(-1)
    sub = flat[rng.integers(0, flat.size, size=min(flat.size, 2_000_000))].astype(np.float64)
    lo, hi = -1000.0, 1000.0
    for _ in range(60):
        mu = 0.5 * (lo + hi)
        if np.mean(np.rint(sub + mu) <= 0.0) > zero_frac:
            lo = mu
        else:
            hi = mu
    mu = 0.5 * (lo + hi)
    for s in range(0, n + nq, chunk):
        e = min(n + nq, s + chunk)
        y[s:e] = np.clip(np.rint(y[s:e].astype(np.float64) + mu), 0.0, 255.0)
    x = y[rng.permutation(n + nq)]
    base = np.ascontiguousarray(x[:n])
    queries = np.ascontiguousarray(x[n:])
    return Workload("sift_like", base, queries, K=200, L=100, R=50, alpha=60.0, n_nav=10,
                    info={"seed": seed, "n_clusters": n_clusters, "mu": float(mu),
                          "zero_frac": float(np.mean(base == 0.0))})


def gist_like(n: int = 1_000_000, d: int = 960, nq: int = 1_000, n_clusters: int = 500,
              seed: int = SEED_GIST, gamma: float = 0.67, centre_scale: float = 0.5,
              jitter: float = 0.3, chunk: int = 65_536) -> Workload:
    """Non-negative data in [0, 1]: the softplus of a mixture of anisotropic Gaussians
    (the construction of sift_like, a flatter spectrum), divided by the global max.

    In 960 dimensions clusters whose centres spread as widely as their points do come out
    as separate islands (no point's 100 nearest neighbours leave its cluster at 200,000
    points), unlike GIST descriptors, so here the centres spread half as widely as the
    points (94% of the 100 nearest neighbours lie in other clusters).  The latent spectrum
    is scaled so that every coordinate has about unit variance before the softplus bends
    it, and gamma = 0.67 puts the local intrinsic dimension (maximum-likelihood estimate
    from 20 neighbours at 1,000 sampled points of 50,000) at 2.3 times sift_like's under
    the same estimate (41.9 against 18.1), the ratio of GIST1M's 29.1 to SIFT1M's 12.9
    (Table 2)."""
    rng = _rng(seed)
    k = np.arange(1, d + 1, dtype=np.float64)
    top = float(np.sqrt(d / np.sum(k ** (-2.0 * gamma))))
    x = _aniso_mixture(rng, n + nq, d, n_clusters, gamma, top, jitter, chunk, centre_scale)
    for s in range(0, n + nq, chunk):
        e = min(n + nq, s + chunk)
        x[s:e] = np.logaddexp(np.float32(0.0), x[s:e])
    x /= x.max()
    return Workload("gist_like", np.ascontiguousarray(x[:n]), np.ascontiguousarray(x[n:]),
                    K=100, L=500, R=70, alpha=60.0, n_nav=10,
                    info={"seed": seed, "n_clusters": n_clusters, "gamma": gamma,
                          "centre_scale": centre_scale})


def deep_like(n: int = 10_000_000, d: int = 96, nq: int = 10_000, n_clusters: int = 2_000,
              seed: int = SEED_DEEP, gamma: float = 1.4, jitter: float = 0.3,
              chunk: int = 262_144) -> Workload:
    """L2-normalised mixture of 2,000 anisotropic Gaussians (the construction of sift_like,
    without rounding) with a steeper spectrum: measured by the same maximum-likelihood
    estimate (20 neighbours, 200,000 points), its local intrinsic dimension is 0.79 of
    sift_like's, the ratio of Deep100M's to SIFT1M's (10.2 / 12.9, Table 2)."""
    rng = _rng(seed)
    x = _aniso_mixture(rng, n + nq, d, n_clusters, gamma, 1.0, jitter, chunk)
    for s in range(0, n + nq, chunk):
        e = min(n + nq, s + chunk)
        x[s:e] /= np.linalg.norm(x[s:e], axis=1, keepdims=True)
    return Workload("deep_like", np.ascontiguousarray(x[:n]), np.ascontiguousarray(x[n:]),
                    K=100, L=100, R=32, alpha=60.0, n_nav=10,
                    info={"seed": seed, "n_clusters": n_clusters, "gamma": gamma})


def uniform_points(n: int, d: int, seed: int, integer: bool = False, hi: int = 255) -> np.ndarray:
    """Uniform points for tiny test cases: [0,1)^d floats, or integers 0..hi."""
    rng = _rng(seed)
    if integer:
        return rng.integers(0, hi + 1, size=(n, d)).astype(np.float32)
    return rng.random(size=(n, d)).astype(np.float32)


# --- navigating-node ids -------------------------------------------------------------
# SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable pseudorandom number
# generators", OOPSLA 2014; the constants are those of the published finaliser).
_M64 = (1 << 64) - 1


def splitmix64_stream(seed: int):
    state = seed & _M64
    while True:
        state = (state + 0x9E3779B97F4A7C15) & _M64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        yield z ^ (z >> 31)


def nav_ids(n: int, s: int, seed: int) -> np.ndarray:
    """s distinct node ids in draw order: successive SplitMix64 outputs modulo n,
    repeats skipped.  The library draws the same ids when it is given only a seed."""
    if s > n:
        raise ValueError("more navigating nodes than points")
    out: list[int] = []
    seen: set[int] = set()
    for z in splitmix64_stream(seed):
        v = int(z % n)
        if v not in seen:
            seen.add(v)
            out.append(v)
            if len(out) == s:
                break
    return np.asarray(out, dtype=np.int32)


CONFIGS = {
    "small": small,
    "sift_like": sift_like,
    "gist_like": gist_like,
    "deep_like": deep_like,
}
