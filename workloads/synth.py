"""Seeded synthetic KDE workloads shaped like the paper's experiments.

The paper (Section 7) evaluates monochromatic kernel density estimation on
real datasets scaled to the unit hypercube, swept over bandwidths spanning
several decades around the LSCV-optimal one.  Those datasets are not
available here, so these generators produce clustered Gaussian-mixture data
of the same kind (points in [0,1]^D, monochromatic unless stated, bandwidths
log-spaced over three decades of the data diameter).

This module only draws random numbers and arranges them into arrays.  It holds
none of the summation arithmetic: the CUDA path and the CPU oracle both consume
its output, and neither imports the other.

Every generator is deterministic: one numpy PCG64 stream per role (means,
covariances, labels, points, weights) spawned from a fixed seed, so the oracle
and the GPU path see byte-identical inputs.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEEDS = {1: 1206685701, 2: 1206685702, 3: 1206685703, 4: 1206685704, 5: 1206685705}


@dataclasses.dataclass
class Workload:
    name: str
    queries: np.ndarray          # M x D, row-major, float32 or float64
    refs: np.ndarray             # N x D (the same array object when monochromatic)
    weights: np.ndarray          # N, float32, all > 0
    h: np.ndarray                # nh bandwidths, float64
    eps: float
    leaf_size: int
    mono: bool
    diameter: float

    @property
    def D(self) -> int:
        return int(self.refs.shape[1])

    @property
    def M(self) -> int:
        return int(self.queries.shape[0])

    @property
    def N(self) -> int:
        return int(self.refs.shape[0])


def _streams(seed: int, n: int):
    ss = np.random.SeedSequence(seed)
    return [np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(n)]


def bbox_diagonal(x: np.ndarray) -> float:
    """Data diameter: length of the bounding-box diagonal of a point set."""
    x64 = np.asarray(x, dtype=np.float64)
    ext = x64.max(axis=0) - x64.min(axis=0)
    return float(np.sqrt(np.sum(ext * ext)))


def log_bandwidths(diameter: float, n: int, lo: float = 1e-3, hi: float = 1.0) -> np.ndarray:
    """n bandwidths log-spaced from lo*diameter to hi*diameter."""
    return diameter * np.logspace(math.log10(lo), math.log10(hi), n)


def _haar_orthogonal(rng: np.random.Generator, d: int) -> np.ndarray:
    a = rng.standard_normal((d, d))
    q, r = np.linalg.qr(a)
    return q * np.sign(np.diag(r))


def _rejection_mixture(rng_lab, rng_pts, means, chol, n, lo=0.0, hi=1.0):
    """Draw n points from an equal-mass Gaussian mixture, rejecting points
    outside [lo,hi]^D (redrawn until n are accepted)."""
    k, d = means.shape
    out = np.empty((0, d))
    while out.shape[0] < n:
        m = (n - out.shape[0]) * 2 + 16
        lab = rng_lab.integers(0, k, m)
        z = rng_pts.standard_normal((m, d))
        x = means[lab] + np.einsum("mij,mj->mi", chol[lab], z)
        ok = np.all((x >= lo) & (x <= hi), axis=1)
        out = np.concatenate([out, x[ok]])
    return out[:n]


def config1(scale: float = 1.0) -> Workload:
    """D=2 monochromatic KDE: 4 isotropic Gaussians (sigma 0.05), FP64 points,
    w=1/N, one bandwidth h=0.01, eps=1e-2, leaf size 32."""
    n = max(2, int(round(10_000 * scale)))
    r_mean, r_cov, r_lab, r_pts, r_w = _streams(SEEDS[1], 5)
    means = r_mean.uniform(0.15, 0.85, (4, 2))
    chol = np.broadcast_to(0.05 * np.eye(2), (4, 2, 2))
    x = _rejection_mixture(r_lab, r_pts, means, chol, n)
    w = np.full(n, 1.0 / n, dtype=np.float32)
    return Workload("kde_d2_n%d_mono_fp64" % n, x, x, w, np.array([0.01]), 1e-2, 32, True,
                    bbox_diagonal(x))


def config2(scale: float = 1.0, nh: int = 16) -> Workload:
    """D=3 monochromatic bandwidth sweep: 95% from 16 anisotropic Gaussians
    (Haar rotations, eigenvalues log-uniform in [s^2/10, s^2], s=0.04) plus 5%
    uniform background, FP32, w=1/N, 16 log-spaced bandwidths 1e-3..1 times the
    diameter, eps=1e-2."""
    n = max(2, int(round(1_000_000 * scale)))
    r_mean, r_cov, r_lab, r_pts, r_w = _streams(SEEDS[2], 5)
    k, d, s = 16, 3, 0.04
    means = r_mean.uniform(0.1, 0.9, (k, d))
    chol = np.empty((k, d, d))
    for i in range(k):
        rot = _haar_orthogonal(r_cov, d)
        lam = np.exp(r_cov.uniform(math.log(s * s / 10), math.log(s * s), d))
        chol[i] = rot @ np.diag(np.sqrt(lam))
    n_bg = int(round(0.05 * n))
    x_mix = _rejection_mixture(r_lab, r_pts, means, chol, n - n_bg)
    x_bg = r_pts.uniform(0.0, 1.0, (n_bg, d))
    x = np.concatenate([x_mix, x_bg])
    x = x[r_lab.permutation(n)].astype(np.float32)
    w = np.full(n, 1.0 / n, dtype=np.float32)
    diam = bbox_diagonal(x)
    return Workload("kde_d3_n%d_mono_sweep%d" % (n, nh), x, x, w, log_bandwidths(diam, nh), 1e-2,
                    32, True, diam)


def config3(scale: float = 1.0, nh: int = 8, eps: float = 1e-3) -> Workload:
    """D=5 monochromatic series-expansion regime: 64 isotropic clusters
    (sigma 0.02), FP32, w=1/N, 8 log-spaced bandwidths, eps 1e-3 or 1e-4."""
    n = max(2, int(round(500_000 * scale)))
    r_mean, r_cov, r_lab, r_pts, r_w = _streams(SEEDS[3], 5)
    k, d = 64, 5
    means = r_mean.uniform(0.1, 0.9, (k, d))
    chol = np.broadcast_to(0.02 * np.eye(d), (k, d, d))
    x = _rejection_mixture(r_lab, r_pts, means, chol, n).astype(np.float32)
    w = np.full(n, 1.0 / n, dtype=np.float32)
    diam = bbox_diagonal(x)
    return Workload("kde_d5_n%d_mono_eps%g" % (n, eps), x, x, w, log_bandwidths(diam, nh), eps,
                    32, True, diam)


def config4(scale: float = 1.0, nh: int = 8) -> Workload:
    """D=16 bichromatic: 32 Gaussians on a random 4-D subspace (sigma 0.05 in
    the subspace, means U[0.2,0.8]^4, offset 0.5 in every coordinate) plus
    isotropic noise 0.01; N refs, M=N/10 queries from separate streams, weights
    U(0.5,1.5), 8 bandwidths, eps=1e-2."""
    n = max(2, int(round(2_000_000 * scale)))
    m = max(1, int(round(200_000 * scale)))
    r_mean, r_basis, r_lab, r_pts, r_w, r_qlab, r_qpts = _streams(SEEDS[4], 7)
    k, d, sub = 32, 16, 4
    basis = np.linalg.qr(r_basis.standard_normal((d, sub)))[0]      # d x 4 orthonormal
    means = r_mean.uniform(0.2, 0.8, (k, sub))

    def draw(rl, rp, cnt):
        lab = rl.integers(0, k, cnt)
        z = means[lab] + 0.05 * rp.standard_normal((cnt, sub))
        x = 0.5 + (z - 0.5) @ basis.T + 0.01 * rp.standard_normal((cnt, d))
        return x.astype(np.float32)

    refs = draw(r_lab, r_pts, n)
    qs = draw(r_qlab, r_qpts, m)
    w = r_w.uniform(0.5, 1.5, n).astype(np.float32)
    diam = bbox_diagonal(refs)
    return Workload("kde_d16_n%d_m%d_bichromatic" % (n, m), qs, refs, w, log_bandwidths(diam, nh),
                    1e-2, 32, False, diam)


def config5_problem(index: int, scale: float = 1.0, nh: int = 8) -> Workload:
    """One of the 256 independent batched problems: N=M log-uniform in
    [1e3, 2e5] (times scale), D uniform in {2..8}, k~U{2..16} clusters with
    sigma~U[0.01,0.08], w=1/N, 8 bandwidths, eps=1e-2."""
    ss = np.random.SeedSequence([SEEDS[5], index])
    r_meta, r_mean, r_lab, r_pts = [np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(4)]
    n = int(round(math.exp(r_meta.uniform(math.log(1e3), math.log(2e5))) * scale))
    n = max(2, n)
    d = int(r_meta.integers(2, 9))
    k = int(r_meta.integers(2, 17))
    sig = r_meta.uniform(0.01, 0.08, k)
    means = r_mean.uniform(0.1, 0.9, (k, d))
    chol = sig[:, None, None] * np.eye(d)[None]
    x = _rejection_mixture(r_lab, r_pts, means, chol, n).astype(np.float32)
    w = np.full(n, 1.0 / n, dtype=np.float32)
    diam = bbox_diagonal(x)
    return Workload("kde_batch%03d_d%d_n%d" % (index, d, n), x, x, w, log_bandwidths(diam, nh),
                    1e-2, 32, True, diam)


def config5(scale: float = 1.0, count: int = 256, nh: int = 8):
    return [config5_problem(i, scale, nh) for i in range(count)]


def lscv_bandwidths(h: np.ndarray) -> np.ndarray:
    """The bandwidth list an LSCV evaluation sums over: every h followed by
    every sqrt(2)*h (the self-convolution width of a Gaussian kernel)."""
    h = np.asarray(h, dtype=np.float64)
    return np.concatenate([h, h * math.sqrt(2.0)])


def small_random(seed: int, n: int, d: int, m: int | None = None, dtype=np.float32,
                 clusters: int = 3, sigma: float = 0.05, wlo: float = 0.5, whi: float = 1.5):
    """A small seeded clustered problem for unit tests: returns
    (queries, refs, weights); queries is refs when m is None."""
    r_mean, r_lab, r_pts, r_w, r_q = _streams(seed, 5)
    means = r_mean.uniform(0.2, 0.8, (clusters, d))
    lab = r_lab.integers(0, clusters, n)
    refs = (means[lab] + sigma * r_pts.standard_normal((n, d))).astype(dtype)
    w = r_w.uniform(wlo, whi, n).astype(np.float32)
    if m is None:
        return refs, refs, w
    qlab = r_q.integers(0, clusters, m)
    qs = (means[qlab] + sigma * r_q.standard_normal((m, d))).astype(dtype)
    return qs, refs, w
