"""Seeded synthetic video frames for the illumination decomposition solver.

This module only *draws inputs*: it holds none of the solver's arithmetic and is
shared by the CUDA path, the FP64 oracle, the tests and the benchmark.  Every
array is float64 / uint8 numpy; callers cast as they need.

The frames follow the image-formation model of Sec. 3 (eq:imageformation),
``I = R * (T_0 + sum_k b_k T_k) + noise``, with

* reflectance ``R = b_label`` on a Voronoi partition (piecewise constant, as the
  reflectance sparsity prior of Sec. 5.1 assumes);
* direct shading ``T_0 = 0.2 + 0.8 * normalise(q(u, v))``, q a seeded quadratic
  whose linear part rotates with a light angle ``theta_t = theta_0 + 0.03 t``;
* indirect layers ``T_k = 0.15 * (G_sigma * 1[label = k]) * T_0 * 1[label != k]``
  -- light bounced off nearby surfaces of base colour k (first bounce only, the
  third assumption of Sec. 3), sigma = W / 80;
* Gaussian pixel noise, sigma 0.01.

Labels are the ground-truth Voronoi labels (the ideal output of the
chromaticity clustering of Sec. 4.1); the initial base colours are the mean RGB
of each label's pixels, the initialisation Sec. 4.1 prescribes.
Random pair offsets for the spatio-temporal consistency prior are drawn here too
and passed to both implementations as inputs.
"""
from __future__ import annotations

import dataclasses

import numpy as np
from scipy.ndimage import gaussian_filter


@dataclasses.dataclass
class Frame:
    I: np.ndarray          # (3, H, W) float64, planar RGB
    labels: np.ndarray     # (H, W) uint8, 0..K-1 -> base colour k = label + 1
    R: np.ndarray          # (3, H, W) ground-truth reflectance
    T: np.ndarray          # (K + 1, H, W) ground-truth T_0..T_K
    b: np.ndarray          # (K, 3) ground-truth base colours b_1..b_K


def base_colors(rng: np.random.Generator, K: int, lo=0.1, hi=0.9, min_dist=0.1) -> np.ndarray:
    """K colours uniform in [lo, hi]^3, redrawn until every pair is >= min_dist apart."""
    for _ in range(10000):
        b = rng.uniform(lo, hi, size=(K, 3))
        d = np.linalg.norm(b[:, None, :] - b[None, :, :], axis=-1)
        d[np.arange(K), np.arange(K)] = np.inf
        if K < 2 or d.min() >= min_dist:
            return b
    raise RuntimeError("could not draw separated base colours")


def _grid(H: int, W: int):
    v, u = np.meshgrid((np.arange(H) + 0.5) / H * 2 - 1, (np.arange(W) + 0.5) / W * 2 - 1, indexing="ij")
    return u, v


def voronoi_labels(H: int, W: int, sites: np.ndarray, cell_label: np.ndarray) -> np.ndarray:
    """Label of the nearest site (sites are (n, 2) float pixel positions y, x)."""
    from scipy.spatial import cKDTree
    yy, xx = np.meshgrid(np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
    _, nearest = cKDTree(np.asarray(sites, np.float64)).query(np.stack([yy.ravel(), xx.ravel()], axis=1))
    return np.asarray(cell_label, np.uint8)[nearest].reshape(H, W)


def direct_shading(H: int, W: int, coef: np.ndarray, theta: float) -> np.ndarray:
    u, v = _grid(H, W)
    a1, a2, a3, a4 = coef
    q = a1 * (u * np.cos(theta) + v * np.sin(theta)) + a2 * u * u + a3 * v * v + a4 * u * v
    q = (q - q.min()) / max(q.max() - q.min(), 1e-12)
    return 0.2 + 0.8 * q


def indirect_layers(labels: np.ndarray, T0: np.ndarray, K: int, sigma: float, strength=0.15) -> np.ndarray:
    T = np.zeros((K,) + labels.shape)
    for k in range(K):
        m = (labels == k).astype(np.float64)
        T[k] = strength * gaussian_filter(m, sigma, mode="nearest") * T0 * (1.0 - m)
    return T


def compose(labels, b, T0, Tk):
    """Noise-free I = R * (T_0 + sum_k b_k T_k) and R, for the synthetic ground truth."""
    R = b[labels].transpose(2, 0, 1)                     # (3, H, W)
    S = T0[None] + np.einsum("kc,khw->chw", b, Tk)
    return R * S, R


def initial_base_colors(I: np.ndarray, labels: np.ndarray, K: int) -> np.ndarray:
    """Mean RGB of each label's pixels (Sec. 4.1 initial base colours)."""
    b = np.zeros((K, 3))
    for k in range(K):
        m = labels == k
        b[k] = I[:, m].mean(axis=1) if m.any() else 0.5
    return b


def pair_offsets(rng: np.random.Generator, n: int, radius: int, include_zero: bool) -> np.ndarray:
    """n distinct (dy, dx) offsets in [-radius, radius]^2; no offset is the negative of another.

    With include_zero the first offset is (0, 0) (same pixel in the previous
    frame) and n - 1 non-zero ones follow.
    """
    cand = [(dy, dx) for dy in range(-radius, radius + 1) for dx in range(-radius, radius + 1)
            if (dy, dx) != (0, 0)]
    out = [(0, 0)] if include_zero else []
    order = rng.permutation(len(cand))
    for i in order:
        if len(out) >= n:
            break
        o = cand[i]
        if o in out or (-o[0], -o[1]) in out:
            continue
        out.append(o)
    return np.asarray(out, dtype=np.int32).reshape(-1, 2)


class SyntheticVideo:
    """Seeded video: Voronoi reflectance moving 1-3 px/frame, rotating light."""

    def __init__(self, H: int, W: int, K: int, n_cells: int, seed: int = 0, noise: float = 0.01,
                 motion: bool = True):
        self.H, self.W, self.K, self.noise = H, W, K, noise
        rng = np.random.default_rng(seed)
        self.rng_noise = np.random.default_rng(seed + 7919)
        self.b = base_colors(rng, K)
        self.sites = rng.uniform([0, 0], [H, W], size=(n_cells, 2))
        lab = rng.integers(0, K, size=n_cells)
        lab[: min(K, n_cells)] = rng.permutation(K)[: min(K, n_cells)]
        self.cell_label = lab.astype(np.uint8)
        ang = rng.uniform(0, 2 * np.pi, size=n_cells)
        speed = rng.uniform(1.0, 3.0, size=n_cells) if motion else np.zeros(n_cells)
        self.vel = np.stack([np.sin(ang) * speed, np.cos(ang) * speed], axis=1)
        self.coef = np.concatenate([rng.uniform(0.5, 1.0, 1), rng.uniform(-0.5, 0.5, 3)])
        self.theta0 = rng.uniform(0, 2 * np.pi)
        self.sigma = W / 80.0

    def frame(self, t: int, noise: bool = True) -> Frame:
        H, W = self.H, self.W
        sites = np.mod(self.sites + t * self.vel, [H, W])
        labels = voronoi_labels(H, W, sites, self.cell_label)
        T0 = direct_shading(H, W, self.coef, self.theta0 + 0.03 * t)
        Tk = indirect_layers(labels, T0, self.K, self.sigma)
        I, R = compose(labels, self.b, T0, Tk)
        if noise and self.noise > 0:
            I = I + self.rng_noise.normal(0.0, self.noise, size=I.shape)
        T = np.concatenate([T0[None], Tk], axis=0)
        return Frame(I=I, labels=labels, R=R, T=T, b=self.b.copy())


# Workloads: (H, W, K, Voronoi cells, outer GN steps N, PCG steps M, frames, temporal)
SINGLE_64x48 = dict(H=48, W=64, K=4, n_cells=12, N=5, M=10, frames=1, temporal=False)
VIDEO_640x480 = dict(H=480, W=640, K=6, n_cells=40, N=8, M=20, frames=30, temporal=True)
STREAM_1080P = dict(H=1080, W=1920, K=8, n_cells=80, N=8, M=20, frames=300, temporal=True)

# Consistency prior pair sampling (spatial and temporal), same for every pixel.
N_SPATIAL_PAIRS = 4
N_TEMPORAL_PAIRS = 4
PAIR_RADIUS = 3


def offsets_for(seed: int):
    rng = np.random.default_rng(seed + 104729)
    return (pair_offsets(rng, N_SPATIAL_PAIRS, PAIR_RADIUS, include_zero=False),
            pair_offsets(rng, N_TEMPORAL_PAIRS, PAIR_RADIUS, include_zero=True))
