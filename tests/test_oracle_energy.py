"""Pins of the oracle's exact energy terms and per-frame precompute (CPU only).

Each test builds a state whose energy the paper's definitions fix in closed form
by a route other than the oracle's loops (a count of pixels times a per-pixel
value, a ramp's constant gradient, ...), so a dropped term, wrong sign, wrong
index or transposed operand in the oracle fails here.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_1908_01961_b300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def make_problem(H, W, K, seed=0, I=None, labels=None, b=None, wsr=None, off_s=((1, 2), (-2, 1)), omega=None,
                 **weights):
    rng = np.random.default_rng(seed)
    if labels is None:
        labels = rng.integers(0, K, size=(H, W)).astype(np.uint8)
    if b is None:
        b = rng.uniform(0.2, 0.8, size=(K, 3))
    if I is None:
        I = rng.uniform(0.1, 0.9, size=(3, H, W))
    if wsr is None:
        wsr = rng.uniform(0, 1, size=(H, W))
    off_s = np.asarray(off_s, np.int32).reshape(-1, 2)
    if omega is None:
        omega = rng.uniform(0, 1, size=(len(off_s), H, W))
    return O.Problem(I, labels, b, wsr, omega, off_s, **weights)


def test_default_parameters_match_paper():
    g = json.load(open(os.path.join(GOLDEN, "parameters.json")))
    for k, v in g.items():
        if k.startswith("_") or k == "pcg_steps_paper":
            continue
        assert O.DEFAULT_WEIGHTS[k] == v, k


def test_data_residual_zero_at_ground_truth():
    """eq:data-term vanishes on a noise-free frame built by eq:imageformation."""
    v = synth.SyntheticVideo(24, 32, 4, 6, seed=3, noise=0.0)
    f = v.frame(0, noise=False)
    X = np.concatenate([np.log(f.R), f.T])
    pb = make_problem(24, 32, 4, I=f.I, labels=f.labels, b=f.b)
    E = pb.energy(X)
    assert abs(E[0]) <= 1e-20 * 5000 * 24 * 32 * 3 + 1e-18
    # and the clustering term then vanishes too, since R = b_label
    assert abs(E[1]) < 1e-18


def test_data_term_closed_form():
    """Scaling T_0 of a grey-shaded frame by s leaves residual (1-s) I per channel."""
    H, W, K = 5, 7, 2
    rng = np.random.default_rng(1)
    labels = rng.integers(0, K, size=(H, W)).astype(np.uint8)
    b = rng.uniform(0.2, 0.8, size=(K, 3))
    R = b[labels].transpose(2, 0, 1)
    T0 = rng.uniform(0.3, 1.0, size=(H, W))
    I = R * T0
    X = np.concatenate([np.log(R), T0[None] * 0.9, np.zeros((K, H, W))])
    pb = make_problem(H, W, K, I=I, labels=labels, b=b)
    assert pb.energy(X)[0] == pytest.approx(5000 * np.sum((0.1 * I) ** 2), rel=1e-12)


def test_clustering_term_closed_form():
    H, W, K = 4, 6, 3
    pb = make_problem(H, W, K)
    d = np.array([0.1, -0.2, 0.05])
    X = pb.init_cold()
    X[:3] += d[:, None, None]
    assert pb.energy(X)[1] == pytest.approx(200 * H * W * np.sum(d ** 2), rel=1e-12)


@pytest.mark.parametrize("p", [1.0, 0.5])
def test_reflectance_sparsity_ramp(p):
    """r_c = a_c x + d_c y: interior gradient norm sqrt(|a|^2+|d|^2); the last
    column keeps only the y part, the last row only the x part, the corner none."""
    H, W, K = 5, 6, 2
    a, d = np.array([0.3, -0.1, 0.2]), np.array([-0.05, 0.15, 0.1])
    pb = make_problem(H, W, K, p=p)
    X = np.zeros((K + 4, H, W))
    yy, xx = np.mgrid[0:H, 0:W]
    for c in range(3):
        X[c] = a[c] * xx + d[c] * yy
    A, D = np.linalg.norm(a), np.linalg.norm(d)
    expect = 20 * ((H - 1) * (W - 1) * np.hypot(A, D) ** p + (H - 1) * D ** p + (W - 1) * A ** p)
    assert pb.energy(X)[2] == pytest.approx(expect, rel=1e-12)


def test_consistency_ramp_and_constant():
    H, W, K = 6, 7, 2
    offs = np.array([[1, 2], [-2, 1], [0, -3]], np.int32)
    pb = make_problem(H, W, K, off_s=offs, omega=np.ones((3, H, W)))
    X = np.zeros((K + 4, H, W))
    X[:3] = 0.37
    assert pb.energy(X)[3] == 0.0
    slope = 0.2
    X[:3] = slope * np.mgrid[0:H, 0:W][1]
    expect = sum(10 * (H - abs(dy)) * (W - abs(dx)) * 3 * (slope * dx) ** 2 for dy, dx in offs)
    assert pb.energy(X)[3] == pytest.approx(expect, rel=1e-12)


def test_monochrome_term():
    """Grey S (only T_0) gives 0; T_1 = t with b_1 = (1, 0, 0) gives 2 t^2 / 3 per pixel."""
    H, W, K = 4, 5, 2
    b = np.array([[1.0, 0.0, 0.0], [0.3, 0.6, 0.2]])
    pb = make_problem(H, W, K, b=b)
    X = pb.init_cold()
    assert abs(pb.energy(X)[4]) < 1e-25
    t = 0.3
    X[4] = t
    assert pb.energy(X)[4] == pytest.approx(10 * pb.wsr.sum() * 2 * t * t / 3, rel=1e-12)


def test_isparsity_smoothness_nonneg():
    H, W, K = 4, 5, 3
    pb = make_problem(H, W, K)
    X = pb.init_cold()
    X[3:] = 0.25
    E = pb.energy(X)
    assert E[5] == pytest.approx(3 * K * H * W * 0.25, rel=1e-12)   # T_0 excluded from i-sparsity
    assert E[6] == 0.0 and E[7] == 0.0                                # constant, non-negative layers
    s = 0.07
    X[3:] = -s * np.mgrid[0:H, 0:W][0]                                # ramp down the rows
    E = pb.energy(X)
    assert E[6] == pytest.approx(3 * (K + 1) * (H - 1) * W * s, rel=1e-12)
    assert E[7] == pytest.approx(1000 * (K + 1) * W * s * sum(range(H)), rel=1e-12)


def test_precompute_uniform_and_two_colour():
    """Uniform image: dC = 0, w_SR = 0, pair weights 1 inside and 0 outside.
    Two-colour split: w_SR = 1 - exp(-50 d) on the two boundary columns only."""
    H, W = 4, 6
    col = np.array([0.2, 0.5, 0.3])
    I = np.broadcast_to(col[:, None, None], (3, H, W)).copy()
    offs = np.array([[0, 2], [1, -1]], np.int32)
    C, wsr, om, _ = O.precompute(I, offs)
    assert np.allclose(C, (col / (col.sum() + 1e-6))[:, None, None], atol=1e-15)
    assert np.all(wsr == 0)
    assert np.all(om[0][:, : W - 2] == 1) and np.all(om[0][:, W - 2:] == 0)
    assert np.all(om[1][: H - 1, 1:] == 1) and np.all(om[1][H - 1] == 0) and np.all(om[1][:, 0] == 0)
    col2 = np.array([0.6, 0.1, 0.3])
    I[:, :, 3:] = col2[:, None, None]
    C, wsr, om, _ = O.precompute(I, offs)
    d = np.linalg.norm(col / (col.sum() + 1e-6) - col2 / (col2.sum() + 1e-6))
    expect = np.zeros((H, W))
    expect[:, 2:4] = 1 - np.exp(-50 * d)
    assert np.allclose(wsr, expect, atol=1e-15)
    # pair (x, x + (0, 2)) crosses the split for x = 1, 2
    assert np.allclose(om[0][:, 1:3], np.exp(-d * d / 0.05 ** 2), rtol=1e-12)


def test_temporal_pairs_weight_and_energy():
    H, W, K = 4, 5, 2
    rng = np.random.default_rng(5)
    I = rng.uniform(0.1, 0.9, size=(3, H, W))
    offs_t = np.array([[0, 0], [1, 1]], np.int32)
    C, wsr, om_s, om_t = O.precompute(I, np.zeros((0, 2), np.int32), offs_t, Iprev=I)
    assert np.all(om_t[0] == 1.0)                     # the same pixel, same chromaticity
    rprev = rng.normal(size=(3, H, W))
    pb = O.Problem(I, rng.integers(0, K, (H, W)), rng.uniform(0.2, 0.8, (K, 3)), wsr, om_s, np.zeros((0, 2)),
                   omega_t=om_t, off_t=offs_t, rprev=rprev)
    X = pb.init_cold()
    X[:3] = rprev + 0.1                                   # offset 0.1 against the previous frame
    E = pb.energy(X)[3]
    # offset (0,0) pairs contribute 10 * 1 * 3 * 0.01 per pixel; offset (1,1) its own
    e1 = sum(10 * om_t[1][y, x] * np.sum((X[:3, y, x] - rprev[:, y + 1, x + 1]) ** 2)
             for y in range(H - 1) for x in range(W - 1))
    assert E == pytest.approx(10 * 3 * 0.01 * H * W + e1, rel=1e-12)


def test_fit_direct_recovers_ground_truth_and_minimises_the_data_term():
    """At a noise-free frame the per-pixel refit of T_0 returns the true T_0
    (zero data residual); on a noisy frame it is the minimiser of the data term
    over T_0 (every perturbation raises it) and it is clipped at zero."""
    v = synth.SyntheticVideo(24, 32, 4, 6, seed=5, noise=0.0)
    f = v.frame(0, noise=False)
    X = np.concatenate([np.log(f.R), f.T])
    Xw = X.copy()
    Xw[3] = 0.3                                             # a wrong T_0
    assert np.allclose(O.fit_direct(f.I, Xw, f.b)[3], f.T[0], rtol=1e-12, atol=1e-14)
    rng = np.random.default_rng(2)
    I = f.I + rng.normal(0, 0.02, f.I.shape)
    pb = make_problem(24, 32, 4, I=I, labels=f.labels, b=f.b)
    Xf = O.fit_direct(I, Xw, f.b)
    E0 = pb.energy(Xf)[0]
    for d in (1e-3, -1e-3):
        Xp = Xf.copy()
        Xp[3] += d
        assert pb.energy(Xp)[0] > E0
    Xn = Xw.copy()
    Xn[4:] = 5.0                                            # indirect light far above the image
    assert np.all(O.fit_direct(f.I, Xn, f.b)[3] == 0.0)


def test_recombine_pins():
    """Sec. 7.4 recombination: unchanged colours and gains reproduce the
    image-formation model (the noise-free frame); zero gains leave direct light
    only; recolouring an object by a factor scales exactly its pixels; a new
    colour for one indirect layer changes only pixels that layer reaches."""
    v = synth.SyntheticVideo(24, 32, 4, 6, seed=9, noise=0.0)
    f = v.frame(0, noise=False)
    X = np.concatenate([np.log(f.R), f.T])
    K, ones = 4, np.ones(4)
    mask0 = np.zeros((24, 32), int)
    assert np.allclose(O.recombine(X, f.b, f.b, ones, mask0), f.I, rtol=1e-13, atol=1e-15)
    assert np.allclose(O.recombine(X, f.b, f.b, np.zeros(K), mask0), f.R * f.T[0], rtol=1e-13)
    j = 2
    mask = np.where(f.labels == j - 1, j, 0)
    bn = f.b.copy()
    bn[j - 1] *= 1.5
    out = O.recombine(X, f.b, bn, ones, mask)
    base = O.recombine(X, f.b, bn, ones, mask0)
    sel = f.labels == j - 1
    assert np.allclose(out[:, sel], 1.5 * base[:, sel], rtol=1e-13)
    assert np.allclose(out[:, ~sel], base[:, ~sel], rtol=1e-13)
    bk = f.b.copy()
    bk[0] = [0.9, 0.1, 0.1]
    key = O.recombine(X, f.b, bk, ones, mask0)
    untouched = f.T[1] == 0
    assert np.allclose(key[:, untouched], f.I[:, untouched], rtol=1e-13, atol=1e-15)
    assert not np.allclose(key[:, ~untouched], f.I[:, ~untouched])


def _blocks(colors, H=20, W=30):
    """An image of vertical stripes, one per colour."""
    I = np.zeros((3, H, W))
    n = len(colors)
    for i, c in enumerate(colors):
        I[:, :, i * W // n:(i + 1) * W // n] = np.asarray(c)[:, None, None]
    return I


def test_cluster_uniform_and_separated_colours():
    """One colour -> one cluster of that colour; colours whose chromaticities are
    far apart (> 0.2) -> one cluster each, the stripes as labels and the exact
    colours as initial base colours (Sec. 4.1)."""
    lab, b, _ = O.cluster(_blocks([(0.3, 0.5, 0.2)]), 10)
    assert b.shape == (1, 3) and np.all(lab == 0) and np.allclose(b[0], [0.3, 0.5, 0.2])
    cols = [(0.8, 0.1, 0.1), (0.1, 0.8, 0.1), (0.1, 0.1, 0.8)]
    I = _blocks(cols)
    lab, b, _ = O.cluster(I, 10)
    assert b.shape == (3, 3)
    for i, c in enumerate(cols):
        stripe = lab[:, i * 10:(i + 1) * 10]
        assert np.all(stripe == stripe[0, 0])
        assert np.allclose(b[stripe[0, 0]], c)
    assert len(set(lab[0, ::10])) == 3


def test_cluster_merges_close_chromaticities_and_respects_k_max():
    """Two colours 0.05 apart in chromaticity merge into the larger cluster (the
    0.2 threshold); with k_max = 2, four well separated colours give at most two
    clusters; brightness alone (same chromaticity) never separates pixels."""
    I = _blocks([(0.6, 0.3, 0.1), (0.55, 0.33, 0.12), (0.6, 0.3, 0.1)])
    lab, b, _ = O.cluster(I, 10)
    assert b.shape[0] == 1 and np.all(lab == 0)
    I = _blocks([(0.8, 0.1, 0.1), (0.1, 0.8, 0.1), (0.1, 0.1, 0.8), (0.45, 0.45, 0.1)], W=40)
    lab, b, _ = O.cluster(I, 2)
    assert 1 <= b.shape[0] <= 2
    I = _blocks([(0.2, 0.4, 0.1), (0.4, 0.8, 0.2)])             # same chromaticity, twice as bright
    lab, b, _ = O.cluster(I, 10)
    assert b.shape[0] == 1 and np.allclose(b[0], [0.3, 0.6, 0.15])


def test_cluster_weighted_kmeans_centre_is_population_weighted():
    """Bins of one cluster: the centre is the population-weighted mean of their
    mid-points (two bins 0.1 apart, populations 3:1)."""
    H, W = 4, 4
    I = np.zeros((3, H, W))
    I[:, :, :3] = np.array([0.62, 0.33, 0.05])[:, None, None]     # bin (6, 3, 0)
    I[:, :, 3:] = np.array([0.55, 0.42, 0.03])[:, None, None]     # bin (5, 4, 0)
    lab, b, cen = O.cluster(I, 10)
    assert cen.shape == (1, 3)
    assert np.allclose(cen[0], (3 * np.array([0.65, 0.35, 0.05]) + np.array([0.55, 0.45, 0.05])) / 4)


def test_cold_start_recovers_direct_shading_when_reflectance_is_the_cluster_colour():
    """Cold start (the paper states only R's initialisation, from R_cluster, Sec.
    4.1; T_0 = mean_c I / mean_c R_cluster is this build's reading): on a
    noise-free frame built by eq:imageformation with R = R_cluster and no
    indirect light, I_c = R_c T_0, so the cold start must return the true T_0
    at every pixel and the data residual must vanish."""
    H, W, K = 9, 13, 3
    rng = np.random.default_rng(7)
    labels = rng.integers(0, K, size=(H, W)).astype(np.uint8)
    b = rng.uniform(0.1, 0.9, size=(K, 3))
    T0 = rng.uniform(0.2, 1.0, size=(H, W))
    R = b[labels].transpose(2, 0, 1)
    I = R * T0[None]
    pb = make_problem(H, W, K, I=I, labels=labels, b=b)
    X = pb.init_cold()
    assert np.abs(X[3] - T0).max() <= 1e-14
    assert np.all(X[4:] == 0.0)
    assert np.abs(np.exp(X[:3]) - R).max() <= 1e-15
    assert pb.energy(X)[0] <= 1e-12


def test_cold_start_one_pixel_by_hand():
    """One pixel with non-grey reflectance and indirect light present:
    R = (0.2, 0.5, 0.8), T_0 = 0.7, T_1 = 0.3, b_1 = (0.9, 0.1, 0.4), so
    I = R * (T_0 + b_1 T_1) = (0.194, 0.365, 0.656).  The cold start ignores the
    indirect light: T_0 = mean_c I / mean_c R = 1.215 / 1.5 = 0.81, T_1 = 0."""
    b = np.array([[0.2, 0.5, 0.8], [0.9, 0.1, 0.4]])      # colour 1: the reflectance; colour 2: b_1
    I = np.array([0.194, 0.365, 0.656]).reshape(3, 1, 1)
    labels = np.zeros((1, 1), np.uint8)
    pb = make_problem(1, 1, 2, I=I, labels=labels, b=b, off_s=np.zeros((0, 2)), omega=np.zeros((0, 1, 1)))
    X = pb.init_cold()
    assert X[3, 0, 0] == pytest.approx(0.81, abs=1e-15)
    assert np.allclose(np.exp(X[:3, 0, 0]), [0.2, 0.5, 0.8], atol=1e-15)
    assert X[4, 0, 0] == 0.0 and X[5, 0, 0] == 0.0
