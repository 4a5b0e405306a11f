"""Chromaticity clustering (Sec. 4.1) on the GPU against the oracle's clustering.

The oracle computes the chromaticity in FP64, the GPU in FP32 (at most a few
units in the last place apart, 4 * 2^-24 relative, for one add chain and one
division).  So the two may bin a pixel whose FP64 chromaticity lies within that
rounding of a bin edge differently; such a pixel moves one unit of population
between two bins, which shifts a centre by at most (bin spacing) * (pixels
binned differently) / (the cluster's population).  A pixel's label may then
differ only where its distances to its two closest centres differ by less than
twice (that shift + the chromaticity's rounding): every other label must match,
the cluster count must match, and the initial base colours (means of the
clusters' RGB) may move by at most the mismatched pixels' share of a cluster.
The counts of edge-ambiguous pixels and of mismatched labels are reported.
Then the whole path from RGB alone: clustering, then the decomposition, at the
solver's parity bar.
"""
import numpy as np
import pytest

import oracle as O
from paper_1908_01961_b300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ULP = 4 * 2.0 ** -24     # relative rounding of the FP32 chromaticity (add chain, division)


def ambiguity(I, centres, labels_o):
    """Per pixel: edge-ambiguous (within the FP32 rounding of a bin edge in some
    channel), the gap between its two closest FP64 centre distances, and the
    smallest oracle cluster population."""
    C = O.chromaticity(I)
    f = C * O.CLUSTER_BINS
    edge = (np.abs(f - np.round(f)) <= O.CLUSTER_BINS * ULP * np.maximum(np.abs(C), 1e-6) + 1e-12).any(axis=0)
    d = np.sqrt(((C[None] - centres[:, :, None, None]) ** 2).sum(1))
    ds = np.sort(d, axis=0)
    gap = ds[1] - ds[0] if len(centres) > 1 else np.full(C.shape[1:], np.inf)
    pop = np.bincount(labels_o.ravel(), minlength=len(centres))
    return edge, gap, C, pop


# the last case is the 640 x 480 K = 6 frame the benchmark clusters
@pytest.mark.parametrize("H,W,K,n_cells,seed", [(48, 64, 4, 12, 0), (120, 160, 6, 20, 3), (37, 29, 3, 7, 1),
                                                (480, 640, 6, 40, 0)])
def test_cluster_matches_oracle(H, W, K, n_cells, seed, record_property):
    from paper_1908_01961_b300 import gid
    f = synth.SyntheticVideo(H, W, K, n_cells, seed=seed).frame(0)
    I = f.I.astype(np.float32)
    lab, b = gid.cluster(torch.from_numpy(I).cuda(), 10, 0.2)
    lo, bo, cen = O.cluster(I, 10, 0.2)
    assert b.shape == bo.shape, (b.shape, bo.shape)
    edge, gap, C, pop = ambiguity(I, cen, lo)
    n_edge = int(edge.sum())
    shift = 0.1 * np.sqrt(3.0) * n_edge / max(int(pop.min()), 1)
    tol = 2.0 * (shift + ULP * np.sqrt((C * C).sum(0)))
    lg = lab.cpu().numpy()
    mism = lg != lo
    record_property("edge_ambiguous_pixels", n_edge)
    record_property("label_mismatches", int(mism.sum()))
    print(f"{H}x{W}: {n_edge} pixels within FP32 rounding of a bin edge, {int(mism.sum())} labels differ")
    assert np.all(gap[mism] <= tol[mism]), (int(mism.sum()), float(gap[mism].max()) if mism.any() else 0.0)
    # colours: the oracle's cluster means; a mismatched pixel moves at most its own RGB between two means
    bound = 1e-5 + float(mism.sum()) / max(int(pop.min()), 1) * 2.0 * float(np.abs(I).max())
    assert np.abs(b - bo).max() <= bound


def test_decomposition_from_rgb_alone():
    """Frame -> GPU clustering -> solve (3 x 8, cold), against the oracle's
    clustering and solve of the same frame."""
    from paper_1908_01961_b300 import gid
    H, W = 48, 64
    f = synth.SyntheticVideo(H, W, 4, 12, seed=5).frame(0)
    I = f.I.astype(np.float32)
    rgb = torch.from_numpy(I).cuda()
    lab, b = gid.cluster(rgb, 10, 0.2)
    lo, bo, _ = O.cluster(I, 10, 0.2)
    K = b.shape[0]
    off_s, _ = synth.offsets_for(5)
    s = gid.Solver(H, W, K, gid.default_weights(off_s))
    s.set_base_colors(b)
    s.set_frame(rgb, lab)
    s.init(0)
    s.run(3, 8)
    R, T = s.layers()
    E, _ = s.energy()
    I64 = I.astype(np.float64)
    C, wsr, om, _ = O.precompute(I64, off_s)
    pb = O.Problem(I64, lo, b.astype(np.float64), wsr, om, off_s)
    Xo, b_o, hist = O.solve_frame(pb, pb.init_cold(), 3, 8)
    assert np.abs(R.cpu().numpy() - np.exp(Xo[:3])).max() <= 1e-3
    assert np.abs(T.cpu().numpy() - Xo[3:]).max() <= 1e-3
    assert np.abs(s.base_colors() - b_o).max() <= 1e-3
    assert E == pytest.approx(hist[-1].sum(), rel=1e-4)
