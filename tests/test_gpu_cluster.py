"""Chromaticity clustering (Sec. 4.1) on the GPU against the oracle's clustering.

The histogram counts are integers and every decision (bin, nearest centre,
merge) is taken on the same values on both sides (FP32 chromaticity with the
same operation order, FP64 distances), so the cluster count and every pixel's
label must be identical; the initial base colours (FP64 means of FP32 values,
summed in a different order) within 1e-5.  Then the whole path from RGB alone:
clustering, then the decomposition, at the solver's parity bar.
"""
import numpy as np
import pytest

import oracle as O
from paper_1908_01961_b300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


# the last case is the 640 x 480 K = 6 frame the benchmark clusters
@pytest.mark.parametrize("H,W,K,n_cells,seed", [(48, 64, 4, 12, 0), (120, 160, 6, 20, 3), (37, 29, 3, 7, 1),
                                                (480, 640, 6, 40, 0)])
def test_cluster_matches_oracle(H, W, K, n_cells, seed):
    from paper_1908_01961_b300 import gid
    f = synth.SyntheticVideo(H, W, K, n_cells, seed=seed).frame(0)
    I = f.I.astype(np.float32)
    lab, b = gid.cluster(torch.from_numpy(I).cuda(), 10, 0.2)
    lo, bo, _ = O.cluster(I, 10, 0.2)
    assert b.shape == bo.shape, (b.shape, bo.shape)
    assert np.array_equal(lab.cpu().numpy(), lo)
    assert np.abs(b - bo).max() <= 1e-5


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
