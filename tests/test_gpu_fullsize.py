"""The 640 x 480, K = 6 video workload at full size against the FP64 oracle.

The GPU runs frame 0 (cold start) and frame 1 (warm start, temporal pairs) with
8 Gauss-Newton x 20 PCG steps each, in the configuration the benchmark times
(autotuned operator tile, graph replay).  The oracle runs frame 0 from the same
start, and frame 1 from the GPU's own frame-0 state (cast to FP64), so that it
need not replay the chain.  Bar: every layer within 1e-3 max-abs, energy within
1e-4 relative.  About a minute of single-core oracle time.
"""
import numpy as np
import pytest

import oracle as O
from harness import Case
from paper_1908_01961_b300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")


def test_video_640x480_two_frames_against_oracle():
    cfg = synth.VIDEO_640x480
    N, M = cfg["N"], cfg["M"]
    case = Case(cfg["H"], cfg["W"], cfg["K"], cfg["n_cells"], seed=0, frames=2, temporal=True)
    s = case.solver()
    rgb, lab = case.gpu_inputs(0)
    s.set_frame(rgb, lab)
    s.init(0)
    rows, _ = s.autotune(5)
    s.init(0)
    s.run(N, M)
    R0, T0 = s.layers()
    X0_gpu = s.state().cpu().numpy().astype(np.float64)
    b0_gpu = s.base_colors().astype(np.float64)
    E0, _ = s.energy()
    pb0 = case.oracle_problem(0)
    X0, b0, hist0 = O.solve_frame(pb0, pb0.init_cold(), N, M)
    assert np.abs(R0.cpu().numpy() - np.exp(X0[:3])).max() <= 1e-3
    assert np.abs(T0.cpu().numpy() - X0[3:]).max() <= 1e-3
    assert np.abs(b0_gpu - b0).max() <= 1e-3
    assert E0 == pytest.approx(hist0[-1].sum(), rel=1e-4)
    # frame 1: warm start with temporal pairs; the oracle starts from the GPU's frame-0 state
    rgb, lab = case.gpu_inputs(1)
    s.set_frame(rgb, lab)
    s.init(1)
    s.run(N, M)
    R1, T1 = s.layers()
    E1, _ = s.energy()
    pb1 = case.oracle_problem(1, rprev=X0_gpu[:3], b=b0_gpu)
    X1, b1, hist1 = O.solve_frame(pb1, X0_gpu, N, M)
    assert np.abs(R1.cpu().numpy() - np.exp(X1[:3])).max() <= 1e-3
    assert np.abs(T1.cpu().numpy() - X1[3:]).max() <= 1e-3
    assert np.abs(s.base_colors() - b1).max() <= 1e-3
    assert E1 == pytest.approx(hist1[-1].sum(), rel=1e-4)
