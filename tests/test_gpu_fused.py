"""The fused PCG step (gid_set_apply_tile(rows | GID_PCG_FUSED)) against the FP64 oracle.

One kernel per PCG step: the operator tile also performs the previous step's
vector update on its tile and halo, z and M^-1 q alternate between two buffers,
and rho of the next step comes from the expanded recurrence
rho - 2 alpha <z, q> + alpha^2 <q, M^-1 q> (one set of block partials per
step).  The arithmetic of a pixel is otherwise that of the two-kernel loop, so
the bars are the same: PCG delta within 1e-4 of its max after 10 steps, the
recorded rho history within 1e-4, layers within 1e-3 max-abs and energy within
1e-4 relative after the same N x M from the same start.  Frames cover several
tiles in both directions, ragged right and bottom tiles, K from 3 to 6 and
three tile heights; the 640 x 480 K = 6 frame runs with 128 x 17 tiles.
"""
import numpy as np
import pytest

import oracle as O
from harness import Case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = {
    "64x48_K4": dict(H=48, W=64, K=4, n_cells=12),
    "37x29_K3": dict(H=29, W=37, K=3, n_cells=7),
    "70x41_K6": dict(H=41, W=70, K=6, n_cells=9),
    "203x117_K5": dict(H=117, W=203, K=5, n_cells=15),
}


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def close(gpu, ref, tol, what=""):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    assert gpu.shape == ref.shape, (gpu.shape, ref.shape)
    err = np.abs(gpu - ref).max()
    scale = max(np.abs(ref).max(), 1e-30)
    assert err <= tol * scale, f"{what}: max err {err:.3e} vs scale {scale:.3e} (rel {err / scale:.3e})"


def fused_solver(case, rows=17):
    from paper_1908_01961_b300 import gid
    s = case.solver()
    s.set_apply_tile(rows | gid.FUSED)
    return s


def random_state(pb, seed):
    rng = np.random.default_rng(seed)
    X = pb.init_cold()
    X[:3] += rng.normal(0, 0.2, size=X[:3].shape)
    X[3:] += rng.normal(0, 0.05, size=X[3:].shape)
    return f32(X)


def test_layout_reports_the_fused_loop():
    from paper_1908_01961_b300 import gid
    s = gid.Solver(48, 64, 4, gid.default_weights())
    s.set_apply_tile(8 | gid.FUSED)
    rows, _ = s.pcg_layout()
    assert rows == 8 | gid.FUSED
    s.set_apply_tile(8)
    assert s.pcg_layout()[0] == 8


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("M", [1, 2, 10])
@pytest.mark.parametrize("rows", [2, 8, 17])
def test_fused_pcg_delta_and_rho(name, M, rows):
    case = Case(**CASES[name], seed=3)
    s = fused_solver(case, rows)
    rgb, lab = case.gpu_inputs()
    s.set_frame(rgb, lab)
    pb = case.oracle_problem()
    X = random_state(pb, 5)
    s.set_state(torch.from_numpy(X.astype(np.float32)).cuda())
    delta = s.stage_pcg(M)
    ref, rho = pb.pcg(X, M)
    close(delta.cpu().numpy(), ref, 1e-4, f"PCG delta, {M} steps, 128x{rows} tiles")
    h = s.pcg_history()
    assert len(h) == M
    np.testing.assert_allclose(h, rho[:M], rtol=1e-4, atol=1e-4 * rho[0])


@pytest.mark.parametrize("name", list(CASES))
def test_fused_end_to_end(name):
    """5 Gauss-Newton x 10 PCG, cold start, refinement on."""
    case = Case(**CASES[name], seed=0)
    s = fused_solver(case)
    rgb, lab = case.gpu_inputs()
    s.set_frame(rgb, lab)
    s.init(0)
    s.run(5, 10)
    R, T = s.layers()
    E, _ = s.energy()
    pb = case.oracle_problem()
    Xo, bo, hist = O.solve_frame(pb, pb.init_cold(), 5, 10)
    assert np.abs(R.cpu().numpy() - np.exp(Xo[:3])).max() <= 1e-3
    assert np.abs(T.cpu().numpy() - Xo[3:]).max() <= 1e-3
    assert np.abs(s.base_colors() - bo).max() <= 1e-3
    assert E == pytest.approx(hist[-1].sum(), rel=1e-4)


def test_fused_two_frames_temporal():
    """Frame 0 cold, frame 1 warm with temporal pairs (3 x 8 each)."""
    case = Case(H=48, W=64, K=4, n_cells=12, seed=1, frames=2, temporal=True)
    s = fused_solver(case, 8)
    rgb, lab = case.gpu_inputs(0)
    s.set_frame(rgb, lab)
    s.init(0)
    s.run(3, 8)
    X0 = s.state().cpu().numpy().astype(np.float64)
    b0 = s.base_colors().astype(np.float64)
    rgb, lab = case.gpu_inputs(1)
    s.set_frame(rgb, lab)
    s.init(1)
    s.run(3, 8)
    R, T = s.layers()
    E, _ = s.energy()
    pb = case.oracle_problem(1, rprev=X0[:3], b=b0)
    Xo, bo, hist = O.solve_frame(pb, X0, 3, 8)
    assert np.abs(R.cpu().numpy() - np.exp(Xo[:3])).max() <= 1e-3
    assert np.abs(T.cpu().numpy() - Xo[3:]).max() <= 1e-3
    assert E == pytest.approx(hist[-1].sum(), rel=1e-4)


def test_fused_is_bitwise_reproducible_and_agrees_with_the_two_kernel_loop():
    """Two fused solves give the same bits (fixed-order reductions, halo values
    computed by the same operation as their owners'); the two-kernel loop
    differs by the grouping of FP32 partial sums and by the rho recurrence."""
    case = Case(**CASES["70x41_K6"], seed=2)
    out = []
    for mode in ("fused", "fused", 17):
        s = fused_solver(case) if mode == "fused" else case.solver()
        if mode != "fused":
            s.set_apply_tile(mode)
        rgb, lab = case.gpu_inputs()
        s.set_frame(rgb, lab)
        s.init(0)
        s.run(4, 12)
        out.append(s.state().cpu().numpy())
    assert np.array_equal(out[0], out[1])
    assert np.abs(out[0] - out[2]).max() <= 1e-3


def test_autotune_times_the_fused_loops():
    from paper_1908_01961_b300 import gid
    case = Case(**CASES["203x117_K5"], seed=4)
    s = case.solver()
    rgb, lab = case.gpu_inputs()
    s.set_frame(rgb, lab)
    s.init(0)
    rows, us = s.autotune(3)
    assert set(us) == set(gid.AUTOTUNE_LOOPS)
    for r in (2, 4, 8, 17):
        assert us[r | gid.FUSED] > 0
    assert rows in gid.AUTOTUNE_LOOPS and us[rows] > 0
    assert us[rows] <= min(v for v in us.values() if v > 0) + 1e-6
    assert s.pcg_layout()[0] == rows


def test_fused_full_size_640x480_K6_pcg_delta():
    """The benchmark's frame size with 128 x 17 tiles: the PCG delta of one
    Gauss-Newton step (20 steps) from the cold start against the oracle's,
    over every pixel."""
    from paper_1908_01961_b300 import synth
    cfg = synth.VIDEO_640x480
    case = Case(cfg["H"], cfg["W"], cfg["K"], cfg["n_cells"], seed=0)
    s = fused_solver(case)
    rgb, lab = case.gpu_inputs()
    s.set_frame(rgb, lab)
    s.init(0)
    X = s.state().cpu().numpy().astype(np.float64)
    delta = s.stage_pcg(cfg["M"])
    ref, _ = case.oracle_problem().pcg(X, cfg["M"])
    close(delta.cpu().numpy(), ref, 1e-4, "PCG delta at 640x480")


@pytest.mark.parametrize("rows", [8, 17])
def test_fused_pcg_delta_k8(rows):
    """K = 8: at 17 rows the two staged tiles do not fit in shared memory, so the
    halo's M^-1 q comes from global memory (four chunks in flight per thread);
    at 8 rows both are staged.  PCG delta and rho history after 10 steps
    against the oracle."""
    case = Case(H=57, W=150, K=8, n_cells=10, seed=5)
    s = fused_solver(case, rows)
    rgb, lab = case.gpu_inputs()
    s.set_frame(rgb, lab)
    pb = case.oracle_problem()
    X = random_state(pb, 2)
    s.set_state(torch.from_numpy(X.astype(np.float32)).cuda())
    delta = s.stage_pcg(10)
    ref, rho = pb.pcg(X, 10)
    close(delta.cpu().numpy(), ref, 1e-4, f"fused PCG delta K=8, {rows} rows")
    np.testing.assert_allclose(s.pcg_history(), rho[:10], rtol=1e-4, atol=1e-4 * rho[0])
