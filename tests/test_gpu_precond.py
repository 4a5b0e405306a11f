"""Block-Jacobi PCG on the GPU (gid_set_preconditioner) against the oracle's
block-Jacobi PCG, element by element.

The per-pixel blocks are factored in FP32 (Cholesky), so the preconditioner
step carries the rounding of a small dense solve on top of the Jacobi path's:
the PCG-delta bar stays at 1e-4 of max |delta| after 10 steps, and the
end-to-end bar is the solver's (layers within 1e-3 max-abs, energy within 1e-4
relative).
"""
import numpy as np
import pytest

import oracle as O
from harness import Case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = {
    "64x48_K4": dict(H=48, W=64, K=4, n_cells=12),
    "37x29_K3": dict(H=29, W=37, K=3, n_cells=7),      # partial tiles in x and y
    "70x41_K6": dict(H=41, W=70, K=6, n_cells=9),
    "150x33_K9": dict(H=33, W=150, K=9, n_cells=10),   # the largest block (13 x 13)
}


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def random_state(pb, seed):
    rng = np.random.default_rng(seed)
    X = pb.init_cold()
    X[:3] += rng.normal(0, 0.2, size=X[:3].shape)
    X[3:] += rng.normal(0, 0.05, size=X[3:].shape)
    return f32(X)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("M", [1, 10])
def test_block_jacobi_pcg_delta(name, M):
    case = Case(**CASES[name], seed=3)
    s = case.solver()
    s.set_preconditioner("block")
    assert s.preconditioner() == "block"
    rgb, lab = case.gpu_inputs()
    s.set_frame(rgb, lab)
    pb = case.oracle_problem()
    X = random_state(pb, 5)
    s.set_state(torch.from_numpy(X.astype(np.float32)).cuda())
    delta = s.stage_pcg(M).cpu().numpy()
    ref, _ = pb.pcg_variant(X, M, block=True)
    err = np.abs(delta - ref).max()
    assert err <= 1e-4 * np.abs(ref).max(), f"max err {err:.3e} vs {np.abs(ref).max():.3e}"
    # and it is not the Jacobi iterate
    jac, _ = pb.pcg(X, M)
    assert np.abs(jac - ref).max() > 1e-2 * np.abs(ref).max()


@pytest.mark.parametrize("name", ["64x48_K4", "37x29_K3", "70x41_K6"])
def test_block_jacobi_end_to_end(name):
    """5 Gauss-Newton x 10 PCG, cold start, base-colour refinement on (graph replay)."""
    case = Case(**CASES[name], seed=0)
    s = case.solver()
    s.set_preconditioner("block")
    rgb, lab = case.gpu_inputs()
    s.set_frame(rgb, lab)
    s.init(0)
    s.run(5, 10)
    R, T = s.layers()
    E, _ = s.energy()
    pb = case.oracle_problem()
    Xo, bo, hist = O.solve_frame(pb, pb.init_cold(), 5, 10, block=True)
    assert np.abs(R.cpu().numpy() - np.exp(Xo[:3])).max() <= 1e-3
    assert np.abs(T.cpu().numpy() - Xo[3:]).max() <= 1e-3
    assert np.abs(s.base_colors() - bo).max() <= 1e-3
    assert E == pytest.approx(hist[-1].sum(), rel=1e-4)


def test_block_jacobi_two_frames_temporal():
    """Frame 1 warm-started with temporal pairs: the block path under the temporal prior."""
    case = Case(H=48, W=64, K=4, n_cells=12, seed=1, frames=2, temporal=True)
    s = case.solver()
    s.set_preconditioner("block")
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
    Xo, bo, hist = O.solve_frame(pb, X0, 3, 8, block=True)
    assert np.abs(R.cpu().numpy() - np.exp(Xo[:3])).max() <= 1e-3
    assert np.abs(T.cpu().numpy() - Xo[3:]).max() <= 1e-3
    assert E == pytest.approx(hist[-1].sum(), rel=1e-4)


def test_switching_back_to_jacobi_is_the_default_path():
    """Block, then Jacobi again: the cached graphs are dropped and the result is
    bit for bit a fresh Jacobi solver's."""
    case = Case(**CASES["70x41_K6"], seed=0)
    rgb, lab = case.gpu_inputs()
    out = []
    for switch in (False, True):
        s = case.solver()
        s.set_frame(rgb, lab)
        if switch:
            s.set_preconditioner("block")
            s.init(0)
            s.run(2, 5)
            s.set_preconditioner("jacobi")
            s.new_sequence()
            s.set_base_colors(case.b_init)
            s.set_frame(rgb, lab)
        s.init(0)
        s.run(3, 6)
        out.append(s.state().cpu().numpy())
    assert np.array_equal(out[0], out[1])


def test_bad_preconditioner_is_rejected():
    from paper_1908_01961_b300 import gid
    case = Case(**CASES["37x29_K3"], seed=0)
    s = case.solver()
    with pytest.raises(gid.GidError):
        s._chk(s.lib.gid_set_preconditioner(s.h, 7))
    assert s.preconditioner() == "jacobi"


@pytest.mark.slow
def test_block_jacobi_full_size_640x480_K6():
    """The 640 x 480 K = 6 frame in the launch configuration the benchmark times
    (128 x 17 operator tile): 20 block-Jacobi PCG steps from the cold start
    against the oracle's, then one outer iteration end to end."""
    case = Case(H=480, W=640, K=6, n_cells=40, seed=0)
    s = case.solver()
    s.set_preconditioner("block")
    s.set_apply_tile(17)
    rgb, lab = case.gpu_inputs()
    s.set_frame(rgb, lab)
    s.init(0)
    X = s.state().cpu().numpy().astype(np.float64)
    pb = case.oracle_problem()
    delta = s.stage_pcg(20).cpu().numpy()
    ref, _ = pb.pcg_variant(X, 20, block=True)
    err = np.abs(delta - ref).max()
    assert err <= 1e-4 * np.abs(ref).max(), f"max err {err:.3e} vs {np.abs(ref).max():.3e}"
    s.run(1, 20)
    R, T = s.layers()
    E, _ = s.energy()
    Xo, bo, hist = O.solve_frame(pb, X, 1, 20, block=True)
    assert np.abs(R.cpu().numpy() - np.exp(Xo[:3])).max() <= 1e-3
    assert np.abs(T.cpu().numpy() - Xo[3:]).max() <= 1e-3
    assert np.abs(s.base_colors() - bo).max() <= 1e-3
    assert E == pytest.approx(hist[-1].sum(), rel=1e-4)


def test_batch_uses_each_contexts_preconditioner():
    """Contexts of a batch set to block-Jacobi before its first run give, bit for
    bit, what the same videos give solved one context at a time."""
    from paper_1908_01961_b300 import gid
    shapes = [dict(H=48, W=64, K=4, n_cells=12), dict(H=41, W=70, K=6, n_cells=9)]
    cs = [Case(**sh, seed=20 + i, frames=2, temporal=True) for i, sh in enumerate(shapes)]
    single = []
    for c in cs:
        s = c.solver()
        s.set_preconditioner("block")
        s.set_apply_tile(8)
        for t in range(2):
            rgb, lab = c.gpu_inputs(t)
            s.set_frame(rgb, lab)
            s.init(0 if t == 0 else 1)
            s.run(3, 6)
        single.append((s.state().cpu().numpy(), s.base_colors()))
    weights = [gid.default_weights(c.off_s, c.off_t, temporal=1) for c in cs]
    b = gid.Batch([(c.H, c.W, c.K) for c in cs], weights)
    for v, c in zip(b.videos, cs):
        v.set_base_colors(c.b_init)
        v.set_apply_tile(8)
        v.set_preconditioner("block")
    for t in range(2):
        ins = [c.gpu_inputs(t) for c in cs]
        b.set_frames([i[0] for i in ins], [i[1] for i in ins])
        b.init(0 if t == 0 else 1)
        b.run(3, 6)
    for v, (X, bc) in zip(b.videos, single):
        assert v.preconditioner() == "block"
        assert np.array_equal(v.state().cpu().numpy(), X)
        assert np.array_equal(v.base_colors(), bc)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("loop", ["fused", "resident"])
def test_single_reduction_pcg_matches_its_oracle_recurrence(name, loop):
    """The single-reduction (one grid-wide reduction per PCG step) recurrence on
    the GPU, as the fused step and as the resident loop run it, against the
    oracle's single-reduction variant: PCG delta after 10 steps within 1e-4 of
    its max, and the rho history within 1e-4; the oracle's two recurrences agree
    in exact arithmetic, so the GPU is also within the bar of the textbook one."""
    from paper_1908_01961_b300 import gid
    case = Case(**CASES[name], seed=3)
    s = case.solver()
    if loop == "fused":
        s.set_apply_tile(17 | gid.FUSED)
    else:
        try:
            s.set_apply_tile(gid.RESIDENT)
        except gid.GidError as e:
            assert e.code == gid.ERR_INVALID_ARG
            pytest.skip("the resident loop does not fit this frame on this device")
    rgb, lab = case.gpu_inputs()
    s.set_frame(rgb, lab)
    pb = case.oracle_problem()
    X = random_state(pb, 5)
    s.set_state(torch.from_numpy(X.astype(np.float32)).cuda())
    delta = s.stage_pcg(10).cpu().numpy()
    ref, rz = pb.pcg_variant(X, 10, single_reduction=True)
    err = np.abs(delta - ref).max()
    assert err <= 1e-4 * np.abs(ref).max(), f"max err {err:.3e} vs {np.abs(ref).max():.3e}"
    np.testing.assert_allclose(s.pcg_history(), rz[:10], rtol=1e-4, atol=1e-4 * rz[0])
    textbook, _ = pb.pcg(X, 10)
    assert np.abs(delta - textbook).max() <= 1e-4 * np.abs(textbook).max()
