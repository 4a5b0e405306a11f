"""CUDA path against the FP64 oracle, element by element, through the C ABI.

Stage checks (one kernel each) use the same float32-rounded inputs and state on
both sides.  Their tolerance is derived from the arithmetic: every output is a
sum of at most ~40 FP32 products, so its rounding error is below
40 * 2^-24 * (largest summand) ~ 2.4e-6 of the largest magnitude in the field;
the tests allow 2e-5 of the field's max (an 8x margin).  The end-to-end checks
use the solver's bar: every layer within 1e-3 max-abs after the same N x M
iterations from the same start, energy within 1e-4 relative.
"""
import numpy as np
import pytest

import oracle as O
from harness import Case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = {
    "64x48_K4": dict(H=48, W=64, K=4, n_cells=12),      # the 64 x 48 single-frame workload: 2 x 6 tiles
    "37x29_K3": dict(H=29, W=37, K=3, n_cells=7),       # ragged: partial tiles in x and y
    "70x41_K6": dict(H=41, W=70, K=6, n_cells=9),
}
STAGE_TOL = 2e-5


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def close(gpu, ref, tol=STAGE_TOL, what=""):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    assert gpu.shape == ref.shape, (gpu.shape, ref.shape)
    err = np.abs(gpu - ref).max()
    scale = max(np.abs(ref).max(), 1e-30)
    assert err <= tol * scale, f"{what}: max err {err:.3e} vs scale {scale:.3e} (rel {err / scale:.3e})"


def random_state(case, pb, seed):
    rng = np.random.default_rng(seed)
    X = pb.init_cold()
    X[:3] += rng.normal(0, 0.2, size=X[:3].shape)
    X[3:] += rng.normal(0, 0.05, size=X[3:].shape)
    return f32(X)


@pytest.fixture(params=list(CASES))
def setup(request):
    case = Case(**CASES[request.param], seed=3)
    s = case.solver()
    rgb, lab = case.gpu_inputs()
    s.set_frame(rgb, lab)
    pb = case.oracle_problem()
    return case, s, pb


def test_precompute(setup):
    case, s, pb = setup
    wsr, ws, _ = s.stage_precompute()
    torch.cuda.synchronize()
    close(wsr.cpu().numpy(), pb.wsr, what="w_SR")
    close(ws.cpu().numpy(), pb.omega_s, what="omega spatial")


def test_linearize_apply_energy(setup):
    case, s, pb = setup
    X = random_state(case, pb, 1)
    s.set_state(torch.from_numpy(X.astype(np.float32)).cuda())
    g, d = s.stage_linearize()
    close(g.cpu().numpy(), pb.rhs(X), what="-J^T F")
    close(d.cpu().numpy(), pb.diag(X), what="diag J^T J")
    p = np.random.default_rng(2).normal(size=X.shape).astype(np.float32)
    q = s.stage_apply(torch.from_numpy(p).cuda())
    close(q.cpu().numpy(), pb.apply(X, f32(p)), what="J^T J p")
    tot, per = s.energy()
    E = pb.energy(X)
    for t in range(8):
        assert per[t] == pytest.approx(E[t], rel=2e-5, abs=1e-6 * E.sum()), O.TERMS[t]
    assert tot == pytest.approx(E.sum(), rel=2e-5)


def test_dense_normal_equations(setup):
    case, s, pb = setup
    X = random_state(case, pb, 4)
    X[4:] = np.abs(X[4:])
    s.set_state(torch.from_numpy(X.astype(np.float32)).cuda())
    A, g = s.stage_dense_normal()
    Ao, go = pb.dense_normal(X)
    close(A, Ao, 1e-5, "A")
    close(g, go, 1e-4, "g")


def test_pcg_update(setup):
    """delta after 10 PCG steps from the same state: rounding grows with the
    Krylov recursion, so the bar is 1e-4 of max |delta|."""
    case, s, pb = setup
    X = random_state(case, pb, 5)
    s.set_state(torch.from_numpy(X.astype(np.float32)).cuda())
    delta = s.stage_pcg(10)
    ref, _ = pb.pcg(X, 10)
    close(delta.cpu().numpy(), ref, 1e-4, "PCG delta")


def run_both(case, N, M, t=0):
    s = case.solver()
    rgb, lab = case.gpu_inputs(t)
    s.set_frame(rgb, lab)
    s.init(0)
    s.run(N, M)
    R, T = s.layers()
    tot, per = s.energy()
    b = s.base_colors()
    pb = case.oracle_problem(t)
    Xo, bo, hist = O.solve_frame(pb, pb.init_cold(), N, M)
    return (R.cpu().numpy(), T.cpu().numpy(), b, tot), (np.exp(Xo[:3]), Xo[3:], bo, hist[-1].sum())


@pytest.mark.parametrize("name", ["64x48_K4", "37x29_K3"])
def test_end_to_end_single_frame(name):
    """The 64x48 K=4 workload: 5 Gauss-Newton x 10 PCG, cold start, refinement on."""
    case = Case(**CASES[name], seed=0)
    (R, T, b, E), (Ro, To, bo, Eo) = run_both(case, 5, 10)
    assert np.abs(R - Ro).max() <= 1e-3
    for k in range(case.K + 1):
        assert np.abs(T[k] - To[k]).max() <= 1e-3, k
    assert np.abs(b - bo).max() <= 1e-3
    assert E == pytest.approx(Eo, rel=1e-4)


def test_end_to_end_two_frames_temporal():
    """Frame 0 cold, frame 1 warm with temporal pairs to frame 0 (3 x 8 each)."""
    case = Case(H=48, W=64, K=4, n_cells=12, seed=1, frames=2, temporal=True)
    s = case.solver()
    pb0 = case.oracle_problem(0)
    X0, b0, _ = O.solve_frame(pb0, pb0.init_cold(), 3, 8)
    for t in range(2):
        rgb, lab = case.gpu_inputs(t)
        s.set_frame(rgb, lab)
        s.init(0 if t == 0 else 1)
        s.run(3, 8)
    R, T = s.layers()
    b = s.base_colors()
    E, _ = s.energy()
    pb1 = case.oracle_problem(1, rprev=X0[:3], b=b0)
    X1, b1, hist = O.solve_frame(pb1, X0, 3, 8)
    assert np.abs(R.cpu().numpy() - np.exp(X1[:3])).max() <= 1e-3
    assert np.abs(T.cpu().numpy() - X1[3:]).max() <= 1e-3
    assert np.abs(b - b1).max() <= 1e-3
    assert E == pytest.approx(hist[-1].sum(), rel=1e-4)


def test_host_buffer_entry_point_matches_device_path():
    case = Case(**CASES["37x29_K3"], seed=2)
    s1 = case.solver()
    rgb, lab = case.gpu_inputs()
    s1.set_frame(rgb, lab)
    s1.init(0)
    s1.run(2, 5)
    R1, T1 = s1.layers()
    s2 = case.solver()
    f = case.frames[0]
    R2 = np.zeros((3, case.H, case.W), np.float32)
    T2 = np.zeros((case.K + 1, case.H, case.W), np.float32)
    b2 = np.zeros((case.K, 3), np.float32)
    s2.solve_frame_host(np.ascontiguousarray(f.I, np.float32), np.ascontiguousarray(f.labels, np.uint8), 0, 2, 5,
                        R2, T2, b2)
    assert np.array_equal(R1.cpu().numpy(), R2) and np.array_equal(T1.cpu().numpy(), T2)
    assert np.array_equal(s1.base_colors(), b2)


def test_runs_are_bitwise_reproducible():
    case = Case(**CASES["70x41_K6"], seed=4)
    out = []
    for _ in range(2):
        s = case.solver()
        rgb, lab = case.gpu_inputs()
        s.set_frame(rgb, lab)
        s.init(0)
        s.run(2, 6)
        out.append(s.state().cpu().numpy())
    assert np.array_equal(out[0], out[1])


def test_errors_are_reported():
    from paper_1908_01961_b300 import gid
    case = Case(**CASES["37x29_K3"], seed=2)
    s = case.solver()
    with pytest.raises(gid.GidError) as e:
        s.run(1, 1)
    assert e.value.code == -4
    with pytest.raises(gid.GidError) as e:
        gid.Solver(8, 8, 11)
    assert e.value.code == -1
    rgb, lab = case.gpu_inputs()
    lab[0, 0] = case.K                                    # out-of-range label
    s.set_frame(rgb, lab)
    s.init(0)
    with pytest.raises(gid.GidError) as e:
        s.energy()
    assert e.value.code == -1
    with pytest.raises(gid.GidError):
        s.set_base_colors(np.zeros((case.K, 3)))


def test_graph_replay_matches_direct_launches():
    """gid_run replays a captured CUDA graph; it must give the bits the direct launches give."""
    case = Case(H=48, W=64, K=4, n_cells=12, seed=6, frames=2, temporal=True)
    out = []
    for graphs in (False, True):
        s = case.solver()
        s.set_graphs(graphs)
        for t in range(2):
            rgb, lab = case.gpu_inputs(t)
            s.set_frame(rgb, lab)
            s.init(0 if t == 0 else 1)
            s.run(3, 7)
        out.append((s.state().cpu().numpy(), s.base_colors(), s.launch_count()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2]


@pytest.mark.parametrize("rows", [2, 4, 8, 16, 17])
def test_operator_tile_shapes_agree(rows):
    """Every operator tile shape computes the same J^T J p (up to FP32 rounding order)."""
    case = Case(**CASES["70x41_K6"], seed=3)
    s = case.solver()
    rgb, lab = case.gpu_inputs()
    s.set_frame(rgb, lab)
    pb = case.oracle_problem()
    X = random_state(case, pb, 1)
    s.set_state(torch.from_numpy(X.astype(np.float32)).cuda())
    s.set_apply_tile(rows)
    p = np.random.default_rng(2).normal(size=X.shape).astype(np.float32)
    q = s.stage_apply(torch.from_numpy(p).cuda())
    close(q.cpu().numpy(), pb.apply(X, f32(p)), what=f"J^T J p, {rows} rows")


@pytest.mark.parametrize("name", ["64x48_K4", "70x41_K6"])
def test_persistent_pcg_matches_oracle(name):
    """All PCG steps of a Gauss-Newton step in one cooperative launch (grid
    barriers between the operator and vector phases): same bar as the
    multi-kernel path."""
    case = Case(**CASES[name], seed=0)
    s = case.solver()
    s.set_apply_tile(0)
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


def test_base_color_step_matches_oracle():
    """gid_base_color_step on a set state: b = b_init + Delta b of the oracle's
    SVD solve of the same normal equations."""
    case = Case(**CASES["64x48_K4"], seed=7)
    s = case.solver()
    rgb, lab = case.gpu_inputs()
    s.set_frame(rgb, lab)
    pb = case.oracle_problem()
    X = random_state(case, pb, 8)
    X[4:] = np.abs(X[4:])
    s.set_state(torch.from_numpy(X.astype(np.float32)).cuda())
    s.base_color_step()
    A, g = pb.dense_normal(X)
    assert np.abs(s.base_colors() - (case.b_init + O.dense_solve(A, g))).max() <= 1e-4


@pytest.mark.parametrize("H,W,K,n_cells", [(5, 3, 1, 2), (9, 7, 2, 3), (30, 40, 10, 14)])
def test_end_to_end_edge_shapes(H, W, K, n_cells):
    """Degenerate and extreme cases at the solver's bar: a single base colour
    (K = 1, every indirect layer is zero), frames smaller than one operator tile
    and than the consistency pairs' reach in both directions (most pairs fall
    outside), and the maximum K = 10."""
    case = Case(H=H, W=W, K=K, n_cells=n_cells, seed=2)
    (R, T, b, E), (Ro, To, bo, Eo) = run_both(case, 3, 8)
    assert np.abs(R - Ro).max() <= 1e-3
    assert np.abs(T - To).max() <= 1e-3
    assert np.abs(b - bo).max() <= 1e-3
    assert E == pytest.approx(Eo, rel=1e-4)


def test_pipelined_video_host_entry_matches_frame_by_frame():
    """gid_solve_video_host (uploads and downloads overlapped with the solves)
    gives, frame for frame, the bits of consecutive gid_solve_frame_host calls."""
    case = Case(H=48, W=64, K=4, n_cells=12, seed=8, frames=4, temporal=True)
    F, H, W, K = 4, case.H, case.W, case.K
    rgb = np.ascontiguousarray(np.stack([f.I for f in case.frames]), np.float32)
    lab = np.ascontiguousarray(np.stack([f.labels for f in case.frames]), np.uint8)
    s1 = case.solver()
    R1 = np.zeros((F, 3, H, W), np.float32)
    T1 = np.zeros((F, K + 1, H, W), np.float32)
    b1 = np.zeros((F, K, 3), np.float32)
    for t in range(F):
        s1.solve_frame_host(rgb[t], lab[t], 0 if t == 0 else 1, 2, 6, R1[t], T1[t], b1[t])
    s2 = case.solver()
    R2, T2, b2 = np.zeros_like(R1), np.zeros_like(T1), np.zeros_like(b1)
    s2.solve_video_host(rgb, lab, 0, 2, 6, R2, T2, b2)
    assert np.array_equal(R1, R2) and np.array_equal(T1, T2) and np.array_equal(b1, b2)


def test_recombine_matches_oracle():
    """gid_recombine (Sec. 7.4 editing) on a solved state against the oracle's
    recombination with the GPU's own layers and refined colours: new colours,
    mixed gains (a suppressed layer, an amplified one), a recoloured object and
    out-of-range mask values (treated as 0)."""
    case = Case(**CASES["70x41_K6"], seed=4)
    s = case.solver()
    rgb, lab = case.gpu_inputs()
    s.set_frame(rgb, lab)
    s.init(0)
    s.run(2, 6)
    X = s.state().cpu().numpy().astype(np.float64)
    b = s.base_colors().astype(np.float64)
    rng = np.random.default_rng(3)
    bn = (b * rng.uniform(0.5, 1.5, b.shape)).astype(np.float32)
    g = np.array([1.0, 0.0, 1.0, 0.5, 2.0, 1.0], np.float32)
    mask = np.where(case.frames[0].labels == 2, 3, 0).astype(np.uint8)
    mask[0, :5] = 200
    out = s.recombine(bn, g, torch.from_numpy(mask).cuda())
    ref = O.recombine(X, b, bn.astype(np.float64), g.astype(np.float64), mask)
    close(out.cpu().numpy(), ref, 1e-5, "recombined image")
    same = s.recombine()                                  # b and unit gains: the model's reconstruction
    close(same.cpu().numpy(), O.recombine(X, b, b, np.ones(6), np.zeros_like(mask)), 1e-5, "reconstruction")


def test_recombine_full_size_640x480_K6():
    """The benchmark's editing call at its size: a 640 x 480 K = 6 state, one
    recoloured object, one suppressed layer, against the oracle's recombination."""
    case = Case(H=480, W=640, K=6, n_cells=40, seed=0)
    s = case.solver()
    rgb, lab = case.gpu_inputs()
    s.set_frame(rgb, lab)
    s.init(0)
    s.run(1, 4)
    X = s.state().cpu().numpy().astype(np.float64)
    b = s.base_colors().astype(np.float64)
    bn = b.astype(np.float32).copy()
    bn[0] = bn[0][::-1]
    g = np.ones(6, np.float32)
    g[1] = 0.0
    mask = np.where(case.frames[0].labels == 2, 3, 0).astype(np.uint8)
    out = s.recombine(bn, g, torch.from_numpy(mask).cuda())
    ref = O.recombine(X, b, bn.astype(np.float64), g.astype(np.float64), mask)
    close(out.cpu().numpy(), ref, 1e-5, "recombined image")


@pytest.mark.parametrize("rows", [8, 16, 17])
def test_k8_pcg_delta_each_tile_shape(rows):
    """K = 8 (the 1080p stream's K), 10 PCG steps from a perturbed state with
    the unrolled 8-row, and the rolled 16- and 17-row tiles (128 and 96
    registers): delta within 1e-4 of its max against the oracle; ragged tiles in
    both directions."""
    case = Case(H=57, W=150, K=8, n_cells=10, seed=5)
    s = case.solver()
    s.set_apply_tile(rows)
    rgb, lab = case.gpu_inputs()
    s.set_frame(rgb, lab)
    pb = case.oracle_problem()
    X = random_state(case, pb, 2)
    s.set_state(torch.from_numpy(X.astype(np.float32)).cuda())
    delta = s.stage_pcg(10)
    ref, _ = pb.pcg(X, 10)
    close(delta.cpu().numpy(), ref, tol=1e-4, what=f"PCG delta K=8, {rows} rows")


def test_default_tile_by_frame_size():
    """A new context starts on 128 x 17 tiles where they fit in one wave (at most
    one per SM: 640 x 480 is 145 tiles), else on 128 x 4 tiles (1920 x 1080)."""
    from paper_1908_01961_b300 import gid
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    small = gid.Solver(480, 640, 6, gid.default_weights())
    big = gid.Solver(1080, 1920, 8, gid.default_weights())
    assert small.pcg_layout()[0] == (17 if 5 * 29 <= sms else 4)
    assert big.pcg_layout()[0] == 4
    small.close()
    big.close()
