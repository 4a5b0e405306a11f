"""The 1920 x 1080, K = 8 stream size (80 Voronoi cells, temporal pairs) against
the FP64 oracle.

The GPU solves frame 0 (cold start, 8 Gauss-Newton x 20 PCG, autotuned tile,
graph replay) and takes frame 1 with a warm start and temporal pairs.  At the
GPU's own warm-start state (cast to FP64, so the oracle need not replay frame 0)
every stage is compared over the whole frame: the linearisation (-J^T F and
diag), the operator on a random vector, the eight energy terms and the
base-colour normal equations; then one full outer iteration (Gauss-Newton step
of 20 PCG steps and the base-colour step) from that state.  Bars as in the
other parity tests: stages at 2e-5 of the field's max (1e-5 / 1e-4 for the
normal equations), layers within 1e-3 max-abs, energy within 1e-4 relative.
Several minutes of single-core oracle time.
"""
import numpy as np
import pytest

import oracle as O
from harness import Case
from paper_1908_01961_b300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")


def close(gpu, ref, tol, what):
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    err = np.abs(gpu - ref).max()
    scale = max(np.abs(ref).max(), 1e-30)
    assert err <= tol * scale, f"{what}: max err {err:.3e} vs scale {scale:.3e}"


def test_stream_1920x1080_K8_stages_and_one_outer_iteration():
    cfg = synth.STREAM_1080P
    N, M = cfg["N"], cfg["M"]
    case = Case(cfg["H"], cfg["W"], cfg["K"], cfg["n_cells"], seed=5, frames=2, temporal=True)
    s = case.solver()
    rgb, lab = case.gpu_inputs(0)
    s.set_frame(rgb, lab)
    s.init(0)
    s.autotune(5)
    s.init(0)
    s.run(N, M)
    X0 = s.state().cpu().numpy().astype(np.float64)
    b0 = s.base_colors().astype(np.float64)
    rgb, lab = case.gpu_inputs(1)
    s.set_frame(rgb, lab)
    s.init(1)
    pb = case.oracle_problem(1, rprev=X0[:3], b=b0)

    g, d = s.stage_linearize()
    close(g.cpu().numpy(), pb.rhs(X0), 2e-5, "-J^T F")
    close(d.cpu().numpy(), pb.diag(X0), 2e-5, "diag J^T J")
    p = np.random.default_rng(1).normal(size=X0.shape).astype(np.float32)
    q = s.stage_apply(torch.from_numpy(p).cuda())
    close(q.cpu().numpy(), pb.apply(X0, p.astype(np.float64)), 2e-5, "J^T J p")
    tot, per = s.energy()
    E = pb.energy(X0)
    for t in range(8):
        assert per[t] == pytest.approx(E[t], rel=2e-5, abs=1e-6 * E.sum()), O.TERMS[t]
    A, gb = s.stage_dense_normal()
    Ao, go = pb.dense_normal(X0)
    close(A, Ao, 1e-5, "A")
    close(gb, go, 1e-4, "g")

    s.run(1, M)
    R1, T1 = s.layers()
    E1, _ = s.energy()
    X1, b1, hist = O.solve_frame(pb, X0, 1, M)
    assert np.abs(R1.cpu().numpy() - np.exp(X1[:3])).max() <= 1e-3
    assert np.abs(T1.cpu().numpy() - X1[3:]).max() <= 1e-3
    assert np.abs(s.base_colors() - b1).max() <= 1e-3
    assert E1 == pytest.approx(hist[-1].sum(), rel=1e-4)


def test_1920x1080_K10_stages_and_one_outer_iteration():
    """The largest frame of the workloads with the largest K (GID_MAX_K = 10: 14
    unknowns and 49 coefficient planes per pixel), no temporal pairs: every stage
    at the GPU's cold-start state, then one outer iteration from it, at the same
    bars as above."""
    cfg = synth.STREAM_1080P
    M = cfg["M"]
    case = Case(cfg["H"], cfg["W"], 10, cfg["n_cells"], seed=6)
    s = case.solver()
    rgb, lab = case.gpu_inputs(0)
    s.set_frame(rgb, lab)
    s.init(0)
    X0 = s.state().cpu().numpy().astype(np.float64)
    pb = case.oracle_problem(0)
    g, d = s.stage_linearize()
    close(g.cpu().numpy(), pb.rhs(X0), 2e-5, "-J^T F")
    close(d.cpu().numpy(), pb.diag(X0), 2e-5, "diag J^T J")
    p = np.random.default_rng(2).normal(size=X0.shape).astype(np.float32)
    q = s.stage_apply(torch.from_numpy(p).cuda())
    close(q.cpu().numpy(), pb.apply(X0, p.astype(np.float64)), 2e-5, "J^T J p")
    A, gb = s.stage_dense_normal()
    Ao, go = pb.dense_normal(X0)
    close(A, Ao, 1e-5, "A")
    close(gb, go, 1e-4, "g")
    s.run(1, M)
    R1, T1 = s.layers()
    E1, _ = s.energy()
    X1, b1, hist = O.solve_frame(pb, X0, 1, M)
    assert np.abs(R1.cpu().numpy() - np.exp(X1[:3])).max() <= 1e-3
    assert np.abs(T1.cpu().numpy() - X1[3:]).max() <= 1e-3
    assert np.abs(s.base_colors() - b1).max() <= 1e-3
    assert E1 == pytest.approx(hist[-1].sum(), rel=1e-4)
