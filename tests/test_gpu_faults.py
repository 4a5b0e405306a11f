"""Failure detection without a GPU fault: every failure here is made on the
host (a NaN poked into the input frame, a base-colour system made singular by
zero indirect layers with the ridge terms off, grid-barrier participants that
never arrive) and the device side only gives up a bounded wait or records a
status bit.  Each test then checks the reported error and that the context
still solves correctly afterwards."""
import numpy as np
import pytest

import oracle as O
from harness import Case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def clean_solve_matches_oracle(case, s, N=2, M=5):
    rgb, lab = case.gpu_inputs()
    s.new_sequence()
    s.set_base_colors(case.b_init)
    s.set_frame(rgb, lab)
    s.init(0)
    s.run(N, M)
    R, T = s.layers()
    E, _ = s.energy()
    pb = case.oracle_problem()
    Xo, bo, hist = O.solve_frame(pb, pb.init_cold(), N, M)
    assert np.abs(R.cpu().numpy() - np.exp(Xo[:3])).max() <= 1e-3
    assert np.abs(T.cpu().numpy() - Xo[3:]).max() <= 1e-3
    assert E == pytest.approx(hist[-1].sum(), rel=1e-4)


def test_nan_in_the_frame_is_reported_as_numeric():
    from paper_1908_01961_b300 import gid
    case = Case(H=29, W=37, K=3, n_cells=7, seed=4)
    s = case.solver()
    rgb, lab = case.gpu_inputs()
    rgb[1, 7, 11] = float("nan")
    s.set_frame(rgb, lab)
    s.init(0)
    s.run(2, 5)
    with pytest.raises(gid.GidError) as e:
        s.energy()
    assert e.value.code == gid.ERR_NUMERIC
    clean_solve_matches_oracle(case, s)


def test_singular_base_colour_system_is_reported_and_leaves_the_colours():
    """With lambda_IR = lambda_CR = 0 the K x K systems have no ridge; with every
    indirect layer zero they are exactly zero, hence not positive definite."""
    from paper_1908_01961_b300 import gid
    case = Case(H=29, W=37, K=3, n_cells=7, seed=4)
    s = case.solver(lambda_IR=0.0, lambda_CR=0.0)
    rgb, lab = case.gpu_inputs()
    s.set_frame(rgb, lab)
    s.init(0)
    X = s.state()
    X[4:] = 0.0
    s.set_state(X)
    b_before = s.base_colors()
    s.base_color_step()
    with pytest.raises(gid.GidError) as e:
        s.energy()
    assert e.value.code == gid.ERR_NUMERIC
    assert np.array_equal(s.base_colors(), b_before)
    s.energy()  # the status was cleared with the report


def test_grid_barrier_that_never_completes_times_out_and_the_context_recovers():
    """One phantom participant in the persistent kernel's grid barrier: every
    block's wait gives up after 2000 polls, the kernel returns without touching
    the state, GID_ERR_TIMEOUT is reported; with the injection removed the same
    context solves as the oracle does."""
    from paper_1908_01961_b300 import gid
    case = Case(H=48, W=64, K=4, n_cells=12, seed=6)
    s = case.solver()
    try:
        s.set_apply_tile(0)
    except gid.GidError:
        pytest.skip("the persistent PCG kernel cannot be co-scheduled on this device")
    rgb, lab = case.gpu_inputs()
    s.set_frame(rgb, lab)
    s.init(0)
    X0 = s.state().cpu().numpy()
    s.debug_inject(phantom_blocks=1, spin_limit=2000)
    s.run(1, 4)
    with pytest.raises(gid.GidError) as e:
        s.energy()
    assert e.value.code == gid.ERR_TIMEOUT
    assert np.array_equal(s.state().cpu().numpy(), X0)
    s.debug_inject(0, 0)
    clean_solve_matches_oracle(case, s)


def test_run_checked_rolls_the_layers_back():
    """Frame 1 of a video carries a NaN: run_checked raises GID_ERR_NUMERIC and
    restores the warm-start state it began from; frame 1 without the NaN then
    solves from there.  (Temporal pairs off: with them, setting a frame again
    would make the failed frame the previous one.)"""
    from paper_1908_01961_b300 import gid
    case = Case(H=48, W=64, K=4, n_cells=12, seed=1, frames=2, temporal=False)
    s = case.solver()
    rgb, lab = case.gpu_inputs(0)
    s.set_frame(rgb, lab)
    s.init(0)
    s.run_checked(2, 5)
    rgb1, lab1 = case.gpu_inputs(1)
    bad = rgb1.clone()
    bad[0, 20, 30] = float("nan")
    s.set_frame(bad, lab1)
    s.init(1)
    X_start = s.state().cpu().numpy()
    assert np.isfinite(X_start).all()
    with pytest.raises(gid.GidError) as e:
        s.run_checked(2, 5)
    assert e.value.code == gid.ERR_NUMERIC
    assert np.array_equal(s.state().cpu().numpy(), X_start)
    s.set_frame(rgb1, lab1)
    E, _ = s.run_checked(2, 5)
    assert np.isfinite(E)


def test_bad_injection_arguments_are_rejected():
    from paper_1908_01961_b300 import gid
    case = Case(H=29, W=37, K=3, n_cells=7, seed=4)
    s = case.solver()
    with pytest.raises(gid.GidError) as e:
        s.debug_inject(-1, 0)
    assert e.value.code == -1
