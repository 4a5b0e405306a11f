"""The L2 persistence window over the operator coefficients (gid_set_l2_window):
a cache hint only, so the solve's bits do not change; refused where the
coefficient planes do not fit in the device's persisting set-aside (GPU)."""
import numpy as np
import pytest

from harness import Case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def solve(case, window, rows=17):
    s = case.solver()
    s.set_apply_tile(rows)
    if window:
        s.set_l2_window(True)
        assert s.l2_window()
    rgb, lab = case.gpu_inputs()
    s.set_frame(rgb, lab)
    s.init(0)
    s.run(3, 8)
    return s.state().cpu().numpy(), s.base_colors()


@pytest.mark.parametrize("rows", [8, 17])
def test_window_changes_no_bits(rows):
    case = Case(H=117, W=203, K=5, n_cells=15, seed=3)
    X0, b0 = solve(case, False, rows)
    X1, b1 = solve(case, True, rows)
    assert np.array_equal(X0, X1) and np.array_equal(b0, b1)


def test_window_refused_where_the_coefficients_do_not_fit():
    from paper_1908_01961_b300 import gid
    s = gid.Solver(1080, 1920, 8, gid.default_weights())
    with pytest.raises(gid.GidError) as e:
        s.set_l2_window(True)
    assert e.value.code == gid.ERR_INVALID_ARG
    assert not s.l2_window()
    s.close()


def test_autotune_decides_the_window_and_the_solve_is_unchanged():
    case = Case(H=117, W=203, K=5, n_cells=15, seed=4)
    s = case.solver()
    rgb, lab = case.gpu_inputs()
    s.set_frame(rgb, lab)
    s.init(0)
    rows, _ = s.autotune(3)
    assert s.l2_window() in (True, False)
    s.init(0)
    s.run(3, 8)
    X = s.state().cpu().numpy()
    r = Case(H=117, W=203, K=5, n_cells=15, seed=4).solver()
    r.set_apply_tile(rows)
    r.set_frame(rgb, lab)
    r.init(0)
    r.run(3, 8)
    assert np.array_equal(X, r.state().cpu().numpy())
