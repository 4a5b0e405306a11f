"""Degenerate frame shapes and the extremes of K against the FP64 oracle (GPU).

A frame of one row (no vertical neighbours, every consistency pair with a
vertical offset outside it), one column, one narrower than a float4 chunk
(three of its four lanes past the right edge), exactly one 128 x 17 tile and
one pixel more in each direction (a second, one-pixel tile column and row),
and K = 1 and K = GID_MAX_K = 10.  Each is solved 3 x 5 from the cold start
with refinement on, with the context's default tile and, where it differs,
the 2- and 17-row tiles; every layer within 1e-3 max-abs, the base colours
within 1e-3 and the energy within 1e-4 relative of the oracle's.
"""
import numpy as np
import pytest

import oracle as O
from harness import Case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHAPES = {
    "3x7_K2": dict(H=3, W=7, K=2, n_cells=2),
    "1x130_K2": dict(H=1, W=130, K=2, n_cells=3),
    "40x1_K2": dict(H=40, W=1, K=2, n_cells=3),
    "17x128_K3": dict(H=17, W=128, K=3, n_cells=5),
    "18x129_K3": dict(H=18, W=129, K=3, n_cells=5),
    "30x40_K1": dict(H=30, W=40, K=1, n_cells=3),
    "30x40_K10": dict(H=30, W=40, K=10, n_cells=14),
}


@pytest.mark.parametrize("rows", [None, 2, 17])
@pytest.mark.parametrize("name", list(SHAPES))
def test_degenerate_shapes_match_oracle(name, rows):
    case = Case(**SHAPES[name], seed=7)
    s = case.solver()
    if rows is not None:
        s.set_apply_tile(rows)
    rgb, lab = case.gpu_inputs()
    s.set_frame(rgb, lab)
    s.init(0)
    s.run(3, 5)
    R, T = s.layers()
    E, _ = s.energy()
    pb = case.oracle_problem()
    Xo, bo, hist = O.solve_frame(pb, pb.init_cold(), 3, 5)
    assert np.abs(R.cpu().numpy() - np.exp(Xo[:3])).max() <= 1e-3
    assert np.abs(T.cpu().numpy() - Xo[3:]).max() <= 1e-3
    assert np.abs(s.base_colors() - bo).max() <= 1e-3
    assert E == pytest.approx(hist[-1].sum(), rel=1e-4)
