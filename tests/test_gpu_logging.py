"""Per-outer-iteration logging (Solver.solve_logged, gid_pcg_history) against
the FP64 oracle and against gid_run itself."""
import json

import numpy as np
import pytest

import oracle as O
from harness import Case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("precond", ["jacobi", "block"])
def test_solve_logged_matches_run_and_the_oracle(tmp_path, precond):
    case = Case(H=48, W=64, K=4, n_cells=12, seed=0)
    N, M = 3, 6
    rgb, lab = case.gpu_inputs()
    s_ref = case.solver()
    s_ref.set_preconditioner(precond)
    s_ref.set_frame(rgb, lab)
    s_ref.init(0)
    s_ref.run(N, M)
    s = case.solver()
    s.set_preconditioner(precond)
    s.set_frame(rgb, lab)
    s.init(0)
    path = tmp_path / "log.jsonl"
    recs = s.solve_logged(N, M, path)
    # the same launches as one gid_run: the same bits
    assert np.array_equal(s.state().cpu().numpy(), s_ref.state().cpu().numpy())
    lines = [json.loads(l) for l in open(path)]
    assert [l["outer"] for l in lines] == [1, 2, 3] and len(recs) == 3
    pb = case.oracle_problem()
    X = pb.init_cold()
    for n in range(N):
        # the oracle's rho history of this outer iteration's Gauss-Newton step
        _, rz = pb.pcg_variant(X, M, block=precond == "block")
        rho = np.array(recs[n]["pcg_rho"])
        assert rho.shape == (M,)
        assert np.abs(rho - rz[:M]).max() <= 1e-4 * rz[0], (n, rho, rz[:M])
        X, _, hist = O.solve_frame(pb, X, 1, M, block=precond == "block")
        assert recs[n]["energy"] == pytest.approx(hist[-1].sum(), rel=1e-4)
        for t, name in enumerate(O.TERMS):
            assert recs[n]["terms"][name] == pytest.approx(hist[-1][t], rel=2e-4, abs=1e-6 * hist[-1].sum())


def test_pcg_history_before_any_step_is_empty():
    case = Case(H=29, W=37, K=3, n_cells=7, seed=1)
    s = case.solver()
    assert s.pcg_history().shape == (0,)
