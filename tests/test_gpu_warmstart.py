"""What the trained warm-start network gains over the method without it, on
held-out 640 x 480, K = 6 frames (seeds the training never saw).

Measured facts this test pins (weights: paper_1908_01961_b300/weights, the
network trained on the plain solver's layers, then fine-tuned on the energy):
  - training works: the trained network's initial state is several times
    closer to the plain solver's result (cold start, 8 Gauss-Newton x 20 PCG)
    than an untrained network's, and about as close as the cold start;
  - its start has a lower exact energy than the cold start (about 4 % lower on
    every one of 50 held-out frames) and is still lower after the first
    Gauss-Newton step (50 of 50);
  - started from it, the same 8 Gauss-Newton steps end within 1% of the cold
    start's final energy (the learned start does not derail the solve).
It does not claim fewer Gauss-Newton steps to the cold start's final energy:
on 50 held-out frames that takes 8 (35 frames) or 9 (15) steps against the cold
start's 8.  The reason is measured by warmstart.sensitivity: even the 8-step
solution itself, blurred by a Gaussian of 1 pixel (the best any predictor of
its smooth part could do), needs 3-4 steps to return to its energy, and a
2-pixel blur 6-9; the steps are spent on pixel-scale detail (mostly the
frame's noise taken into the layers) that the image does not determine
without solving.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def rms(a):
    return float(np.sqrt(np.mean(np.square(a))))


def test_trained_network_start_against_cold_start_and_untrained_network():
    from paper_1908_01961_b300 import gid, warmstart as WS
    net = WS.load_net()
    untrained = gid.Net(WS.K, WS.WIDTHS, seed=123)
    frames = WS.generate([WS.EVAL_SEED0 + 100, WS.EVAL_SEED0 + 101], workers=1)
    s = gid.Solver(WS.H, WS.W, WS.K, WS.solver_weights())
    for I, lab, b in frames:
        rgb, lb = torch.from_numpy(I).cuda(), torch.from_numpy(lab).cuda()
        s.set_base_colors(b)
        s.set_frame(rgb, lb)
        s.init(0)
        X_cold = s.state().cpu().numpy()
        s.run(WS.N_OUTER, WS.M_INNER)
        X_star = s.state().cpu().numpy()
        E_cold, _ = s.energy()
        s.set_base_colors(b)
        s.init_learned(untrained, WS.ZERO_BELOW)
        X_u = s.state().cpu().numpy()
        s.set_base_colors(b)
        s.init(0)
        E_c0, _ = s.energy()
        s.run(1, WS.M_INNER)
        E_c1, _ = s.energy()
        s.set_base_colors(b)
        s.init_learned(net, WS.ZERO_BELOW)
        X_l = s.state().cpu().numpy()
        E_l0, _ = s.energy()
        e_cold, e_l, e_u = rms(X_cold - X_star), rms(X_l - X_star), rms(X_u - X_star)
        print(f"state RMS distance to the plain solution: cold {e_cold:.4f}, learned {e_l:.4f}, untrained {e_u:.4f}")
        assert e_l < 0.25 * e_u
        assert e_l < 1.5 * e_cold
        print(f"energy at the start: cold {E_c0:.5e}, learned {E_l0:.5e}")
        assert E_l0 < E_c0
        s.run(1, WS.M_INNER)
        E_l1, _ = s.energy()
        print(f"energy after one Gauss-Newton step: cold {E_c1:.5e}, learned {E_l1:.5e}")
        assert E_l1 < E_c1
        s.run(WS.N_OUTER - 1, WS.M_INNER)
        E_l, _ = s.energy()
        print(f"final energy: cold start {E_cold:.5e}, learned start {E_l:.5e}")
        assert E_l <= 1.01 * E_cold
