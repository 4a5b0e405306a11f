"""Misclustering correction (Sec. 4.2) and the energy over a region, on the GPU
against the oracle.

The correction solves the frame once per candidate base colour (as one batch)
and picks the candidate with the sparsest indirect layers over the region.  The
per-candidate i-sparsity values must agree with the oracle's own solves within
the solver's bar (every layer within 1e-3, so the region sum within
1e-3 x lambda_is x K x region pixels) and the winner must be the same.  On this
case (seed 0) the criterion recovers the colour the region really has; it does
not on every synthetic case (the decomposition may put the colour error into
the reflectance instead of the indirect layers), which is the method's
property, not this implementation's.
"""
import numpy as np
import pytest

import oracle as O
from harness import Case
from paper_1908_01961_b300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_energy_over_a_region():
    from paper_1908_01961_b300 import gid
    case = Case(H=41, W=70, K=6, n_cells=9, seed=3)
    s = case.solver()
    rgb, lab = case.gpu_inputs()
    s.set_frame(rgb, lab)
    s.init(0)
    s.run(2, 6)
    tot, per = s.energy()
    rng = np.random.default_rng(4)
    m = (rng.uniform(size=(case.H, case.W)) < 0.3).astype(np.uint8)
    mask = torch.from_numpy(m).cuda()
    t1, p1 = s.energy_region(mask)
    t2, p2 = s.energy_region(1 - mask)
    ta, pa = s.energy_region(torch.ones_like(mask))
    assert ta == pytest.approx(tot, rel=1e-12)
    assert np.allclose(p1 + p2, per, rtol=1e-5, atol=1e-9 * tot)
    X = s.state().cpu().numpy().astype(np.float64)
    assert p1[5] == pytest.approx(O.region_isparsity(X, m, s.weights.lambda_isparsity), rel=1e-5)


def test_correction_matches_oracle_and_recovers_the_region_colour():
    from paper_1908_01961_b300 import gid
    H, W, K, seed, N, M = 32, 48, 3, 0, 4, 10
    f = synth.SyntheticVideo(H, W, K, 6, seed=seed).frame(0)
    I = f.I.astype(np.float32)
    b0 = synth.initial_base_colors(f.I, f.labels, K).astype(np.float32)
    true = int(f.labels[H // 2, W // 4])
    region = (f.labels == true)
    region[:, W // 2:] = False
    wrong = np.where(region, (true + 1) % K, f.labels).astype(np.uint8)
    off_s, _ = synth.offsets_for(seed)
    w = gid.default_weights(off_s)
    best, sp, fixed = gid.correct_region(torch.from_numpy(I).cuda(), torch.from_numpy(wrong).cuda(), b0,
                                         torch.from_numpy(region.astype(np.uint8)).cuda(), w, N, M)
    best_o, sp_o = O.correct_region(I.astype(np.float64), wrong, b0.astype(np.float64), region.astype(np.uint8),
                                    off_s, N, M)
    assert best == best_o == true
    assert np.all(np.abs(sp - sp_o) <= 1e-3 * w.lambda_isparsity * K * region.sum())
    fixed = fixed.cpu().numpy()
    assert np.array_equal(fixed[region], np.full(region.sum(), true)) and np.array_equal(fixed[~region], wrong[~region])
