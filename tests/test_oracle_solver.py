"""Pins of the oracle's Gauss-Newton / PCG / base-colour steps (CPU only).

* PCG against a dense direct solve of the materialised normal equations;
* PCG iterate m against the Krylov-space minimiser computed densely, and the
  monotone decrease of the quadratic model (conjugate-gradient properties);
* the Gauss-Newton step against a least-squares solve of the finite-difference
  linearisation (eq:optimization);
* the dense step: exact recovery of the base colours on a noise-free frame
  (the data term is linear in Delta b), and the ridge solution against an
  explicit tall least-squares system;
* the IRLS fixed point of a one-pixel problem against the closed-form
  soft-threshold solution;
* the energy history of the 64x48 workload.
"""
import numpy as np
import pytest

import oracle as O
from paper_1908_01961_b300 import synth

from test_oracle_energy import make_problem
from test_oracle_jacobian import fd_jacobian, random_state


def normal_matrix(pb, X):
    n = X.size
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = pb.apply(X, e.reshape(X.shape)).ravel()
    return A


@pytest.fixture(scope="module")
def small():
    pb = make_problem(8, 8, 4, seed=21)
    X = random_state(pb, 22)
    return pb, X, normal_matrix(pb, X), pb.rhs(X).ravel(), pb.diag(X).ravel()


def test_pcg_converges_to_direct_solve(small):
    pb, X, A, g, d = small
    direct = np.linalg.solve(A, g)
    delta, rz = pb.pcg(X, 3000)
    assert rz[-1] < 1e-20 * rz[0]
    np.testing.assert_allclose(delta.ravel(), direct, rtol=0, atol=1e-9 * np.abs(direct).max())


@pytest.mark.parametrize("M", [1, 2, 5])
def test_pcg_iterate_is_krylov_minimiser(small, M):
    """delta_M minimises the A-norm error over x0 + span{z0, (D^-1 A) z0, ...}."""
    pb, X, A, g, d = small
    Dinv = 1.0 / d
    basis = [Dinv * g]
    for _ in range(M - 1):
        basis.append(Dinv * (A @ basis[-1]))
    B = np.stack(basis, axis=1)
    Q, _ = np.linalg.qr(B)
    y = np.linalg.solve(Q.T @ A @ Q, Q.T @ g)
    expect = Q @ y
    delta, _ = pb.pcg(X, M)
    np.testing.assert_allclose(delta.ravel(), expect, rtol=0, atol=1e-8 * np.abs(expect).max())


def test_pcg_quadratic_model_decreases(small):
    pb, X, A, g, d = small
    q = []
    for M in range(0, 12):
        delta = pb.pcg(X, M)[0].ravel()
        q.append(0.5 * delta @ A @ delta - g @ delta)
    assert all(b < a for a, b in zip(q, q[1:]))


def test_gauss_newton_step_is_linearised_least_squares():
    pb = make_problem(5, 4, 2, seed=13)
    X = random_state(pb, 14)
    J, F = fd_jacobian(pb, X, X, O.ALL)
    expect = np.linalg.lstsq(J, -F, rcond=None)[0]
    X1 = pb.gn_step(X, 2000)
    np.testing.assert_allclose((X1 - X).ravel(), expect, rtol=0, atol=1e-7 * np.abs(expect).max())


def test_dense_step_recovers_base_colours_noise_free():
    v = synth.SyntheticVideo(48, 64, 4, 12, seed=0, noise=0.0)
    f = v.frame(0, noise=False)
    X = np.concatenate([np.log(f.R), f.T])
    b_init = f.b + 0.05 * np.sign(np.random.default_rng(1).normal(size=f.b.shape))
    C, wsr, om, _ = O.precompute(f.I, np.array([[1, 1]]))
    pb = O.Problem(f.I, f.labels, b_init, wsr, om, np.array([[1, 1]]), lambda_IR=0.0, lambda_CR=0.0)
    A, g = pb.dense_normal(X)
    np.testing.assert_allclose(b_init + O.dense_solve(A, g), f.b, rtol=0, atol=1e-10)


def test_dense_step_with_ridge_matches_tall_least_squares():
    pb = make_problem(6, 7, 3, seed=31)
    X = random_state(pb, 32)
    X[4:] = np.abs(X[4:])
    A, g = pb.dense_normal(X)
    db = O.dense_solve(A, g)
    P = pb.H * pb.W
    R = np.exp(X[:3]).reshape(3, P)
    T = X[3:].reshape(pb.K + 1, P)
    for c in range(3):
        e = pb.I[c].ravel() - R[c] * (T[0] + pb.b_init[:, c] @ T[1:])
        D = np.sqrt(5000) * (R[c][:, None] * T[1:].T)
        tall = np.vstack([D, np.sqrt(110.0) * np.eye(pb.K)])
        rhs = np.concatenate([np.sqrt(5000) * e, np.zeros(pb.K)])
        np.testing.assert_allclose(db[:, c], np.linalg.lstsq(tall, rhs, rcond=None)[0], rtol=1e-10, atol=1e-13)


def test_irls_one_pixel_fixed_point_is_soft_threshold():
    """One pixel, data + i-sparsity only (r pinned by a stiff clustering prior).
    The literal reweighting (no 1/2 factor) converges to the minimiser of
    l_data |I - R(T_0 + b_1 T_1)|^2 + 2 l_is |T_1|, a soft threshold."""
    Rc = np.array([0.5, 0.4, 0.3])
    b1 = np.array([0.9, 0.2, 0.1])
    I = (Rc * (0.8 + b1 * 0.05) + np.array([0.002, -0.001, 0.001]))[:, None, None]
    lam = dict(lambda_clustering=1e9, lambda_rsparsity=0.0, lambda_rconsistency=0.0, lambda_monochrome=0.0,
               lambda_smoothness=0.0, lambda_nonneg=0.0, lambda_isparsity=0.02, eps=1e-9)
    pb = O.Problem(I, np.zeros((1, 1), np.uint8), Rc[None, :], np.zeros((1, 1)), np.zeros((0, 1, 1)),
                   np.zeros((0, 2)), b=b1[None, :], **lam)
    X = pb.init_cold()
    X[4] = 0.03
    for _ in range(60):
        X = pb.gn_step(X, 50)
    a, u = Rc, Rc * b1
    Pp = np.eye(3) - np.outer(a, a) / (a @ a)
    y, v = Pp @ I[:, 0, 0], Pp @ u
    t_ls = (v @ y) / (v @ v)
    thr = 2 * lam["lambda_isparsity"] / (2 * 5000 * (v @ v))
    t_star = np.sign(t_ls) * max(abs(t_ls) - thr, 0.0)
    assert 0 < t_star < t_ls                                       # the threshold is active
    assert X[4, 0, 0] == pytest.approx(t_star, rel=1e-4)
    t0 = a @ (I[:, 0, 0] - u * t_star) / (a @ a)
    assert X[3, 0, 0] == pytest.approx(t0, rel=1e-6)


def test_energy_history_64x48():
    """The decomposition + refinement on the 64x48 K=4 frame (5 x 10): the total
    energy is non-increasing across outer iterations with the default readings."""
    cfg = synth.SINGLE_64x48
    v = synth.SyntheticVideo(cfg["H"], cfg["W"], cfg["K"], cfg["n_cells"], seed=0)
    f = v.frame(0)
    off_s, _ = synth.offsets_for(0)
    C, wsr, om, _ = O.precompute(f.I, off_s)
    pb = O.Problem(f.I, f.labels, synth.initial_base_colors(f.I, f.labels, cfg["K"]), wsr, om, off_s)
    X, b, hist = O.solve_frame(pb, pb.init_cold(), cfg["N"], cfg["M"])
    tot = hist.sum(axis=1)
    assert np.all(np.isfinite(hist)) and np.all(np.isfinite(X)) and np.all(np.isfinite(b))
    assert np.all(np.diff(tot) <= 1e-9 * tot[0]), tot
