"""Pins of the oracle's residual rows, Jacobians and normal-equation products (CPU).

The Jacobian rows are checked against central finite differences of the
residual vector, and the residual vector against the exact energy: with the
IRLS weights taken at the evaluation point and eps -> 0, the reweighted
squared residuals of Sec. 5.3 equal the l1 / l_p / max terms they replace, and
the exact energy is pinned to closed forms in test_oracle_energy.py.
"""
import numpy as np
import pytest

import oracle as O

from test_oracle_energy import make_problem


def fd_jacobian(pb, X, Xw, mask, h=1e-6):
    F0 = pb.residuals(X, Xw, mask)
    n = X.size
    J = np.zeros((len(F0), n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = h
        e = e.reshape(X.shape)
        J[:, j] = (pb.residuals(X + e, Xw, mask) - pb.residuals(X - e, Xw, mask)) / (2 * h)
    return J, F0


def random_state(pb, seed=0):
    rng = np.random.default_rng(seed)
    X = pb.init_cold()
    X[:3] += rng.normal(0, 0.2, size=X[:3].shape)
    X[3:] += rng.normal(0, 0.1, size=X[3:].shape)      # both signs: exercises the non-neg branch
    return X


@pytest.mark.parametrize("term", list(range(8)) + ["all"])
def test_jacobian_products_match_finite_differences(term):
    H, W, K = 5, 6, 2
    offs_t = np.array([[0, 0], [1, -1]], np.int32)
    rng = np.random.default_rng(11)
    pb = make_problem(H, W, K, seed=2, off_s=((1, 2), (-1, 1)))
    pb = O.Problem(pb.I, pb.labels, pb.b_init, pb.wsr, pb.omega_s, pb.off_s,
                   omega_t=rng.uniform(0, 1, (2, H, W)), off_t=offs_t, rprev=rng.normal(-0.5, 0.3, (3, H, W)),
                   b=pb.b_init + 0.05)
    mask = O.ALL if term == "all" else (1 << term)
    X = random_state(pb, 1)
    Xw = random_state(pb, 2)
    J, F = fd_jacobian(pb, X, Xw, mask)
    p = np.random.default_rng(3).normal(size=X.shape)
    scale = np.abs(J).max() ** 2 * 10 + 1e-300
    np.testing.assert_allclose(pb.apply(X, p, Xw, mask).ravel(), J.T @ (J @ p.ravel()), rtol=0, atol=1e-6 * scale)
    np.testing.assert_allclose(pb.rhs(X, Xw, mask).ravel(), -J.T @ F, rtol=0,
                               atol=1e-6 * (np.abs(J).max() * np.abs(F).max() * 10 + 1e-300))
    np.testing.assert_allclose(pb.diag(X, Xw, mask).ravel(), (J ** 2).sum(0), rtol=0, atol=1e-6 * scale)


@pytest.mark.parametrize("p", [1.0, 0.5])
def test_surrogate_equals_exact_energy_at_its_own_weights(p):
    """|F_t|^2 with weights from X itself and eps -> 0 equals the exact E_t."""
    pb = make_problem(6, 5, 3, seed=4, eps=1e-14, p=p)
    X = random_state(pb, 5)
    np.testing.assert_allclose(pb.surrogate(X), pb.energy(X), rtol=1e-9, atol=0)


def test_surrogate_quadratic_terms_independent_of_eps():
    pb = make_problem(6, 5, 3, seed=4)
    X = random_state(pb, 6)
    S, E = pb.surrogate(X), pb.energy(X)
    for t in (0, 1, 3, 4):                                  # data, clustering, consistency, monochrome
        assert S[t] == pytest.approx(E[t], rel=1e-12)


def test_normal_matrix_symmetric():
    pb = make_problem(7, 6, 3, seed=8)
    X = random_state(pb, 9)
    rng = np.random.default_rng(1)
    u, v = rng.normal(size=X.shape), rng.normal(size=X.shape)
    assert np.vdot(u, pb.apply(X, v)) == pytest.approx(np.vdot(v, pb.apply(X, u)), rel=1e-12)


def test_consistency_residual_zero_for_constant_r():
    pb = make_problem(6, 6, 2, seed=3)
    X = random_state(pb, 1)
    X[:3] = 0.42
    F = pb.residuals(X, mask=1 << 3)
    assert len(F) > 0 and np.all(F == 0)
