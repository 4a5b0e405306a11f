"""Pins of the oracle's preconditioner and PCG variants (Sec. 6.1 leaves the
preconditioner unnamed; the solver offers Jacobi and per-pixel block-Jacobi, and
the oracle also carries the single-reduction CG recurrence).

Each pin reaches the result by a route that shares no arithmetic with the
variant under test: the per-pixel blocks are read off the operator itself by
probing it with unit vectors, the first block-Jacobi iterate is formed in numpy
from those probed blocks, the converged iterates are compared with a dense
solve of the probed normal matrix, and the two recurrences are compared with
each other.
"""
import numpy as np
import pytest

import oracle as O
from harness import Case


def tiny(**w):
    case = Case(H=5, W=6, K=2, n_cells=3, seed=2)
    pb = case.oracle_problem(**w)
    rng = np.random.default_rng(4)
    X = pb.init_cold()
    X[:3] += rng.normal(0, 0.2, size=X[:3].shape)
    X[3:] += rng.normal(0, 0.05, size=X[3:].shape)
    return pb, X


def dense_operator(pb, X):
    """J^T J as a dense (n, n) matrix, column j = the operator applied to e_j."""
    V, H, W = pb.shape
    n = V * H * W
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = pb.apply(X, e.reshape(V, H, W)).ravel()
    return A


def probed_blocks(A, V, H, W):
    P = H * W
    B = np.zeros((H, W, V, V))
    for y in range(H):
        for x in range(W):
            ids = [v * P + y * W + x for v in range(V)]
            B[y, x] = A[np.ix_(ids, ids)]
    return B


def test_block_diag_equals_the_operators_diagonal_blocks():
    pb, X = tiny()
    V, H, W = pb.shape
    A = dense_operator(pb, X)
    assert np.abs(A - A.T).max() <= 1e-9 * np.abs(A).max()
    B = pb.block_diag(X)
    Bp = probed_blocks(A, V, H, W)
    assert np.abs(B - Bp).max() <= 1e-10 * np.abs(Bp).max()
    # the data and monochrome terms couple the unknowns of a pixel: the blocks are not diagonal
    dg = np.diagonal(B, axis1=2, axis2=3)
    corr = B / np.sqrt(dg[..., :, None] * dg[..., None, :]) - np.eye(V)
    assert np.abs(corr).max() > 0.3
    # their diagonal is the Jacobi preconditioner's
    d = pb.diag(X)
    assert np.abs(np.diagonal(B, axis1=2, axis2=3).transpose(2, 0, 1) - d).max() <= 1e-12 * np.abs(d).max()


def test_first_block_jacobi_iterate_from_the_probed_blocks():
    """delta_1 = alpha z_0, z_0 = B^-1 g solved pixel by pixel, alpha = <g, z_0> / <z_0, A z_0>."""
    pb, X = tiny()
    V, H, W = pb.shape
    A = dense_operator(pb, X)
    Bp = probed_blocks(A, V, H, W)
    g = pb.rhs(X)
    z = np.zeros_like(g)
    for y in range(H):
        for x in range(W):
            z[:, y, x] = np.linalg.solve(Bp[y, x], g[:, y, x])
    alpha = (g * z).sum() / (z.ravel() @ A @ z.ravel())
    d1, rz = pb.pcg_variant(X, 1, block=True)
    assert np.abs(d1 - alpha * z).max() <= 1e-10 * np.abs(alpha * z).max()
    assert rz[0] == pytest.approx((g * z).sum(), rel=1e-12)


@pytest.mark.parametrize("block", [False, True])
@pytest.mark.parametrize("single_reduction", [False, True])
def test_pcg_variants_reach_the_dense_solution(block, single_reduction):
    """Run long enough, every variant solves J^T J delta = -J^T F (checked against numpy's dense solve)."""
    pb, X = tiny()
    A = dense_operator(pb, X)
    g = pb.rhs(X).ravel()
    ref = np.linalg.solve(A, g)
    d, _ = pb.pcg_variant(X, 600, block=block, single_reduction=single_reduction)
    assert np.abs(d.ravel() - ref).max() <= 1e-7 * np.abs(ref).max()


@pytest.mark.parametrize("block", [False, True])
def test_single_reduction_recurrence_matches_the_textbook_one(block):
    """Same iterates in exact arithmetic; in FP64 after 20 steps they agree to ~1e-12."""
    case = Case(H=24, W=32, K=4, n_cells=6, seed=1)
    pb = case.oracle_problem()
    X = pb.init_cold()
    d1, r1 = pb.pcg_variant(X, 20, block=block)
    d2, r2 = pb.pcg_variant(X, 20, block=block, single_reduction=True)
    assert np.abs(d1 - d2).max() <= 1e-9 * np.abs(d1).max()
    assert np.abs(r1 - r2).max() <= 1e-9 * r1[0]


def test_textbook_jacobi_variant_is_the_pinned_pcg():
    pb, X = tiny()
    d0, r0 = pb.pcg(X, 12)
    d1, r1 = pb.pcg_variant(X, 12)
    assert np.array_equal(d0, d1) and np.array_equal(r0, r1)


def test_block_jacobi_reduces_to_jacobi_without_coupling_terms():
    """With the data and monochrome terms off, every block is diagonal."""
    pb, X = tiny(lambda_data=0.0, lambda_monochrome=0.0)
    B = pb.block_diag(X)
    V = B.shape[-1]
    assert np.abs(B * (1 - np.eye(V))).max() == 0.0
    d0, _ = pb.pcg(X, 12)
    d1, _ = pb.pcg_variant(X, 12, block=True)
    assert np.abs(d0 - d1).max() <= 1e-12 * np.abs(d0).max()


def test_block_jacobi_lowers_the_quadratic_model_at_least_as_fast():
    """At equal step counts the block-Jacobi iterate reaches a quadratic-model
    value m(d) = -g.d + d.A d / 2 no worse than Jacobi's on this frame (the
    measured effect is modest; spatial coupling dominates the conditioning)."""
    case = Case(H=24, W=32, K=4, n_cells=6, seed=1)
    pb = case.oracle_problem()
    X = pb.init_cold()
    g = pb.rhs(X)

    def model(d):
        return -(g * d).sum() + 0.5 * (d * pb.apply(X, d)).sum()

    for M in (5, 10):
        mj = model(pb.pcg_variant(X, M)[0])
        mb = model(pb.pcg_variant(X, M, block=True)[0])
        assert mb <= mj + 1e-9 * abs(mj)
