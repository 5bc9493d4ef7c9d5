"""The multi-core C pieces of the oracle (``oracle/sgo.c`` through
``oracle/par.py``) pinned on CPU: the operator apply against the oracle's
Kronecker form and against properties the Galerkin operator must have (the
sigma = 0 limit, symmetry), the banded substitutions against a sparse direct
solve, and the GMRES solve against the direct solution and a manufactured
one."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import galerkin, par


@pytest.fixture(scope="module")
def small():
    prob = galerkin.build(20, 2, 3, 6, sigma2=0.3, bx=0.5, by=0.5)
    return prob, par.Operator(prob).factor_mean()


def test_apply_matches_kronecker_form(small):
    prob, op = small
    X = np.random.default_rng(1).standard_normal((prob.n, prob.P))
    Y = galerkin.from_vec(op.apply(galerkin.to_vec(X)), prob.n, prob.P)
    Yr = galerkin.apply(prob, X)
    assert np.max(np.abs(Y - Yr)) <= 1e-13 * np.max(np.abs(Yr))


def test_apply_is_symmetric(small):
    prob, op = small
    rng = np.random.default_rng(2)
    x1, x2 = rng.standard_normal(prob.n * prob.P), rng.standard_normal(prob.n * prob.P)
    a = x2 @ op.apply(x1)
    b = op.apply(x2) @ x1
    assert abs(a - b) <= 1e-13 * np.linalg.norm(op.apply(x1)) * np.linalg.norm(x2)


def test_sigma_zero_limit_is_block_diagonal():
    """With sigma = 0 the operator is I kron A_0: every mode column is
    multiplied by the deterministic stiffness matrix alone."""
    prob = galerkin.build(12, 2, 2, 4, sigma2=0.0)
    op = par.Operator(prob)
    X = np.random.default_rng(3).standard_normal((prob.n, prob.P))
    Y = galerkin.from_vec(op.apply(galerkin.to_vec(X)), prob.n, prob.P)
    assert np.max(np.abs(Y - prob.A(0) @ X)) <= 1e-13 * np.max(np.abs(Y))


def test_band_substitutions_match_sparse_direct(small):
    prob, op = small
    B = np.random.default_rng(4).standard_normal((prob.n, prob.P))
    Z = galerkin.from_vec(op.precond(galerkin.to_vec(B)), prob.n, prob.P)
    Zr = spla.spsolve(prob.A(0).tocsc(), B)
    assert np.max(np.abs(Z - Zr)) <= 1e-12 * np.max(np.abs(Zr))
    # in place, as GMRES may call it
    v = galerkin.to_vec(B).copy()
    op.precond(v, v)
    assert np.array_equal(v, galerkin.to_vec(Z))


def test_solve_matches_direct_and_manufactured(small):
    prob, op = small
    X, its, hist, _ = par.solve(prob, tol=1e-12, op=op)
    Xd = galerkin.solve_direct(prob)
    assert galerkin.relres(prob, X) <= 1e-12
    assert np.linalg.norm(X - Xd) <= 1e-10 * np.linalg.norm(Xd)
    assert 0 < its < 100 and hist[-1] <= 1e-12
    Xt = np.random.default_rng(1234).standard_normal((prob.n, prob.P))
    F = galerkin.apply(prob, Xt)
    Xm, _, _, _ = par.solve(prob, F=F, tol=1e-13, op=op)
    assert np.linalg.norm(Xm - Xt) <= 1e-10 * np.linalg.norm(Xt)


def test_gmres_agrees_with_numpy_gmres(small):
    """The same algorithm as galerkin.gmres: the same iteration count and
    residual history (the vector sums differ only in rounding order)."""
    prob, op = small
    _, its, hist, _ = par.solve(prob, tol=1e-10, restart=20, op=op)
    _, its_r, hist_r = galerkin.solve_gmres(prob, tol=1e-10, restart=20)
    assert its == its_r
    np.testing.assert_allclose(hist, hist_r, rtol=1e-6)
