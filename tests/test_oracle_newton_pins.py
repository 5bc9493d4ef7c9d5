"""Pins of the Newton oracle of the quadratic-conductivity problem
(Sec. 2.2, Eqs. NLP_StrongPDE, stonlp_system, AjkTkl with (1 + u^2)) against
facts that do not come from its own formulas: the linear operator at U = 0,
Gauss-Hermite quadrature of the element Galerkin matrix, central differences
of the residual for the Jacobian, the deterministic problem at sigma = 0
(solved by a fixed-point iteration), quadratic convergence, stochastic
collocation for one random variable, and the Kirchhoff transform."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
from numpy.polynomial import hermite_e as H

from oracle import fem, galerkin, newton, nonlinear, pce

pytestmark = pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")


def psi(alpha, xs):
    out = np.ones(len(xs))
    for d, a in enumerate(alpha):
        c = np.zeros(int(a) + 1)
        c[-1] = 1.0
        out *= H.hermeval(xs[:, d], c) / np.sqrt(float(pce.alpha_factorial([a])))
    return out


@pytest.fixture(scope="module")
def small():
    prob = galerkin.build(8, 2, 2, 4, sigma2=0.5, bx=0.4, by=0.4)
    return prob, newton.Problem(prob)


def test_operator_at_zero_is_the_linear_operator(small):
    prob, nl = small
    M0 = nl.operator(np.zeros((prob.n, prob.P)))
    ref = galerkin.assembled(prob)
    assert abs(M0 - ref).max() <= 1e-14 * abs(ref).max()


def test_element_matrix_against_quadrature(small):
    """B_e[l, m] = E[k_e(xi) (1 + w_e(xi)) psi_l psi_m] with k_e the
    truncated input chaos and w_e = Pi_p[ubar_e^2], w_{e,f} = E[ubar_e^2 psi_f],
    by a tensor Gauss-Hermite rule exact for these polynomial degrees."""
    prob, nl = small
    U = 0.6 * np.random.default_rng(1).standard_normal((prob.n, prob.P))
    B = nl.element_matrices(U)
    ub = nl.ubar(U)
    x, w = H.hermegauss(14)
    w = w / np.sqrt(2.0 * np.pi)
    X1, X2 = np.meshgrid(x, x, indexing="ij")
    pts = np.stack([X1.ravel(), X2.ravel()], axis=1)
    wts = np.outer(w, w).ravel()
    vin = np.array([psi(a, pts) for a in pce.multi_indices(prob.L, prob.q)])
    vout = np.array([psi(a, pts) for a in pce.multi_indices(prob.L, prob.p)])
    for e in (0, 7, 33, 90):
        u_e = ub[e] @ vout                                  # ubar_e(xi)
        w_e = np.array([np.sum(wts * u_e * u_e * vout[f]) for f in range(prob.P)])
        k_e = prob.cbar[:, e] @ vin
        cond = k_e * (1.0 + w_e @ vout)
        ref = np.einsum("m,m,lm,km->lk", wts, cond, vout, vout)
        assert np.max(np.abs(B[e] - ref)) <= 1e-12 * np.max(np.abs(ref)), e


def test_jacobian_against_central_differences(small):
    """J(U) dU = -(R(U + h dU) - R(U - h dU)) / (2h) + O(h^2): a dropped
    factor (the 2 of the square, the 1/3 of the average) or a transposed
    index fails."""
    prob, nl = small
    rng = np.random.default_rng(2)
    U = 0.5 * rng.standard_normal((prob.n, prob.P))
    d = rng.standard_normal((prob.n, prob.P))
    J = nl.jacobian(U)
    Jd = J @ galerkin.to_vec(d)
    h = 1e-5
    fd = -(galerkin.to_vec(nl.residual(U + h * d)) - galerkin.to_vec(nl.residual(U - h * d))) / (2 * h)
    assert np.linalg.norm(Jd - fd) <= 1e-8 * np.linalg.norm(fd)
    # the derivative part alone is not negligible here
    Dd = nl.derivative(U) @ galerkin.to_vec(d)
    assert np.linalg.norm(Dd) > 1e-2 * np.linalg.norm(Jd)


def test_sigma_zero_is_the_deterministic_problem():
    prob = galerkin.build(12, 2, 2, 4, sigma2=0.0)
    nl = newton.Problem(prob)
    U, its, hist = newton.newton(nl, tol=1e-12)
    assert hist[-1] <= 1e-12
    u, _ = newton.deterministic_fixed_point(12, np.ones(2 * 12 * 12))
    assert np.max(np.abs(U[:, 0] - u)) <= 1e-12 * np.max(np.abs(u))
    assert np.max(np.abs(U[:, 1:])) <= 1e-14 * np.max(np.abs(u))


def test_newton_converges_quadratically():
    """With a right-hand side that makes u of order one, the relative
    updates fall quadratically once close: e_{k+1} <= C e_k^2."""
    prob = galerkin.build(8, 2, 2, 4, sigma2=0.3, bx=0.5, by=0.5)
    nl = newton.Problem(prob)
    F = 40.0 * prob.rhs()
    U, its, hist = newton.newton(nl, tol=1e-13, F=F)
    assert hist[-1] <= 1e-13 and its <= 12
    assert np.max(np.abs(U[:, 0])) > 0.5
    tail = [h for h in hist if h < 1e-2]
    assert len(tail) >= 2
    for a, b in zip(tail, tail[1:]):
        assert b <= 50.0 * a * a + 1e-15


def test_one_random_variable_against_collocation():
    """L = 1: the SG mean and variance approach those of the exact
    lognormal problem (deterministic solves at 24 Gauss-Hermite nodes) as
    the output order p grows (q = 2p)."""
    N, s2, b = 8, 0.5, 0.5
    errs = []
    for p in (1, 2, 3, 4):
        prob = galerkin.build(N, 1, p, 2 * p, sigma2=s2, bx=b, by=b)
        U, _, _ = newton.newton(newton.Problem(prob), tol=1e-13)
        if p == 1:
            g = prob.gfield[0]
            x, w = H.hermegauss(24)
            w = w / np.sqrt(2.0 * np.pi)
            sols = np.array([newton.deterministic_fixed_point(N, np.exp(g * xi))[0] for xi in x])
            mean = w @ sols
            var = w @ (sols - mean) ** 2
        errs.append((np.max(np.abs(U[:, 0] - mean)) / np.max(np.abs(mean)),
                     np.max(np.abs(np.sum(U[:, 1:] ** 2, axis=1) - var)) / np.max(var)))
    for (m1, v1), (m2, v2) in zip(errs, errs[1:]):
        assert m2 < m1 and v2 < v1
    assert errs[-1][0] < 1e-4 and errs[-1][1] < 1e-2


def test_kirchhoff_transform():
    """k = 1: v = u + u^3/3 solves -lap v = 1, so the discrete solution
    approaches the inverse transform of the P1 Poisson solution at second
    order in h (both are O(h^2) accurate at the nodes)."""
    errs = []
    for N in (8, 16, 32):
        prob = galerkin.build(N, 1, 1, 2, sigma2=0.0)
        U, _, _ = newton.newton(newton.Problem(prob), tol=1e-13, F=30.0 * prob.rhs())
        v = 30.0 * spla.spsolve(prob.A(0).tocsc(), prob.b)
        u = v.copy()
        for _ in range(60):                     # Newton on u + u^3/3 = v, nodewise
            u = u - (u + u ** 3 / 3.0 - v) / (1.0 + u * u)
        errs.append(np.max(np.abs(U[:, 0] - u)))
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0
