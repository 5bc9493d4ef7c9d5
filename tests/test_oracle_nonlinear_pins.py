"""Pins of the nonlinear-problem oracle (Sec. 2.2, Eqs. NLP_StrongPDE,
stonlp_system, AjkTkl) against facts that do not come from the oracle's own
formulas: Gauss-Hermite quadrature for the fourfold products, the linear
solve at alpha = 0, the deterministic problem at sigma = 0, stochastic
collocation of the deterministic problem for one random variable, and the
Kirchhoff transform of the deterministic problem."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
from numpy.polynomial import hermite_e as H

from oracle import fem, galerkin, nonlinear, pce

pytestmark = pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")


def psi(alpha, xs):
    """Orthonormal multivariate Hermite polynomial at points xs [m, L]."""
    out = np.ones(len(xs))
    for d, a in enumerate(alpha):
        c = np.zeros(int(a) + 1)
        c[-1] = 1.0
        out *= H.hermeval(xs[:, d], c) / np.sqrt(float(pce.alpha_factorial([a])))
    return out


def test_four_products_against_gauss_hermite_quadrature():
    """Every t_ijkl (L = 2, p = 2, q = 3) equals the tensor Gauss-Hermite
    quadrature of psi_i psi_j psi_k psi_l (12 points a dimension: exact
    for the degree 9 integrands)."""
    L, p, q = 2, 2, 3
    t4 = nonlinear.four_products(L, p, q)
    x, w = H.hermegauss(12)
    w = w / np.sqrt(2.0 * np.pi)
    X1, X2 = np.meshgrid(x, x, indexing="ij")
    pts = np.stack([X1.ravel(), X2.ravel()], axis=1)
    wts = np.outer(w, w).ravel()
    ins, outs = pce.multi_indices(L, q), pce.multi_indices(L, p)
    vin = np.array([psi(a, pts) for a in ins])
    vout = np.array([psi(a, pts) for a in outs])
    ref = np.einsum("m,im,jm,km,lm->ijkl", wts, vin, vout, vout, vout)
    assert t4.shape == ref.shape
    assert np.max(np.abs(t4 - ref)) <= 1e-12


def test_four_products_with_psi0_are_the_triple_products_and_symmetric():
    """psi_0 = 1: t_i0kl = m_ikl (the triple products of the linear
    problem); t_ijkl is symmetric under permutations of j, k, l."""
    L, p, q = 3, 2, 4
    t4 = nonlinear.four_products(L, p, q)
    G = pce.galerkin_matrices(L, p, q)
    assert np.array_equal(t4[:, 0], G)
    for perm in ((0, 1, 3, 2), (0, 2, 1, 3), (0, 3, 2, 1)):
        assert np.array_equal(t4, np.transpose(t4, perm))


def test_alpha_zero_is_the_linear_solve():
    prob = galerkin.build(10, 2, 2, 4, sigma2=0.3, bx=0.5, by=0.5)
    U, its, hist = nonlinear.picard(prob, alpha=0.0, tol=1e-12)
    assert its == 2 and hist[-1] == 0.0
    Ud = galerkin.solve_direct(prob)
    assert np.linalg.norm(U - Ud) <= 1e-13 * np.linalg.norm(Ud)


def test_sigma_zero_is_the_deterministic_problem():
    """Without randomness only the mean mode is nonzero and equals the
    deterministic nonlinear solution for the coefficient exp(g0)."""
    g0 = 0.4
    prob = galerkin.build(10, 2, 2, 4, sigma2=0.0, bx=0.5, by=0.5, g0=g0)
    U, its, _ = nonlinear.picard(prob, alpha=1.0, tol=1e-13)
    ud, _ = nonlinear.deterministic_picard(10, np.full(2 * 100, np.exp(g0)), alpha=1.0, tol=1e-13)
    assert np.linalg.norm(U[:, 0] - ud) <= 1e-12 * np.linalg.norm(ud)
    assert np.max(np.abs(U[:, 1:])) <= 1e-14 * np.max(np.abs(ud))


def collocation(prob, npts=24):
    """Mean and variance of the deterministic nonlinear solution over the
    Gauss-Hermite nodes of the single random variable."""
    x, w = H.hermegauss(npts)
    w = w / np.sqrt(2.0 * np.pi)
    us = np.array([nonlinear.deterministic_picard(prob.N, np.exp(prob.gfield[0] * xm), alpha=1.0,
                                                  tol=1e-13)[0] for xm in x])
    mean = w @ us
    return mean, w @ (us - mean) ** 2


def test_stochastic_galerkin_approaches_collocation():
    """One random variable (sigma^2 = 0.25): the SG mean and variance
    (sum of the squared higher modes) approach the collocation moments
    spectrally as the output order p grows (input order 2p)."""
    errs = []
    for p in (2, 3):
        prob = galerkin.build(8, 1, p, 2 * p, sigma2=0.25, bx=0.5, by=0.5)
        U, _, _ = nonlinear.picard(prob, alpha=1.0, tol=1e-12)
        mean, var = collocation(prob)
        errs.append((np.linalg.norm(U[:, 0] - mean) / np.linalg.norm(mean),
                     np.linalg.norm((U[:, 1:] ** 2).sum(1) - var) / np.linalg.norm(var)))
    (m2, v2), (m3, v3) = errs
    assert m3 <= 1e-5 and v3 <= 1e-3
    assert m2 / m3 >= 10 and v2 / v3 >= 10


def test_deterministic_reading_converges_to_the_kirchhoff_solution():
    """Constant coefficient c: u + alpha u^2 / 2 solves the linear problem
    c (-Laplace) v = 1, so u = (sqrt(1 + 2 alpha v) - 1) / alpha; the
    element-average discretisation converges to it at second order."""
    errs = []
    for N in (8, 16, 32):
        E = 2 * N * N
        u, _ = nonlinear.deterministic_picard(N, np.full(E, 2.0), alpha=1.0)
        v = spla.spsolve(fem.assemble(N, np.full(E, 2.0)).tocsc(), fem.load_vector(N))
        uk = np.sqrt(1.0 + 2.0 * v) - 1.0
        errs.append(np.max(np.abs(u - uk)) / np.max(np.abs(uk)))
    assert errs[0] < 1e-3
    for a, b in zip(errs, errs[1:]):
        assert 3.5 <= a / b <= 4.5


@pytest.fixture(scope="module")
def built():
    """The library, built in tree if needed (the table needs no GPU)."""
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("L,p,q", [(1, 4, 8), (2, 2, 4), (3, 2, 3), (4, 3, 6)])
def test_library_fourfold_products_match_the_oracle(built, L, p, q):
    """The library's host-only table of fourfold products (no GPU needed):
    the nonzero set and the integers bit-exact, the orthonormal values to
    rounding, against the oracle's linearisation."""
    import paper_2310_14649_gb300 as sg
    ijkl, num, t = sg.sg_fourfold_products(L, p, q)
    t4 = nonlinear.four_products(L, p, q)
    nz = np.argwhere(t4 != 0.0)
    assert np.array_equal(ijkl, nz.astype(np.int32))
    assert np.allclose(t, t4[tuple(nz.T)], rtol=1e-14, atol=0.0)
    # integers: the product over dimensions of the 1D moments
    ins, outs = pce.multi_indices(L, q), pce.multi_indices(L, p)
    for row, v in zip(ijkl[:: max(1, len(ijkl) // 400)], num[:: max(1, len(ijkl) // 400)]):
        i, j, k, l = row
        ref = 1
        for d in range(L):
            ref *= nonlinear.hermite_quad_1d(int(ins[i, d]), int(outs[j, d]), int(outs[k, d]), int(outs[l, d]))
        assert v == ref


def test_library_fourfold_products_arguments(built):
    import ctypes
    import paper_2310_14649_gb300 as sg
    from paper_2310_14649_gb300 import _lib
    lib = _lib.lib()
    n = ctypes.c_int64(0)
    assert lib.sg_fourfold_products(0, 2, 4, ctypes.byref(n), None, None, None) == -1
    assert lib.sg_fourfold_products(2, 9, 4, ctypes.byref(n), None, None, None) == -1
    assert lib.sg_fourfold_products(2, 2, 4, None, None, None, None) == -1
    assert lib.sg_fourfold_products(2, 2, 4, ctypes.byref(n), None, None, None) == 0 and n.value > 0
    small = ctypes.c_int64(n.value - 1)
    buf = (ctypes.c_int64 * n.value)()
    assert lib.sg_fourfold_products(2, 2, 4, ctypes.byref(small), None, buf, None) == -1
    with pytest.raises(sg.SgError):
        sg.sg_fourfold_products(13, 1, 1)
