"""Pins of the FP64 oracle against facts fixed by the paper and by
mathematics, not by the oracle itself (CPU only).

Each test names what it pins.  A plausible slip in the oracle -- a dropped
term, a wrong sign, a transposed operand, a wrong normalisation -- fails at
least one of these.
"""
import math

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fem, galerkin, kl, pce



# --------------------------------------------------------------------------
# Hermite chaos: multi-indices, triple products (Sec. 2.1, Eq. Galerkin_L_exp)
# --------------------------------------------------------------------------

def gauss_hermite_expect(fn, npts):
    """E[fn(xi)] for xi ~ N(0, 1) by probabilists' Gauss-Hermite quadrature."""
    x, w = np.polynomial.hermite_e.hermegauss(npts)
    return np.sum(w * fn(x)) / math.sqrt(2.0 * math.pi)


def he(nu, x):
    c = np.zeros(nu + 1)
    c[nu] = 1.0
    return np.polynomial.hermite_e.hermeval(x, c)


def test_triple_1d_spot_values():
    assert pce.hermite_triple_1d(1, 1, 0) == 1          # <He_1^2> = 1
    assert pce.hermite_triple_1d(2, 2, 2) == 8          # <He_2^3> = 8
    assert pce.hermite_triple_1d(1, 1, 1) == 0          # odd moment
    assert pce.hermite_triple_1d(0, 3, 3) == 6          # <He_3^2> = 3!
    assert pce.hermite_triple_1d(4, 1, 1) == 0          # triangle rule


@pytest.mark.parametrize("dmax", [8])
def test_triple_1d_vs_quadrature(dmax):
    for a in range(dmax + 1):
        for b in range(dmax + 1):
            for c in range(dmax + 1):
                npts = (a + b + c) // 2 + 2
                quad = gauss_hermite_expect(lambda x: he(a, x) * he(b, x) * he(c, x), npts)
                assert round(quad) == pce.hermite_triple_1d(a, b, c), (a, b, c)
                scale = math.sqrt(math.factorial(a) * math.factorial(b) * math.factorial(c))
                assert abs(quad - pce.hermite_triple_1d(a, b, c)) <= 1e-11 * scale


def test_multi_index_order_golden():
    # degree ascending, lexicographically descending within a degree
    got = pce.multi_indices(2, 2).tolist()
    assert got == [[0, 0], [1, 0], [0, 1], [2, 0], [1, 1], [0, 2]]
    got3 = pce.multi_indices(3, 1).tolist()
    assert got3 == [[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]]
    for L, p in [(1, 5), (3, 3), (4, 3), (6, 3)]:
        mi = pce.multi_indices(L, p)
        assert len(mi) == math.comb(L + p, p)
        assert len({tuple(r) for r in mi}) == len(mi)
        assert mi.sum(axis=1).max() == p


# sizes of the five problem families, computed independently when the
# problem was specified (counts of P, K and nonzero triples T)
COUNTS = [((2, 2, 4), 6, 15, 57), ((4, 3, 6), 35, 210, 2395), ((6, 3, 6), 84, 924, 12845),
          ((4, 4, 8), 70, 495, 12585), ((3, 3, 2), 20, 10, 218)]


@pytest.mark.parametrize("lpq,P,K,T", COUNTS)
def test_counts(lpq, P, K, T):
    L, p, q = lpq
    kab, num, g = pce.triple_products(L, p, q)
    assert pce.n_terms(L, p) == P and pce.n_terms(L, q) == K and len(kab) == T
    # ordered by k, then a, then b
    key = kab[:, 0] * 10**8 + kab[:, 1] * 10**4 + kab[:, 2]
    assert np.all(np.diff(key) > 0)


def test_triples_vs_tensor_quadrature():
    """Every <psi_k psi_a psi_b> of (L, p, q) = (2, 2, 4), including the zero
    ones, against 2D tensor Gauss-Hermite quadrature of the orthonormal
    polynomials."""
    L, p, q = 2, 2, 4
    G = pce.galerkin_matrices(L, p, q)
    outs, ins = pce.multi_indices(L, p), pce.multi_indices(L, q)
    x, w = np.polynomial.hermite_e.hermegauss(8)
    w = w / math.sqrt(2 * math.pi)
    X1, X2 = np.meshgrid(x, x, indexing="ij")
    W = np.outer(w, w)

    def psi(al):
        return (he(int(al[0]), X1) / math.sqrt(math.factorial(al[0]))
                * he(int(al[1]), X2) / math.sqrt(math.factorial(al[1])))
    for k, ak in enumerate(ins):
        for a, aa in enumerate(outs):
            for b, ab in enumerate(outs):
                ref = np.sum(W * psi(ak) * psi(aa) * psi(ab))
                assert abs(ref - G[k, a, b]) < 1e-12, (k, a, b)
    # orthonormality: G_0 = I
    assert np.array_equal(G[0], np.eye(len(outs)))


# --------------------------------------------------------------------------
# Lognormal input PCE (Eq. inputlogn)
# --------------------------------------------------------------------------

def test_lognormal_1d_vs_quadrature():
    for gval in [-0.7, 0.1, 0.55]:
        cb = pce.lognormal_coefficients(np.array([0.2]), np.array([[gval]]), 6)[:, 0]
        for nu in range(7):
            ref = gauss_hermite_expect(
                lambda x: np.exp(0.2 + gval * x) * he(nu, x) / math.sqrt(math.factorial(nu)), 40)
            assert abs(cb[nu] - ref) <= 1e-13 * max(1.0, abs(ref)), (gval, nu)


def test_lognormal_2d_vs_quadrature():
    g = np.array([[0.3], [-0.45]])
    cb = pce.lognormal_coefficients(np.zeros(1), g, 4)[:, 0]
    x, w = np.polynomial.hermite_e.hermegauss(30)
    w = w / math.sqrt(2 * math.pi)
    X1, X2 = np.meshgrid(x, x, indexing="ij")
    W = np.outer(w, w)
    for k, al in enumerate(pce.multi_indices(2, 4)):
        psi = (he(int(al[0]), X1) / math.sqrt(math.factorial(al[0]))
               * he(int(al[1]), X2) / math.sqrt(math.factorial(al[1])))
        ref = np.sum(W * np.exp(0.3 * X1 - 0.45 * X2) * psi)
        assert abs(cb[k] - ref) < 1e-13


def test_element_galerkin_matrix_closed_form():
    """sum_k c_bar_k G_k equals c_0 * prod_i Mtilde(g_i)[a_i, b_i] (shifted
    Gaussian identity), exact when q >= 2p."""
    L, p = 3, 3
    q = 2 * p
    g = np.array([0.31, -0.22, 0.15])
    cb = pce.lognormal_coefficients(np.array([0.1]), g[:, None], q)[:, 0]
    G = pce.galerkin_matrices(L, p, q)
    lhs = np.einsum("k,kab->ab", cb, G)
    outs = pce.multi_indices(L, p)
    Ms = [pce.shifted_gaussian_matrix(gi, p + 1) for gi in g]
    c0 = math.exp(0.1 + 0.5 * np.sum(g ** 2))
    rhs = np.empty_like(lhs)
    for a, aa in enumerate(outs):
        for b, ab in enumerate(outs):
            v = c0
            for i in range(L):
                v *= Ms[i][aa[i], ab[i]] / math.sqrt(math.factorial(aa[i]) * math.factorial(ab[i]))
            rhs[a, b] = v
    assert np.max(np.abs(lhs - rhs)) < 1e-13 * np.max(np.abs(rhs))
    # raising q beyond 2p changes no Galerkin entry
    cb2 = pce.lognormal_coefficients(np.array([0.1]), g[:, None], q + 2)[:, 0]
    G2 = pce.galerkin_matrices(L, p, q + 2)
    assert np.max(np.abs(np.einsum("k,kab->ab", cb2, G2) - lhs)) < 1e-14 * np.max(np.abs(lhs))


def test_shifted_gaussian_matrix_vs_quadrature():
    gval = 0.37
    M = pce.shifted_gaussian_matrix(gval, 5)
    for m in range(5):
        for k in range(5):
            ref = gauss_hermite_expect(lambda x: np.exp(gval * x - gval ** 2 / 2) * he(m, x) * he(k, x), 40)
            assert abs(M[m, k] - ref) < 1e-12 * max(1, abs(ref))


# --------------------------------------------------------------------------
# KL expansion (Eqs. KLE, CovarKer2DNLP)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("b", [0.2, 0.5, 1.0])
def test_kl_1d_vs_nystrom(b):
    ev, s, vec = kl.nystrom_1d(b, npts=2000)
    modes = kl.eigen_1d(b, 8)
    for m, mode in enumerate(modes):
        # Nystrom on a kernel with a kink converges like 1/npts^2: 5e-6 relative
        assert abs(mode[0] - ev[m]) <= 5e-6 * ev[0], (m, mode[0], ev[m])
    # eigenfunction shape: Nystrom vector is +-phi
    for m, mode in enumerate(modes[:4]):
        phi = kl.phi_1d(mode, s)
        v = vec[:, m]
        v = v * np.sign(np.dot(v, phi))
        v = v / math.sqrt(np.sum(v * v * (0.5 * np.polynomial.legendre.leggauss(2000)[1])))
        assert np.max(np.abs(v - phi)) < 1e-4


def test_kl_1d_orthonormal_and_trace():
    b = 0.5
    modes = kl.eigen_1d(b, 4000)
    xg, wg = np.polynomial.legendre.leggauss(400)
    s, w = 0.5 * xg, 0.5 * wg
    phis = np.array([kl.phi_1d(m, s) for m in modes[:10]])
    gram = (phis * w) @ phis.T
    assert np.max(np.abs(gram - np.eye(10))) < 1e-12
    # sum of all eigenvalues = trace = |[-1/2, 1/2]| = 1 (tail ~ 2/(b pi^2 n))
    lam = np.array([m[0] for m in modes])
    tail = 2.0 / (b * math.pi ** 2 * 4000)
    assert abs(lam.sum() - 1.0) < 2 * tail
    assert np.all(np.diff(lam) < 0)


def test_kl_eigen_equation():
    """int K(s,t) phi(t) dt = lambda phi(s) at a few points (fine quadrature
    split at the kink)."""
    b = 0.3
    for mode in kl.eigen_1d(b, 5):
        for s0 in [-0.4, 0.05, 0.33]:
            acc = 0.0
            for lo, hi in [(-0.5, s0), (s0, 0.5)]:
                xg, wg = np.polynomial.legendre.leggauss(200)
                t = 0.5 * (hi - lo) * xg + 0.5 * (hi + lo)
                acc += np.sum(0.5 * (hi - lo) * wg * np.exp(-np.abs(s0 - t) / b) * kl.phi_1d(mode, t))
            assert abs(acc - mode[0] * kl.phi_1d(mode, s0)) < 1e-12


def test_kl_2d_order_and_ties():
    modes = kl.modes_2d(0.3, 0.5, 0.5, 6)
    lam = [m[0] for m in modes]
    assert all(lam[i] >= lam[i + 1] for i in range(5))
    assert [(m[1], m[2]) for m in modes[:3]] == [(0, 0), (0, 1), (1, 0)]
    # total variance of the 2D field is sigma^2 per unit area
    ex = kl.eigen_1d(0.5, 3000)
    tot = 0.3 * sum(m[0] for m in ex) ** 2
    assert abs(tot - 0.3) < 1e-3


# --------------------------------------------------------------------------
# FEM (Sec. 2.1 discretisation; appendix Eq. qunlc4 with m = 0)
# --------------------------------------------------------------------------

def test_p1_element_matrices():
    # right-isoceles P1 matrices: right-angle vertex 1, legs -1/2, hypotenuse 0
    assert np.array_equal(fem.p1_stiffness(fem.LOWER),
                          np.array([[0.5, -0.5, 0], [-0.5, 1, -0.5], [0, -0.5, 0.5]]))
    assert np.array_equal(fem.p1_stiffness(fem.UPPER),
                          np.array([[0.5, 0, -0.5], [0, 0.5, -0.5], [-0.5, -0.5, 1]]))


def test_unit_coefficient_is_five_point_laplacian():
    N = 9
    A = fem.assemble(N, np.ones(2 * N * N)).toarray()
    m = N - 1
    T = 2 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1)
    ref = np.kron(np.eye(m), T) + np.kron(T, np.eye(m))
    assert np.array_equal(A, ref)
    assert np.allclose(fem.load_vector(N), 1.0 / N ** 2, rtol=1e-15, atol=0)


def test_linear_solution_reproduced():
    """Appendix problem with m = 0 (q = 1): u = x is in the P1 space, so the
    discrete solution equals it at every node.  The same holds for a
    coefficient that varies only with y (constant on each row of cells)."""
    N = 12
    row = np.arange(2 * N * N) // (2 * N)
    coef = 1.0 + 0.5 * np.sin(row)
    A1, rhs1, ii, jj = fem.assemble_dirichlet_x(N, np.ones(2 * N * N), 0.0, 1.0)
    u1 = spla.spsolve(A1.tocsc(), rhs1)
    assert np.max(np.abs(u1 - ii / N)) < 1e-13
    A, rhs, ii, jj = fem.assemble_dirichlet_x(N, coef, 0.0, 1.0)
    u = spla.spsolve(A.tocsc(), rhs)
    assert np.max(np.abs(u - ii / N)) < 1e-13


def test_fem_second_order_convergence():
    f = lambda x, y: 2 * math.pi ** 2 * np.sin(math.pi * x) * np.sin(math.pi * y)
    errs = []
    for N in [8, 16, 32]:
        A = fem.assemble(N, np.ones(2 * N * N)).tocsc()
        u = spla.spsolve(A, fem.load_vector_f(N, f))
        i, j = np.meshgrid(np.arange(1, N), np.arange(1, N), indexing="xy")
        ex = np.sin(math.pi * i.ravel() / N) * np.sin(math.pi * j.ravel() / N)
        errs.append(np.sqrt(np.mean((u - ex) ** 2)))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.8 < r < 2.3 for r in rates), rates


def test_shared_pattern_is_five_point():
    prob = galerkin.build(16, 2, 1, 2)
    n, N = prob.n, prob.N
    assert len(prob.colidx) == 5 * n - 4 * (N - 1)
    for r in range(n):
        cols = prob.colidx[prob.rowptr[r]:prob.rowptr[r + 1]]
        assert np.all(np.diff(cols) > 0)
        assert set(cols - r) <= {-(N - 1), -1, 0, 1, N - 1}


# --------------------------------------------------------------------------
# The coupled Galerkin system and its solution
# --------------------------------------------------------------------------

def test_sigma_zero_limit():
    """sigma = 0: A = I kron A_det; X[:,0] = deterministic solve, rest 0."""
    prob = galerkin.build(16, 2, 2, 4, sigma2=0.0)
    X = galerkin.solve_direct(prob)
    udet = spla.spsolve(fem.assemble(16, np.ones(2 * 256)).tocsc(), fem.load_vector(16))
    assert np.max(np.abs(X[:, 0] - udet)) < 1e-13 * np.max(np.abs(udet))
    assert np.all(X[:, 1:] == 0.0)


def test_constant_random_field_closed_form():
    """One user mode g_1 = gamma everywhere: X = u_det (B^{-1} e_0)^T with
    B = e^{gamma^2/2} Mtilde(gamma) on the output set."""
    N, p, gamma = 12, 4, 0.4
    E = 2 * N * N
    prob = galerkin.build(N, 1, p, 2 * p, user_modes=np.full((1, E), gamma))
    X = galerkin.solve_direct(prob)
    M = pce.shifted_gaussian_matrix(gamma, p + 1)
    fac = np.array([math.sqrt(math.factorial(i)) for i in range(p + 1)])
    B = math.exp(gamma ** 2 / 2) * M / np.outer(fac, fac)
    w = np.linalg.solve(B, np.eye(p + 1)[0])
    udet = spla.spsolve(fem.assemble(N, np.ones(E)).tocsc(), fem.load_vector(N))
    ref = np.outer(udet, w)
    assert np.max(np.abs(X - ref)) < 1e-12 * np.max(np.abs(ref))


def test_manufactured_solution_direct():
    prob = galerkin.build(16, 3, 2, 4, sigma2=0.3, bx=0.4, by=0.7)
    Xs = np.random.default_rng(1234).standard_normal((prob.n, prob.P))
    F = galerkin.apply(prob, Xs)
    X = galerkin.solve_direct(prob, F)
    assert np.linalg.norm(X - Xs) / np.linalg.norm(Xs) < 1e-10


def test_apply_three_ways_and_symmetry():
    prob = galerkin.build(12, 2, 3, 6, sigma2=0.3, bx=0.5, by=0.5)
    rng = np.random.default_rng(5)
    X1 = rng.standard_normal((prob.n, prob.P))
    X2 = rng.standard_normal((prob.n, prob.P))
    Y1 = galerkin.apply(prob, X1)
    M = galerkin.assembled(prob)
    Y1b = galerkin.from_vec(M @ galerkin.to_vec(X1), prob.n, prob.P)
    rows = [0, 7, prob.n - 1]
    Y1c = galerkin.apply_rows(prob, X1, rows)
    assert np.max(np.abs(Y1 - Y1b)) < 1e-13 * np.max(np.abs(Y1))
    assert np.max(np.abs(Y1[rows] - Y1c)) < 1e-13 * np.max(np.abs(Y1))
    Y2 = galerkin.apply(prob, X2)
    assert abs(np.sum(X2 * Y1) - np.sum(Y2 * X1)) < 1e-13 * abs(np.sum(X2 * Y1)) + 1e-12
    assert np.sum(X1 * Y1) > 0
    ev = np.linalg.eigvalsh(M.toarray())
    assert ev.min() > 0


def edge_form_apply(prob, X):
    """The operator written edge by edge (the P1 "/" mesh: the diagonal
    couplings vanish, rows sum to zero with their Dirichlet neighbours):
    y_r = sum over the four edges e of r of B^e (x_r - x_c), B^e = sum_k
    w_k(e) G_k, w_k(e) half the sum of c_k over the two triangles that
    share e; x = 0 on the boundary."""
    N = prob.N
    G = prob.G()
    cb = prob.cbar
    Y = np.zeros_like(X)

    def flux(w, ra, rb):
        xa = X[ra] if ra >= 0 else 0.0
        xb = X[rb] if rb >= 0 else 0.0
        f = np.tensordot(w, G, axes=1) @ (xa - xb)
        if ra >= 0:
            Y[ra] += f
        if rb >= 0:
            Y[rb] -= f

    for j in range(1, N):
        for i in range(N):
            # (i, j)-(i+1, j): lower triangle of cell (i, j), upper of (i, j-1)
            w = 0.5 * (cb[:, 2 * (j * N + i)] + cb[:, 2 * ((j - 1) * N + i) + 1])
            flux(w, int(fem.interior_index(N, i, j)), int(fem.interior_index(N, i + 1, j)))
    for j in range(N):
        for i in range(1, N):
            # (i, j)-(i, j+1): upper triangle of cell (i, j), lower of (i-1, j)
            w = 0.5 * (cb[:, 2 * (j * N + i) + 1] + cb[:, 2 * (j * N + i - 1)])
            flux(w, int(fem.interior_index(N, i, j)), int(fem.interior_index(N, i, j + 1)))
    return Y


def test_edge_form_equals_kronecker_apply():
    """The edge form of the operator (summed P x P block per edge, applied
    to the difference of the end nodes), which the refinement residual
    uses, against the Kronecker apply sum_k A_k X G_k^T of the assembled
    stiffness matrices (Sec. 2.1, Eq. Galerkin_L_exp)."""
    for args in ((8, 2, 2, 4), (9, 3, 1, 2), (2, 1, 2, 4)):
        prob = galerkin.build(*args, sigma2=0.3, bx=0.5, by=0.5)
        X = np.random.default_rng(3).standard_normal((prob.n, prob.P))
        Y = galerkin.apply(prob, X)
        Ye = edge_form_apply(prob, X)
        assert np.max(np.abs(Ye - Y)) < 1e-12 * np.max(np.abs(Y))


def test_gmres_matches_direct():
    prob = galerkin.build(32, 2, 2, 4, sigma2=0.3, bx=0.5, by=0.5)
    Xd = galerkin.solve_direct(prob)
    Xg, its, hist = galerkin.solve_gmres(prob, tol=1e-12)
    assert galerkin.relres(prob, Xg) < 1e-12
    assert np.linalg.norm(Xg - Xd) / np.linalg.norm(Xd) < 1e-11


def test_monte_carlo_mean_variance():
    """Tiny-mesh Monte Carlo of the deterministic problem with
    c = exp(sum_i g_i xi_i): the SG mean X[:,0] and variance
    sum_{a>=1} X[:,a]^2 agree within 4 standard errors plus the PCE
    truncation error (change from p to p+1)."""
    N, L, s2 = 16, 2, 0.09
    prob = galerkin.build(N, L, 3, 6, sigma2=s2, bx=0.5, by=0.5)
    prob4 = galerkin.build(N, L, 4, 8, sigma2=s2, bx=0.5, by=0.5)
    X = galerkin.solve_direct(prob)
    X4 = galerkin.solve_direct(prob4)
    mean_sg, var_sg = X[:, 0], np.sum(X[:, 1:] ** 2, axis=1)
    trunc_m = np.abs(X4[:, 0] - mean_sg)
    trunc_v = np.abs(np.sum(X4[:, 1:] ** 2, axis=1) - var_sg)
    rng = np.random.default_rng(7)
    S = 20000
    xi = rng.standard_normal((S, L))
    rows, cols, elem, kval = fem.element_entries(N)
    b = fem.load_vector(N)
    n = prob.n
    # dense batched solves of the sampled deterministic systems
    us = np.empty((S, n))
    chunk = 500
    for s0 in range(0, S, chunk):
        cs = np.exp(xi[s0:s0 + chunk] @ prob.gfield)          # [chunk, E]
        A = np.zeros((len(cs), n, n))
        for t in range(len(cs)):
            np.add.at(A[t], (rows, cols), cs[t][elem] * kval)
        us[s0:s0 + chunk] = np.linalg.solve(A, np.broadcast_to(b, (len(cs), n))[..., None])[..., 0]
    mc_mean = us.mean(axis=0)
    mc_var = us.var(axis=0, ddof=1)
    se_mean = np.sqrt(mc_var / S)
    se_var = mc_var * math.sqrt(2.0 / (S - 1))
    assert np.all(np.abs(mc_mean - mean_sg) <= 4 * se_mean + trunc_m + 1e-15)
    assert np.all(np.abs(mc_var - var_sg) <= 4 * se_var + trunc_v + 1e-18)
    # and the variance is genuinely resolved (not trivially inside the band)
    assert np.max(var_sg) > 10 * np.max(se_var)


def test_paper_verification_setting_against_collocation():
    """The paper's verification setting for the linear problem (Sec. 5,
    Fig. mcs_verify_poisson: three random variables, input order 2, output
    order 3, sigma = 0.1), checked against a 6^3-point Gauss-Hermite
    collocation of the exact lognormal problem instead of Monte Carlo: the
    SG mean and standard deviation agree (the input truncation at order 2
    is the only difference)."""
    import itertools
    import scipy.sparse.linalg as spla
    from numpy.polynomial import hermite_e as H
    N = 20
    prob = galerkin.build(N, 3, 3, 2, sigma2=0.01, bx=0.5, by=0.5)
    U = galerkin.solve_direct(prob)
    x, w = H.hermegauss(6)
    w = w / np.sqrt(2.0 * np.pi)
    b = fem.load_vector(N)
    m1 = np.zeros(prob.n)
    m2 = np.zeros(prob.n)
    for i, j, k in itertools.product(range(6), repeat=3):
        xi = np.array([x[i], x[j], x[k]])
        u = spla.spsolve(fem.assemble(N, np.exp(xi @ prob.gfield)).tocsc(), b)
        m1 += w[i] * w[j] * w[k] * u
        m2 += w[i] * w[j] * w[k] * u * u
    std_c = np.sqrt(m2 - m1 ** 2)
    std_sg = np.sqrt((U[:, 1:] ** 2).sum(1))
    assert np.linalg.norm(U[:, 0] - m1) / np.linalg.norm(m1) <= 1e-6
    assert np.linalg.norm(std_sg - std_c) / np.linalg.norm(std_c) <= 1e-3
