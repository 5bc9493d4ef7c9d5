"""Stochastic nonlinear Poisson problem (Sec. 2.2, Eqs. NLP_StrongPDE,
stonlp_system, vectorvalPDENL, AjkTkl):

    -div( c(x, xi) (1 + alpha u(x, xi)) grad u(x, xi) ) = f,   u = 0 on the boundary,

with c the lognormal field of the linear problem.  The Galerkin projection
onto the output chaos gives, for every test mode l,

    sum_{i,k} m_ikl  A(c_i) u_k  +  alpha sum_{i,j,k} t_ijkl  A(c_i u_j) u_k  =  b_l,

with m_ikl = <psi_i psi_k psi_l>, t_ijkl = <psi_i psi_j psi_k psi_l>, i over
the input chaos (the coefficient's modes c_i), j, k, l over the output chaos.
The paper solves it by Picard iteration: the factor u_j of the second term is
taken from the previous iterate, so each step is one linear SG solve with the
operator (A + T^n).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Discretisation reading: A(w) is the P1 stiffness matrix of a piecewise-constant
coefficient w_e, like the linear problem's A_k = A(c_k).  The product c_i u_j
inside the integral is taken per element with u_j replaced by its element
average (the mean of the element's three vertex values, zero at Dirichlet
vertices).  alpha = 1 in the paper's experiments; it is a parameter here.
The stopping rule is the paper's relative change of the solution,
||U^{n+1} - U^n|| / ||U^{n+1}|| <= tol.
"""
from math import factorial

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem, galerkin, pce


def hermite_quad_1d(a, b, c, d):
    """<He_a He_b He_c He_d> (integer) by the linearisation of He_a He_b:

        He_a He_b = sum_m (<He_a He_b He_m> / m!) He_m,

    so the fourfold moment is sum_m <He_a He_b He_m> <He_m He_c He_d> / m!.
    Each <He_a He_b He_m> / m! is an integer (a binomial product), so the
    sum is exact in integers."""
    tot = 0
    for m in range(0, a + b + 1):
        t = pce.hermite_triple_1d(a, b, m)
        if t == 0:
            continue
        lin = t // factorial(m)
        assert lin * factorial(m) == t
        tot += lin * pce.hermite_triple_1d(m, c, d)
    return tot


def four_products(L, p, q):
    """Dense t[i, j, k, l] = <psi_i psi_j psi_k psi_l> in the orthonormal
    basis, i < K (input set, degree q), j, k, l < P (output set, degree p);
    the product over the L dimensions of the 1D integers, divided by
    sqrt(i! j! k! l!) (multi-index factorials)."""
    out_set = pce.multi_indices(L, p)
    in_set = pce.multi_indices(L, q)
    K, P = len(in_set), len(out_set)
    t1 = np.zeros((q + 1, p + 1, p + 1, p + 1), dtype=object)
    for a in range(q + 1):
        for b in range(p + 1):
            for c in range(p + 1):
                for e in range(p + 1):
                    t1[a, b, c, e] = hermite_quad_1d(a, b, c, e)
    num = np.ones((K, P, P, P), dtype=np.float64)
    for i in range(L):
        num *= t1[in_set[:, i][:, None, None, None], out_set[:, i][None, :, None, None],
                  out_set[:, i][None, None, :, None], out_set[:, i][None, None, None, :]].astype(np.float64)
    fin = np.array([pce.alpha_factorial(al) for al in in_set], dtype=np.float64)
    fout = np.array([pce.alpha_factorial(al) for al in out_set], dtype=np.float64)
    norm = np.sqrt(fin[:, None, None, None] * fout[None, :, None, None] * fout[None, None, :, None]
                   * fout[None, None, None, :])
    return num / norm


def element_average(N, U):
    """Per-element average of the vertex values of every column of U
    ([n interior nodes, P] -> [E elements, P]); boundary vertices are 0."""
    el = fem.elements(N)
    idx = fem.interior_index(N, el[:, :, 0], el[:, :, 1])        # [E, 3]
    Upad = np.vstack([np.asarray(U, dtype=np.float64), np.zeros((1, U.shape[1]))])
    return Upad[np.where(idx >= 0, idx, U.shape[0])].mean(axis=1)


def nonlinear_matrix(prob, U, t4, alpha=1.0):
    """The assembled linearised operator (A + alpha T(U)) of one Picard step,
    sum_i kron(G_i, A(c_i)) + alpha sum_{i,j} kron(T_ij, A(c_i ubar_j)),
    with T_ij[l, k] = t_ijkl, in the mode-major unknown order of
    ``galerkin.assembled``."""
    M = galerkin.assembled(prob)
    if alpha == 0.0:
        return M
    ubar = element_average(prob.N, U)                            # [E, P]
    for i in range(prob.K):
        for j in range(prob.P):
            Tij = t4[i, j]                                       # [k, l], symmetric
            if not np.any(Tij) or not np.any(ubar[:, j]):
                continue
            A = fem.assemble(prob.N, prob.cbar[i] * ubar[:, j])
            M = M + alpha * sp.kron(sp.csr_matrix(Tij.T), A, format="csr")
    return M.tocsr()


def picard(prob, alpha=1.0, tol=1e-6, max_it=50, t4=None):
    """Picard iteration of Eq. stonlp_system from U^0 = 0 (the first step is
    the linear SG solve).  Returns (U [n, P], iterations, history of the
    relative change)."""
    if t4 is None:
        t4 = four_products(prob.L, prob.p, prob.q)
    F = galerkin.to_vec(prob.rhs())
    U = np.zeros((prob.n, prob.P))
    hist = []
    for it in range(1, max_it + 1):
        M = nonlinear_matrix(prob, U, t4, alpha).tocsc()
        Unew = galerkin.from_vec(spla.spsolve(M, F), prob.n, prob.P)
        change = np.linalg.norm(Unew - U) / np.linalg.norm(Unew)
        hist.append(change)
        U = Unew
        if change <= tol:
            return U, it, hist
    return U, max_it, hist


def deterministic_picard(N, coef, alpha=1.0, tol=1e-12, max_it=200):
    """The deterministic problem -div(coef (1 + alpha u) grad u) = 1 for one
    coefficient field coef_e (per element), by the same element-average
    reading and Picard iteration from u = 0.  Returns (u [n], iterations)."""
    b = fem.load_vector(N)
    u = np.zeros((N - 1) ** 2)
    for it in range(1, max_it + 1):
        ubar = element_average(N, u[:, None])[:, 0]
        A = fem.assemble(N, np.asarray(coef) * (1.0 + alpha * ubar)).tocsc()
        unew = spla.spsolve(A, b)
        change = np.linalg.norm(unew - u) / np.linalg.norm(unew)
        u = unew
        if change <= tol:
            return u, it
    return u, max_it
