"""Polynomial chaos pieces of the SG method, written from Sec. 2.1.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* multi-index sets of total degree <= p  (Eq. inputpc: (M+p)!/(M!p!) terms)
* Hermite triple products m_ijk = <Psi_i Psi_j Psi_k>  (Eq. Galerkin_L_exp)
* lognormal input coefficients c_bar_alpha  (Eqs. inputlogn and the c_0 line
  below it; the printed formula is garbled, the exact generating-function form
  is used: c = c_0 sum_alpha prod_i g_i^{a_i}/a_i! He_alpha(xi))

Basis convention: the orthonormal probabilists' Hermite chaos
psi_alpha = prod_i He_{a_i}(xi_i)/sqrt(a_i!), so <psi_a psi_b> = delta_ab.
"""
from math import comb, factorial

import numpy as np


def multi_indices(L, p):
    """All alpha in N^L with |alpha| <= p (Eq. inputpc, output/input sets).

    Order: total degree ascending; within a degree, lexicographically
    DESCENDING in (alpha_1, ..., alpha_L), so degree 1 lists e_1 before e_2.
    The paper does not fix an order; this one is a stated reading.
    """
    out = []
    for d in range(p + 1):
        level = []

        def rec(prefix, left, dims):
            if dims == 1:
                level.append(tuple(prefix + [left]))
                return
            for first in range(left, -1, -1):
                rec(prefix + [first], left - first, dims - 1)

        if L == 0:
            if d == 0:
                level.append(())
        else:
            rec([], d, L)
        out.extend(level)
    assert len(out) == comb(L + p, p)
    return np.array(out, dtype=np.int64).reshape(len(out), L)


def hermite_triple_1d(a, b, c):
    """<He_a He_b He_c> under the standard normal law (integer).

    Textbook linearisation: with s = (a+b+c)/2 an integer and s >= max(a,b,c)
    the value is a! b! c! / ((s-a)! (s-b)! (s-c)!); otherwise 0.
    """
    if (a + b + c) % 2:
        return 0
    s = (a + b + c) // 2
    if s < a or s < b or s < c:
        return 0
    return (factorial(a) * factorial(b) * factorial(c)
            // (factorial(s - a) * factorial(s - b) * factorial(s - c)))


def alpha_factorial(alpha):
    out = 1
    for ai in alpha:
        out *= factorial(int(ai))
    return out


def triple_products(L, p, q):
    """Nonzero <psi_k psi_a psi_b> for k < K (input set, degree q) and
    a, b < P (output set, degree p)  -- the m_ijk of Eq. Galerkin_L_exp,
    stored as nonzeros only (Sec. 2.1, the paragraph after Eq. Galerkin_L_exp).

    Returns (kab int64 [T,3], num int64 [T], g float64 [T]) ordered by
    k, then a, then b.  num is the unnormalised integer
    prod_i <He_{k_i} He_{a_i} He_{b_i}>; g = num / sqrt(k! a! b!).
    The product over dimensions is taken with a table of the 1D integers.
    """
    out_set = multi_indices(L, p)
    in_set = multi_indices(L, q)
    t1 = np.zeros((q + 1, p + 1, p + 1), dtype=np.int64)
    for c in range(q + 1):
        for a in range(p + 1):
            for b in range(p + 1):
                t1[c, a, b] = hermite_triple_1d(c, a, b)
    num = np.ones((len(in_set), len(out_set), len(out_set)), dtype=np.int64)
    for i in range(L):
        num *= t1[in_set[:, i][:, None, None], out_set[:, i][None, :, None],
                  out_set[:, i][None, None, :]]
    k, a, b = np.nonzero(num)          # row-major: ordered by k, a, b
    fact = np.array([alpha_factorial(al) for al in in_set], dtype=np.float64)
    facp = np.array([alpha_factorial(al) for al in out_set], dtype=np.float64)
    nums = num[k, a, b]
    g = nums / np.sqrt(fact[k] * facp[a] * facp[b])
    return np.stack([k, a, b], axis=1).astype(np.int64), nums.astype(np.int64), g


def galerkin_matrices(L, p, q):
    """Dense G_k[a, b] = <psi_k psi_a psi_b>, shape [K, P, P] (small cases)."""
    P = comb(L + p, p)
    K = comb(L + q, q)
    kab, _, g = triple_products(L, p, q)
    G = np.zeros((K, P, P))
    G[kab[:, 0], kab[:, 1], kab[:, 2]] = g
    return G


def lognormal_coefficients(g0, gmodes, q):
    """Input PCE coefficients of c = exp(g0 + sum_i g_i xi_i) (Eq. inputlogn).

    g0: array [E]; gmodes: array [L, E] with g_i = sqrt(lambda_i) phi_i.
    Returns c_bar [K, E] in the orthonormal basis:
    c_bar_alpha = c_0 prod_i g_i^{a_i} / sqrt(a_i!),
    c_0 = exp(g0 + 0.5 sum_i g_i^2)  (the mean line under Eq. inputlogn).
    """
    gmodes = np.atleast_2d(np.asarray(gmodes, dtype=np.float64))
    L = gmodes.shape[0]
    in_set = multi_indices(L, q)
    c0 = np.exp(np.asarray(g0, dtype=np.float64) + 0.5 * np.sum(gmodes ** 2, axis=0))
    out = np.empty((len(in_set), gmodes.shape[1]))
    for k, alpha in enumerate(in_set):
        term = c0.copy()
        for i in range(L):
            ai = int(alpha[i])
            if ai:
                term = term * gmodes[i] ** ai / np.sqrt(float(factorial(ai)))
        out[k] = term
    return out


def shifted_gaussian_matrix(g, n):
    """M(g)[m, k] = <exp(g xi - g^2/2) He_m(xi) He_k(xi)>, m, k < n.

    Independent closed form used as a pin: He_m(xi + g) = sum_j C(m,j)
    g^{m-j} He_j(xi) gives M(g)[m,k] = sum_j C(m,j) C(k,j) j! g^{m+k-2j}.
    """
    M = np.zeros((n, n))
    for m in range(n):
        for k in range(n):
            M[m, k] = sum(comb(m, j) * comb(k, j) * factorial(j) * g ** (m + k - 2 * j)
                          for j in range(min(m, k) + 1))
    return M


def n_terms(L, p):
    return comb(L + p, p)
