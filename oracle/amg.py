"""Algebraic multigrid for the coarse problem (the BoomerAMG role of Sec. 3;
the paper states no AMG parameters, so a smoothed-aggregation hierarchy is
the stated reading).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Setup on an SPD matrix A (levels until <= 256 unknowns, at most 10 levels):
* strength: j != i is strong for i when |a_ij| >= theta sqrt(a_ii a_jj),
  theta = 0.08;
* aggregation in index order: (1) a node whose strong neighbours are all
  free starts an aggregate with them; (2) each remaining node joins the
  aggregate of its lowest-index strong neighbour aggregated in step 1;
  (3) each node still free starts an aggregate with its free strong
  neighbours;
* tentative prolongator: 1/sqrt(|aggregate|) on the aggregate;
* P = (I - omega D^{-1} A) P_tent, omega = 4 / (3 rho), rho from 20 power
  iterations on D^{-1} A started at x_i = 1 + (i mod 3);
* A_next = P^T A P; the coarsest matrix is solved by dense Cholesky.
Cycle: V(1,1) with l1-Jacobi, d_i = sum_j |a_ij|, zero initial guess.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

THETA = 0.08
MAX_COARSE = 256
MAX_LEVELS = 10
POWER_ITS = 20


def strength(A):
    A = sp.csr_matrix(A)
    d = A.diagonal()
    strong = []
    for i in range(A.shape[0]):
        cols = A.indices[A.indptr[i]:A.indptr[i + 1]]
        vals = A.data[A.indptr[i]:A.indptr[i + 1]]
        s = [int(c) for c, v in zip(cols, vals)
             if c != i and abs(v) >= THETA * np.sqrt(abs(d[i] * d[c]))]
        strong.append(sorted(s))
    return strong


def aggregate(A):
    """Aggregate id of every node (int64 array) and the aggregate count."""
    n = A.shape[0]
    S = strength(A)
    agg = -np.ones(n, dtype=np.int64)
    na = 0
    for i in range(n):                                   # step 1
        if agg[i] < 0 and all(agg[j] < 0 for j in S[i]):
            agg[i] = na
            for j in S[i]:
                agg[j] = na
            na += 1
    after1 = agg.copy()
    for i in range(n):                                   # step 2
        if agg[i] < 0:
            for j in S[i]:
                if after1[j] >= 0:
                    agg[i] = after1[j]
                    break
    for i in range(n):                                   # step 3
        if agg[i] < 0:
            agg[i] = na
            for j in S[i]:
                if agg[j] < 0:
                    agg[j] = na
            na += 1
    return agg, na


def spectral_radius_dinv_a(A):
    A = sp.csr_matrix(A)
    dinv = 1.0 / A.diagonal()
    x = 1.0 + (np.arange(A.shape[0]) % 3).astype(np.float64)
    x /= np.linalg.norm(x)
    rho = 0.0
    for _ in range(POWER_ITS):
        y = dinv * (A @ x)
        rho = np.linalg.norm(y)
        x = y / rho
    return rho


class Level:
    def __init__(self, A):
        self.A = sp.csr_matrix(A)
        self.dl1 = np.asarray(abs(self.A).sum(axis=1)).ravel()
        self.P = None


def setup(A):
    levels = [Level(A)]
    while levels[-1].A.shape[0] > MAX_COARSE and len(levels) < MAX_LEVELS:
        Al = levels[-1].A
        agg, na = aggregate(Al)
        if na >= Al.shape[0]:
            break
        n = Al.shape[0]
        size = np.bincount(agg, minlength=na).astype(np.float64)
        Pt = sp.csr_matrix((1.0 / np.sqrt(size[agg]), (np.arange(n), agg)), shape=(n, na))
        omega = 4.0 / (3.0 * spectral_radius_dinv_a(Al))
        dinv = sp.diags(1.0 / Al.diagonal())
        P = (Pt - omega * (dinv @ (Al @ Pt))).tocsr()
        levels[-1].P = P
        levels.append(Level((P.T @ Al @ P).tocsr()))
    last = levels[-1]
    last.chol = sla.cho_factor(last.A.toarray(), lower=True)
    return levels


def vcycle(levels, B, lev=0):
    """One V(1,1) cycle from a zero guess on every column of B."""
    L = levels[lev]
    if lev == len(levels) - 1:
        return sla.cho_solve(L.chol, B)
    X = B / L.dl1[:, None]
    Rr = B - L.A @ X
    Xc = vcycle(levels, L.P.T @ Rr, lev + 1)
    X = X + L.P @ Xc
    X = X + (B - L.A @ X) / L.dl1[:, None]
    return X
