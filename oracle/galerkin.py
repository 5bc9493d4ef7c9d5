"""The coupled Galerkin system of the linear SG Poisson problem and its plain
solution (Sec. 2.1, Eq. Galerkin_L_exp and the Kronecker remark after it).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Unknowns: X [n, P], column a = PCE coefficient a of u at every interior
node (orthonormal chaos).  Operator: A(X) = sum_k A_k X G_k^T with
G_k[a, b] = <psi_k psi_a psi_b>; right-hand side F = b e_0^T since
<psi_k> = delta_k0 and f = 1.  The vector form of A stacks the columns of X
(mode-major): vec(A(X)) = (sum_k G_k kron A_k) vec(X).
"""
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem, kl, pce


@dataclass
class Problem:
    N: int
    L: int
    p: int
    q: int
    P: int
    K: int
    n: int
    rowptr: np.ndarray      # int64 [n+1]
    colidx: np.ndarray      # int64 [nnz]
    vals: np.ndarray        # float64 [K, nnz]
    kab: np.ndarray         # int64 [T, 3]
    num: np.ndarray         # int64 [T]
    g: np.ndarray           # float64 [T]
    b: np.ndarray           # float64 [n]
    gfield: np.ndarray      # float64 [L, E]  g_i at element centroids
    cbar: np.ndarray        # float64 [K, E]

    def A(self, k):
        n = self.n
        return sp.csr_matrix((self.vals[k], self.colidx, self.rowptr), shape=(n, n))

    def G(self):
        G = np.zeros((self.K, self.P, self.P))
        G[self.kab[:, 0], self.kab[:, 1], self.kab[:, 2]] = self.g
        return G

    def rhs(self):
        F = np.zeros((self.n, self.P))
        F[:, 0] = self.b
        return F


def build(N, L, p, q, sigma2=0.3, bx=0.5, by=0.5, g0=0.0, user_modes=None):
    """Setup steps: mesh, KL modes at centroids, multi-indices, triple
    products, lognormal coefficients, shared-pattern A_k, load vector."""
    x, y = fem.centroids(N)
    if user_modes is not None:
        gfield = np.asarray(user_modes, dtype=np.float64).reshape(L, len(x))
    elif L > 0:
        gfield = kl.field_modes(sigma2, bx, by, L, x, y)
    else:
        gfield = np.zeros((0, len(x)))
    g0arr = np.full(len(x), float(g0))
    cbar = pce.lognormal_coefficients(g0arr, gfield, q) if L > 0 else np.exp(g0arr)[None, :]
    rowptr, colidx, vals = fem.assemble_all(N, cbar)
    kab, num, g = pce.triple_products(L, p, q)
    return Problem(N=N, L=L, p=p, q=q, P=pce.n_terms(L, p), K=pce.n_terms(L, q),
                   n=(N - 1) ** 2, rowptr=rowptr, colidx=colidx, vals=vals,
                   kab=kab, num=num, g=g, b=fem.load_vector(N), gfield=gfield, cbar=cbar)


def apply(prob, X):
    """Y = sum_k A_k X G_k^T  (X, Y of shape [n, P])."""
    G = prob.G()
    Y = np.zeros((prob.n, prob.P))
    for k in range(prob.K):
        Y += (prob.A(k) @ X) @ G[k].T
    return Y


def apply_rows(prob, X, rows):
    """y_r for selected rows only, from the entrywise definition
    y_r[a] = sum_{c in row r} sum_{(k,a,b)} v_k^{rc} g_kab x_c[b]."""
    out = np.zeros((len(rows), prob.P))
    k, a, b = prob.kab[:, 0], prob.kab[:, 1], prob.kab[:, 2]
    for i, r in enumerate(rows):
        for t in range(prob.rowptr[r], prob.rowptr[r + 1]):
            c = prob.colidx[t]
            np.add.at(out[i], a, prob.vals[k, t] * prob.g * X[c, b])
    return out


def assembled(prob):
    """The full matrix sum_k G_k kron A_k (mode-major unknown order)."""
    G = prob.G()
    M = None
    for k in range(prob.K):
        if not np.any(G[k]):
            continue
        term = sp.kron(sp.csr_matrix(G[k]), prob.A(k), format="csr")
        M = term if M is None else M + term
    return M.tocsr()


def to_vec(X):
    return np.asarray(X).T.reshape(-1)


def from_vec(v, n, P):
    return np.asarray(v).reshape(P, n).T


def solve_direct(prob, F=None):
    """Sparse direct solve of the assembled system (small cases)."""
    F = prob.rhs() if F is None else F
    M = assembled(prob).tocsc()
    x = spla.spsolve(M, to_vec(F))
    return from_vec(x, prob.n, prob.P)


def relres(prob, X, F=None):
    F = prob.rhs() if F is None else F
    return np.linalg.norm(F - apply(prob, X)) / np.linalg.norm(F)


def gmres(matvec, precond, f, tol=1e-12, restart=50, max_it=2000, x0=None):
    """Restarted right-preconditioned GMRES (Saad's algorithm with modified
    Gram-Schmidt and Givens rotations) on flat vectors.  Stops on the true
    residual.  Returns (x, iterations, history of estimated relres)."""
    nf = np.linalg.norm(f)
    x = np.zeros_like(f) if x0 is None else x0.copy()
    hist = []
    its = 0
    if nf == 0.0:
        return x, 0, hist
    while its < max_it:
        r = f - matvec(x)
        beta = np.linalg.norm(r)
        if beta / nf <= tol:
            break
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        gvec = np.zeros(restart + 1)
        gvec[0] = beta
        j_used = 0
        for j in range(restart):
            z = precond(V[j])
            Z.append(z)
            w = matvec(z)
            for i in range(j + 1):
                H[i, j] = np.dot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            hnext = H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            gvec[j + 1] = -sn[j] * gvec[j]
            gvec[j] = cs[j] * gvec[j]
            its += 1
            j_used = j + 1
            hist.append(abs(gvec[j + 1]) / nf)
            if abs(gvec[j + 1]) / nf <= tol * 0.5 or its >= max_it or hnext == 0.0:
                break
            V.append(w / hnext)
        yv = np.linalg.solve(np.triu(H[:j_used, :j_used]), gvec[:j_used])
        for i in range(j_used):
            x = x + yv[i] * Z[i]
    return x, its, hist


def mean_preconditioner(prob):
    """I kron A_0^{-1}: one sparse LU of the mean stiffness matrix applied to
    every PCE column (G_0 = I in the orthonormal basis)."""
    lu = spla.splu(prob.A(0).tocsc())

    def apply_pc(v):
        Xm = from_vec(v, prob.n, prob.P)
        return to_vec(lu.solve(np.ascontiguousarray(Xm)))
    return apply_pc


def solve_gmres(prob, F=None, tol=1e-12, restart=50, max_it=2000):
    """GMRES on the Galerkin system, right-preconditioned by I kron A_0^{-1}."""
    F = prob.rhs() if F is None else F
    mv = lambda v: to_vec(apply(prob, from_vec(v, prob.n, prob.P)))
    x, its, hist = gmres(mv, mean_preconditioner(prob), to_vec(F), tol, restart, max_it)
    return from_vec(x, prob.n, prob.P), its, hist
