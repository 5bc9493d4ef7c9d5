"""Restricted additive Schwarz on the fine grid (Sec. 3, Eqs.
RASstofixedpoint and RASsto).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

  M_RAS^{-1} = sum_i R_i^T D_i (R_i A R_i^T)^{-1} R_i

Readings (the paper fixes none of these details):
* subdomains are Sx x Sy boxes of the interior node grid: node (i, j) is
  owned by box (floor((i-1) Sx / (N-1)), floor((j-1) Sy / (N-1))), id
  by * Sx + bx;
* the overlapped set of a box grows its owned set by `overlap` layers of the
  graph of A_0 (all neighbours of the current set, repeated);
* local order = ascending global index; D_i = 1 on owned nodes, 0 on the
  overlap, so sum_i R_i^T D_i R_i = I;
* the local solve is exact and uses the MEAN block: (I kron A_{0,i})^{-1}
  with A_{0,i} = R_i A_0 R_i^T (the paper's sub-solve is ILU on the coupled
  block; the mean-block exact solve is the stated deviation).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def owner_boxes(N, sx, sy):
    """Owning box id of every interior node (interior numbering)."""
    m = N - 1
    i = np.tile(np.arange(1, N), m)
    j = np.repeat(np.arange(1, N), m)
    bx = (i - 1) * sx // m
    by = (j - 1) * sy // m
    return by * sx + bx


def partitions(A0, N, sx, sy, overlap):
    """List of (idx, owned_flag) per box: idx ascending global indices of the
    overlapped set, owned_flag 1 where the node is owned by the box."""
    owner = owner_boxes(N, sx, sy)
    A0 = sp.csr_matrix(A0)
    out = []
    for box in range(sx * sy):
        member = owner == box
        for _ in range(overlap):
            grow = (A0 @ member.astype(np.float64)) != 0.0
            member = member | grow
        idx = np.nonzero(member)[0]
        out.append((idx.astype(np.int64), (owner[idx] == box).astype(np.int32)))
    return out


def local_solvers(A0, parts):
    A0 = sp.csr_matrix(A0)
    return [spla.splu(A0[idx][:, idx].tocsc()) for idx, _ in parts]


def apply_ras(parts, solvers, R):
    """z = sum_i R_i^T D_i (I kron A_{0,i})^{-1} R_i r for every column of R
    (R has shape [n, P])."""
    Z = np.zeros_like(R)
    for (idx, owned), lu in zip(parts, solvers):
        loc = lu.solve(np.ascontiguousarray(R[idx]))
        keep = owned.astype(bool)
        Z[idx[keep]] += loc[keep]
    return Z


def kronecker_factor(prob):
    """G~ = sum_k (tr(A_k^T A_0) / tr(A_0^T A_0)) G_k: the stochastic factor of
    the best Kronecker approximation G~ kron A_0 of the Galerkin matrix (the
    Kronecker-structure preconditioners the paper cites after
    Eq. Galerkin_L_exp)."""
    A0 = prob.A(0)
    den = A0.multiply(A0).sum()
    w = np.array([prob.A(k).multiply(A0).sum() / den for k in range(prob.K)])
    return np.einsum("k,kab->ab", w, prob.G())


def smoother_radius(prob, ras_apply, its=20):
    """Largest |eigenvalue| of M_RAS^{-1} A by power iteration from the
    seed-free start X[r, a] = 1 + (r + a) mod 3 (normalised)."""
    from . import galerkin
    X = 1.0 + (np.add.outer(np.arange(prob.n), np.arange(prob.P)) % 3).astype(np.float64)
    X /= np.linalg.norm(X)
    rho = 1.0
    for _ in range(its):
        Y = ras_apply(galerkin.apply(prob, X))
        rho = np.linalg.norm(Y)
        X = Y / rho
    return rho
