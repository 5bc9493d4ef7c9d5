"""Coarse space of the two-grid preconditioner (Sec. 3, Eq. coarse).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

A_c = R_0 A R_0^T with R_0^T the P1 interpolation from the nested 2h mesh
to the fine mesh (the text calls R_0^T fine-to-coarse; it interpolates
coarse to fine, which is how it is used here).  Written from the definition:
R_0^T[f, C] is the coarse hat function of node C evaluated at fine node f.
The 2h mesh uses the same "/" split, so the meshes are nested and the ratio
of fine to coarse nodes is about 4 (the paper's default ratio).
"""
import numpy as np
import scipy.sparse as sp


def coarse_hat(I, J, i, j):
    """Value at fine grid node (i, j) (coordinates (i h, j h)) of the P1 hat
    function of coarse node (I, J) on the 2h "/" mesh.  In units of the
    coarse spacing the point is (i/2, j/2), so the barycentric coordinates
    inside the containing coarse triangle are multiples of 1/2 and exact."""
    ci, cj = i // 2, j // 2
    u, v = i / 2 - ci, j / 2 - cj            # local coordinates in [0, 1)^2
    if u >= v:   # lower triangle (0,0), (1,0), (1,1)
        verts = [(ci, cj), (ci + 1, cj), (ci + 1, cj + 1)]
        lam = [1 - u, u - v, v]
    else:        # upper triangle (0,0), (1,1), (0,1)
        verts = [(ci, cj), (ci + 1, cj + 1), (ci, cj + 1)]
        lam = [1 - v, u, v - u]
    for (vi, vj), l in zip(verts, lam):
        if (vi, vj) == (I, J):
            return l
    return 0.0


def interpolation(N):
    """R_0^T as a scipy CSR matrix [n_fine, n_coarse] (interior nodes)."""
    assert N % 2 == 0, "the 2h coarse mesh needs an even N"
    Nc = N // 2
    m, mc = N - 1, Nc - 1
    rows, cols, vals = [], [], []
    for j in range(1, N):
        for i in range(1, N):
            f = (j - 1) * m + (i - 1)
            # candidate coarse nodes: corners of the containing coarse cell
            for J in range(max(1, j // 2 - 1), min(Nc - 1, j // 2 + 1) + 1):
                for I in range(max(1, i // 2 - 1), min(Nc - 1, i // 2 + 1) + 1):
                    w = coarse_hat(I, J, i, j)
                    if w != 0.0:
                        rows.append(f)
                        cols.append((J - 1) * mc + (I - 1))
                        vals.append(w)
    return sp.csr_matrix((vals, (rows, cols)), shape=(m * m, mc * mc))


def coarse_matrices(prob):
    """A_k^c = R_0 A_k R_0^T for every input term, and R_0^T."""
    RT = interpolation(prob.N)
    R = RT.T.tocsr()
    return [(R @ prob.A(k) @ RT).tocsr() for k in range(prob.K)], RT


def coarse_apply(Acs, G, Xc):
    """Coarse Galerkin operator sum_k A_k^c Xc G_k^T."""
    Y = np.zeros_like(Xc)
    for k, Ak in enumerate(Acs):
        if np.any(G[k]):
            Y += (Ak @ Xc) @ G[k].T
    return Y
