"""The paper's own preconditioner variants (Sec. 3 and Sec. 5): restricted
additive Schwarz with incomplete LU (zero fill) of the coupled local block
as the sub-solve, and the 2GV2 coarse solve (inner GMRES preconditioned by a
one-level RAS on the coarse grid, relative tolerance 1e-2, at most 100
iterations).  The library and the rest of the oracle use exact solves of the
local mean block instead (the stated deviation); these variants exist to
compare iteration counts with the paper's.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Readings:
* the coupled local block is R_i A R_i^T of the Galerkin matrix in the
  vector-PDE order the paper assembles (the P chaos coefficients of a node
  contiguous, nodes in ascending global index): sum_k A_{k,i} kron G_k;
* ILU(0) keeps exactly the sparsity pattern of that block (the structural
  pattern of the kron products, zeros included), eliminating in the
  natural order; no damping (the paper's RAS is undamped);
* the coarse-grid boxes of 2GV2 are the same S_x x S_y boxes of the coarse
  interior grid with the same overlap.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import galerkin, ras, twolevel


def ilu0(A):
    """Incomplete LU with zero fill of a square sparse matrix, computed
    densely: Gaussian elimination in the natural order in which every update
    a_ij -= l_ik u_kj outside the pattern of A is dropped.  Returns the
    combined factor (strict lower part: L without its unit diagonal; upper
    part: U) and the pattern mask."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    pat = np.zeros((n, n), dtype=bool)
    rows = np.repeat(np.arange(n), np.diff(A.indptr))
    pat[rows, A.indices] = True
    F = A.toarray()
    for k in range(n - 1):
        piv = F[k, k]
        below = np.nonzero(pat[k + 1:, k])[0] + k + 1
        if below.size == 0:
            continue
        F[below, k] /= piv
        right = np.nonzero(pat[k, k + 1:])[0] + k + 1
        if right.size == 0:
            continue
        upd = np.outer(F[below, k], F[k, right])
        mask = pat[np.ix_(below, right)]
        F[np.ix_(below, right)] -= np.where(mask, upd, 0.0)
    return F, pat


def ilu0_solve(F, b):
    """x = (L U)^{-1} b for the combined factor of ``ilu0`` (b may have
    several columns)."""
    y = sla.solve_triangular(F, b, lower=True, unit_diagonal=True)
    return sla.solve_triangular(F, y, lower=False)


def coupled_block(As, G, idx):
    """R_i (sum_k A_k kron-in-node-order G_k) R_i^T: node-major, P
    coefficients of a node contiguous."""
    M = None
    for Ak, Gk in zip(As, G):
        if not np.any(Gk):
            continue
        t = sp.kron(sp.csr_matrix(Ak)[idx][:, idx], sp.csr_matrix(Gk), format="csr")
        M = t if M is None else M + t
    return M.tocsr()


class CoupledRAS:
    """One-level RAS with ILU(0) of the coupled local blocks:
    z = sum_i R_i^T D_i (ILU0 of R_i A R_i^T)^{-1} R_i r."""

    def __init__(self, As, G, N, sx, sy, overlap):
        self.parts = ras.partitions(As[0], N, sx, sy, overlap)
        self.P = G.shape[1]
        self.factors = [ilu0(coupled_block(As, G, idx))[0] for idx, _ in self.parts]

    def apply(self, R):
        Z = np.zeros_like(R)
        P = self.P
        for (idx, owned), F in zip(self.parts, self.factors):
            loc = ilu0_solve(F, np.ascontiguousarray(R[idx]).reshape(-1)).reshape(len(idx), P)
            keep = owned.astype(bool)
            Z[idx[keep]] += loc[keep]
        return Z


class OneLevel:
    """The one-level RAS preconditioner of the fine problem (ILU(0) coupled
    sub-solves), as an object with ``apply`` for ``twolevel.fgmres``."""

    def __init__(self, prob, sx, sy, overlap):
        self.ras = CoupledRAS([prob.A(k) for k in range(prob.K)], prob.G(), prob.N, sx, sy, overlap)

    def apply(self, R):
        return self.ras.apply(R)


class TwoLevelPaper(twolevel.TwoLevel):
    """The paper's two-grid cycle with ILU(0) coupled RAS sub-solves (no
    damping) and the coarse problem solved exactly, by 2GV2 (inner GMRES +
    one-level coupled RAS on the coarse grid, rtol 1e-2, 100 iterations) or
    by 2GV3 (inner GMRES + the AMG V-cycle, the inherited coarse solve)."""

    def __init__(self, prob, sx, sy, overlap, coarse="2gv2", inner_rtol=None, inner_max=100):
        exact = coarse == "exact"
        rtol = inner_rtol if inner_rtol is not None else (1e-2 if coarse == "2gv2" else 1e-5)
        super().__init__(prob, sx, sy, overlap, exact_coarse=exact, inner_rtol=rtol, inner_max=inner_max,
                         omega=1.0)
        self.variant = coarse
        self.fine_ras = CoupledRAS([prob.A(k) for k in range(prob.K)], self.G, prob.N, sx, sy, overlap)
        if coarse == "2gv2":
            self.coarse_ras = CoupledRAS(self.Acs, self.G, prob.N // 2, sx, sy, overlap)

    def ras(self, Rm):
        return self.fine_ras.apply(Rm)

    def coarse_solve(self, Rc):
        if self.variant != "2gv2":
            return super().coarse_solve(Rc)
        from . import coarse
        n, P = self.nc, self.prob.P
        mv = lambda v: galerkin.to_vec(coarse.coarse_apply(self.Acs, self.G, galerkin.from_vec(v, n, P)))
        pc = lambda v: galerkin.to_vec(self.coarse_ras.apply(galerkin.from_vec(v, n, P)))
        x, its, _ = galerkin.gmres(mv, pc, galerkin.to_vec(Rc), tol=self.inner_rtol, restart=30,
                                   max_it=self.inner_max)
        self.inner_its.append(its)
        return galerkin.from_vec(x, n, P)
