"""Two-level multiplicative RAS preconditioner (Sec. 3, Eq. RAS_2L) and the
outer flexible GMRES.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The printed formula contains "Q P Q^{-1} M^{-1}", which cannot be meant
literally (Q is singular); it is read as (I - Q A) M^{-1}, so that

  B = M^{-1} P + (I - Q A) M^{-1} + Q - M^{-1} P A M^{-1},  P = I - A Q,

which is exactly the pre-smooth / coarse / post-smooth cycle the text
describes:  z1 = M^{-1} r;  z2 = z1 + Q (r - A z1);  z = z2 + M^{-1}(r - A z2).
Q = R_0^T A_c^{-1} R_0; A_c^{-1} is applied either exactly (pins) or by an
inner GMRES (the 2GV3 variant: rtol 1e-5, at most 100 iterations)
preconditioned by the AMG V-cycle on the coarse mean operator combined with
the stochastic Kronecker factor, (G~^{-1} kron V-cycle).
"""
import numpy as np
import scipy.sparse.linalg as spla

from . import amg, coarse, galerkin, ras


class TwoLevel:
    def __init__(self, prob, sx, sy, overlap, exact_coarse=False, inner_rtol=1e-5, inner_max=100,
                 local="kron", omega=None):
        self.prob = prob
        self.G = prob.G()
        A0 = prob.A(0)
        self.parts = ras.partitions(A0, prob.N, sx, sy, overlap)
        self.solvers = ras.local_solvers(A0, self.parts)
        self.Gk_inv = np.linalg.inv(ras.kronecker_factor(prob))
        self.Gt_inv = self.Gk_inv if local == "kron" else None
        self.Acs, self.RT = coarse.coarse_matrices(prob)
        self.R = self.RT.T.tocsr()
        self.nc = self.RT.shape[1]
        self.exact = exact_coarse
        self.inner_rtol, self.inner_max = inner_rtol, inner_max
        self.inner_its = []
        if exact_coarse:
            import scipy.sparse as sp
            M = None
            for k, Ak in enumerate(self.Acs):
                if np.any(self.G[k]):
                    t = sp.kron(sp.csr_matrix(self.G[k]), Ak, format="csr")
                    M = t if M is None else M + t
            self.coarse_lu = spla.splu(M.tocsc())
        else:
            self.levels = amg.setup(self.Acs[0])

        self.omega = 1.0
        if omega is None:
            self.omega = 1.0 / ras.smoother_radius(prob, self.ras)
        else:
            self.omega = omega

    def ras(self, Rm):
        Z = ras.apply_ras(self.parts, self.solvers, Rm)
        return Z if self.Gt_inv is None else Z @ self.Gt_inv

    def coarse_solve(self, Rc):
        n, P = self.nc, self.prob.P
        if self.exact:
            return galerkin.from_vec(self.coarse_lu.solve(galerkin.to_vec(Rc)), n, P)
        mv = lambda v: galerkin.to_vec(coarse.coarse_apply(self.Acs, self.G, galerkin.from_vec(v, n, P)))
        gk = self.Gk_inv
        pc = lambda v: galerkin.to_vec(amg.vcycle(self.levels, galerkin.from_vec(v, n, P)) @ gk)
        x, its, _ = galerkin.gmres(mv, pc, galerkin.to_vec(Rc), tol=self.inner_rtol,
                                   restart=30, max_it=self.inner_max)
        self.inner_its.append(its)
        return galerkin.from_vec(x, n, P)

    def apply(self, Rm):
        """z = B r for an [n, P] block r."""
        A = lambda X: galerkin.apply(self.prob, X)
        w = self.omega
        z = w * self.ras(Rm)
        r1 = Rm - A(z)
        z = z + self.RT @ self.coarse_solve(self.R @ r1)
        r2 = Rm - A(z)
        return z + w * self.ras(r2)


def fgmres(prob, pc, F=None, tol=1e-8, restart=30, max_it=500):
    """Flexible GMRES (right preconditioned, preconditioned vectors kept)."""
    F = prob.rhs() if F is None else F
    n, P = prob.n, prob.P
    mv = lambda v: galerkin.to_vec(galerkin.apply(prob, galerkin.from_vec(v, n, P)))
    pcv = lambda v: galerkin.to_vec(pc.apply(galerkin.from_vec(v, n, P)))
    x, its, hist = galerkin.gmres(mv, pcv, galerkin.to_vec(F), tol, restart, max_it)
    return galerkin.from_vec(x, n, P), its, hist
