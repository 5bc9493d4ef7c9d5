"""The nonlinear stochastic Poisson problem with a quadratic conductivity
and its Newton iteration (Sec. 2.2, Eqs. NLP_StrongPDE, stonlp_system,
vectorvalPDENL, AjkTkl, with the conductivity (1 + u^2) in place of the
paper's (1 + alpha u)):

    -div( k(x, xi) (1 + u(x, xi)^2) grad u(x, xi) ) = 1,   u = 0 on the boundary,

k the lognormal field of the linear problem.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Discretisation (the readings of the Picard oracle in ``nonlinear.py``, with
u^2 in place of u): P1 in space, piecewise constant coefficients; inside
element e the solution enters the conductivity through its element average
ubar_e (mean of the three vertex values, zero at Dirichlet vertices), and
its square is projected onto the output chaos by the triple products,

    w_e = Pi_p[ubar_e^2],   w_{e,f} = sum_{a,b} ubar_{e,a} ubar_{e,b} <psi_a psi_b psi_f>,

so the element conductivity is k_e(xi) (1 + sum_f w_{e,f} psi_f) and its
Galerkin matrix is

    B_e[l, m] = sum_i cbar_i(e) <psi_i psi_l psi_m> + sum_{i,f} cbar_i(e) w_{e,f} <psi_i psi_f psi_l psi_m>.

Residual: R(U) = F - sum_e (K_e kron B_e(U)) U (K_e the unit P1 element
stiffness).  Newton: J(U) dU = R(U), U <- U + dU, with
J(U) = M(U) + D(U), M(U) = sum_e K_e kron B_e(U) and D(U) the derivative of
B_e(U) through w_e:

    D(U) dU |_{(r,l)} = sum_e sum_c K_e[r,c] sum_m dB_e[l,m] U_{c,m},
    dB_e = sum_{i,f} cbar_i(e) dw_{e,f} T_if,   dw_{e,f} = 2 sum_{a,b} ubar_{e,a} dubar_{e,b} <psi_a psi_b psi_f>,

and dubar_e the element average of dU.  The stopping rule is the relative
update ||dU|| / ||U|| <= tol.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem, galerkin, nonlinear, pce


def _vertices(N):
    el = fem.elements(N)
    return fem.interior_index(N, el[:, :, 0], el[:, :, 1])          # [E, 3], -1 on the boundary


def square_triples(L, p):
    """m[a, b, f] = <psi_a psi_b psi_f> with a, b, f in the output set."""
    return pce.galerkin_matrices(L, p, p)


def square_projection(ubar, m3):
    """w_e = Pi_p[ubar_e^2] for every element (ubar [E, P] -> w [E, P])."""
    return np.einsum("ea,eb,abf->ef", ubar, ubar, m3)


class Problem:
    """The nonlinear SG system on a linear problem's setup (mesh, KL modes,
    chaos sets, lognormal coefficients) with the fourfold products."""

    def __init__(self, prob):
        self.prob = prob
        self.t4 = nonlinear.four_products(prob.L, prob.p, prob.q)    # [K, P, P, P]
        self.m3 = square_triples(prob.L, prob.p)                      # [P, P, P]
        self.G = prob.G()                                             # [K, P, P]
        self.vert = _vertices(prob.N)
        self.Ke = [fem.p1_stiffness(np.array(t, dtype=np.float64)) for t in (fem.LOWER, fem.UPPER)]

    def ubar(self, U):
        return nonlinear.element_average(self.prob.N, U)

    def element_matrices(self, U):
        """B_e(U) for every element, [E, P, P]."""
        c = self.prob.cbar                                            # [K, E]
        w = square_projection(self.ubar(U), self.m3)                  # [E, P]
        B = np.einsum("ie,ilm->elm", c, self.G)
        B += np.einsum("ie,ef,iflm->elm", c, w, self.t4)
        return B

    def _scatter(self, blocks):
        """sum_e K_e kron blocks[e] as a sparse matrix in the mode-major
        unknown order ((l, r) at l n + r), blocks [E, P, P]."""
        prob = self.prob
        n, P = prob.n, prob.P
        rows, cols, vals = [], [], []
        for e in range(len(self.vert)):
            Ke = self.Ke[e % 2]
            for i in range(3):
                r = self.vert[e, i]
                if r < 0:
                    continue
                for j in range(3):
                    s = self.vert[e, j]
                    if s < 0 or Ke[i, j] == 0.0:
                        continue
                    blk = Ke[i, j] * blocks[e]
                    li, mi = np.nonzero(blk)
                    rows.append(li * n + r)
                    cols.append(mi * n + s)
                    vals.append(blk[li, mi])
        if not rows:
            return sp.csr_matrix((n * P, n * P))
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(n * P, n * P))

    def operator(self, U):
        """M(U) = sum_e K_e kron B_e(U) (sparse, mode-major order)."""
        return self._scatter(self.element_matrices(U))

    def residual(self, U, F=None):
        F = self.prob.rhs() if F is None else F
        r = galerkin.to_vec(F) - self.operator(U) @ galerkin.to_vec(U)
        return galerkin.from_vec(r, self.prob.n, self.prob.P)

    def derivative(self, U):
        """D(U): the derivative of B_e(U) applied to U, as a sparse matrix.
        Column (s, b): dU = unit vector at node s, mode b; its element
        average is 1/3 at the elements around s, so
        D[(r,l),(s,b)] = sum_{e containing r and s} (2/3) sum_c K_e[r,c]
                          sum_m (sum_{i,f} cbar_i(e) (sum_a ubar_{e,a} m_{abf}) t_{iflm}) U_{c,m}."""
        prob = self.prob
        n, P = prob.n, prob.P
        ub = self.ubar(U)                                             # [E, P]
        Upad = np.vstack([U, np.zeros((1, P))])
        rows, cols, vals = [], [], []
        for e in range(len(self.vert)):
            Ke = self.Ke[e % 2]
            vs = self.vert[e]
            if np.all(vs < 0):
                continue
            # d w_f / d ubar_b = 2 sum_a ubar_a m_{abf}
            dw = 2.0 * np.einsum("a,abf->bf", ub[e], self.m3)          # [b, f]
            # dB[l, m] per unit dubar_b: sum_{i,f} cbar_i dw[b, f] t_{iflm}
            dB = np.einsum("i,bf,iflm->blm", prob.cbar[:, e], dw, self.t4)   # [b, l, m]
            Uc = Upad[np.where(vs >= 0, vs, n)]                       # [3, P] vertex values
            for i in range(3):
                r = vs[i]
                if r < 0:
                    continue
                phi = Ke[i] @ Uc                                      # sum_c K_e[r,c] U_c, [P]
                g = np.einsum("blm,m->lb", dB, phi)                   # [l, b]
                for j in range(3):
                    s = vs[j]
                    if s < 0:
                        continue
                    li, bi = np.nonzero(g)
                    rows.append(li * n + r)
                    cols.append(bi * n + s)
                    vals.append(g[li, bi] / 3.0)
        if not rows:
            return sp.csr_matrix((n * P, n * P))
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(n * P, n * P))

    def jacobian(self, U):
        return (self.operator(U) + self.derivative(U)).tocsr()


def newton(nl, tol=1e-10, max_it=30, F=None, U0=None):
    """Newton's method from U0 (default 0) with sparse direct linear solves.
    Returns (U [n, P], iterations, history of the relative update)."""
    prob = nl.prob
    U = np.zeros((prob.n, prob.P)) if U0 is None else np.array(U0, dtype=np.float64)
    hist = []
    for it in range(1, max_it + 1):
        R = galerkin.to_vec(nl.residual(U, F))
        dU = galerkin.from_vec(spla.spsolve(nl.jacobian(U).tocsc(), R), prob.n, prob.P)
        U = U + dU
        nu = np.linalg.norm(U)
        change = np.linalg.norm(dU) / nu if nu > 0 else 0.0
        hist.append(change)
        if change <= tol:
            return U, it, hist
    return U, max_it, hist


def deterministic_fixed_point(N, coef, tol=1e-13, max_it=500):
    """The deterministic problem -div(coef (1 + ubar^2) grad u) = 1 for one
    per-element coefficient field, by the fixed-point (Picard) iteration
    u <- A(coef (1 + ubar(u)^2))^{-1} b from u = 0 (a method independent of
    Newton's, used as a pin).  Returns (u [n], iterations)."""
    b = fem.load_vector(N)
    u = np.zeros((N - 1) ** 2)
    for it in range(1, max_it + 1):
        ub = nonlinear.element_average(N, u[:, None])[:, 0]
        A = fem.assemble(N, np.asarray(coef) * (1.0 + ub * ub)).tocsc()
        unew = spla.spsolve(A, b)
        change = np.linalg.norm(unew - u) / np.linalg.norm(unew)
        u = unew
        if change <= tol:
            return u, it
    return u, max_it
