"""Pins of the oracle's preconditioner pieces (Sec. 3) against facts fixed
by their definitions and by closed forms (CPU only)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import amg, coarse, fem, galerkin, ras, twolevel


def laplacian5(m):
    T = 2 * np.eye(m) - np.eye(m, k=1) - np.eye(m, k=-1)
    return np.kron(np.eye(m), T) + np.kron(T, np.eye(m))


# ---------------------------------------------------------------- RAS (Eq. RASsto)

@pytest.mark.parametrize("N,sx,sy,ov", [(16, 2, 2, 1), (20, 3, 2, 2), (33, 4, 3, 2)])
def test_partition_of_unity_and_overlap_shape(N, sx, sy, ov):
    A0 = fem.assemble(N, np.ones(2 * N * N))
    parts = ras.partitions(A0, N, sx, sy, ov)
    n, m = (N - 1) ** 2, N - 1
    count = np.zeros(n, dtype=int)
    owner = ras.owner_boxes(N, sx, sy)
    for b, (idx, own) in enumerate(parts):
        count[idx[own == 1]] += 1
        assert np.all(np.diff(idx) > 0)
        # overlap = graph distance <= ov from the owned block; on the 5-point
        # grid graph that is the Manhattan distance to the owned rectangle
        oi, oj = np.nonzero((owner == b).reshape(m, m).T)
        i, j = idx % m, idx // m
        di = np.maximum(0, np.maximum(oi.min() - i, i - oi.max()))
        dj = np.maximum(0, np.maximum(oj.min() - j, j - oj.max()))
        assert np.all(di + dj <= ov)
        ii, jj = np.meshgrid(np.arange(m), np.arange(m), indexing="ij")
        d_all = (np.maximum(0, np.maximum(oi.min() - ii, ii - oi.max()))
                 + np.maximum(0, np.maximum(oj.min() - jj, jj - oj.max())))
        assert (d_all <= ov).sum() == len(idx)
    assert np.all(count == 1)          # sum_i R_i^T D_i R_i = I


def test_ras_one_box_is_exact_inverse_at_sigma_zero():
    prob = galerkin.build(12, 2, 2, 4, sigma2=0.0)
    parts = ras.partitions(prob.A(0), 12, 1, 1, 0)
    sol = ras.local_solvers(prob.A(0), parts)
    R = np.random.default_rng(0).standard_normal((prob.n, prob.P))
    Z = ras.apply_ras(parts, sol, R)
    assert np.max(np.abs(galerkin.apply(prob, Z) - R)) < 1e-12 * np.max(np.abs(R))


def test_kronecker_factor_limits():
    prob0 = galerkin.build(10, 2, 2, 4, sigma2=0.0)
    assert np.allclose(ras.kronecker_factor(prob0), np.eye(prob0.P), atol=1e-15)
    # one constant mode: A_k = c_k A_unit, so G~ kron A_0 equals the Galerkin matrix
    N, p, gam = 10, 3, 0.35
    prob = galerkin.build(N, 1, p, 2 * p, user_modes=np.full((1, 2 * N * N), gam))
    Gt = ras.kronecker_factor(prob)
    M = sp.kron(sp.csr_matrix(Gt), prob.A(0)).toarray()
    assert np.max(np.abs(M - galerkin.assembled(prob).toarray())) < 1e-12 * np.max(np.abs(M))


# ------------------------------------------------------------ coarse space (Eq. coarse)

@pytest.mark.parametrize("N", [8, 16, 30])
def test_galerkin_coarse_operator_is_2h_stiffness(N):
    """For c = 1, R_0 A_h R_0^T is exactly the stiffness matrix of the 2h mesh
    (nested P1 spaces), i.e. the 5-point Laplacian of (N/2 - 1)^2 nodes."""
    RT = coarse.interpolation(N)
    Ah = fem.assemble(N, np.ones(2 * N * N))
    Ac = (RT.T @ Ah @ RT).toarray()
    assert np.array_equal(Ac, laplacian5(N // 2 - 1))


def test_interpolation_reproduces_linear_functions():
    N = 16
    RT = coarse.interpolation(N)
    Nc, m, mc = N // 2, N - 1, N // 2 - 1
    g = lambda x, y: 1.0 + 2.0 * x - 3.0 * y
    I, J = np.meshgrid(np.arange(1, Nc), np.arange(1, Nc), indexing="xy")
    gc = g(I.ravel() / Nc, J.ravel() / Nc)
    gf = RT @ gc
    i, j = np.meshgrid(np.arange(1, N), np.arange(1, N), indexing="xy")
    i, j = i.ravel(), j.ravel()
    inner = (i >= 2) & (i <= N - 2) & (j >= 2) & (j <= N - 2)   # coarse triangle fully interior
    assert np.max(np.abs(gf[inner] - g(i[inner] / N, j[inner] / N))) < 1e-14
    assert RT.shape == (m * m, mc * mc)


# ---------------------------------------------------------------------- AMG

def test_aggregation_invariants_and_tentative_prolongator():
    N = 40
    prob = galerkin.build(N, 2, 1, 2, sigma2=0.3, bx=0.3, by=0.3)
    Acs, RT = coarse.coarse_matrices(prob)
    A = Acs[0]
    agg, na = amg.aggregate(A)
    assert agg.min() == 0 and agg.max() == na - 1 and len(np.unique(agg)) == na
    S = amg.strength(A)
    for a in range(na):                      # aggregates are connected in the strength graph
        nodes = set(np.nonzero(agg == a)[0].tolist())
        start = next(iter(nodes))
        seen, stack = {start}, [start]
        while stack:
            u = stack.pop()
            for v in S[u]:
                if v in nodes and v not in seen:
                    seen.add(v)
                    stack.append(v)
        assert seen == nodes
    size = np.bincount(agg).astype(float)
    Pt = sp.csr_matrix((1 / np.sqrt(size[agg]), (np.arange(len(agg)), agg)))
    assert np.allclose((Pt.T @ Pt).toarray(), np.eye(na), atol=1e-15)


def test_vcycle_is_a_convergent_spd_preconditioner():
    N = 48
    prob = galerkin.build(N, 2, 1, 2, sigma2=0.3, bx=0.5, by=0.5)
    A = coarse.coarse_matrices(prob)[0][0]
    levels = amg.setup(A)
    assert len(levels) >= 2 and levels[-1].A.shape[0] <= amg.MAX_COARSE
    n = A.shape[0]
    Bm = amg.vcycle(levels, np.eye(n))
    assert np.max(np.abs(Bm - Bm.T)) < 1e-12 * np.max(np.abs(Bm))        # symmetric
    ev = np.linalg.eigvals(np.eye(n) - Bm @ A.toarray())
    assert np.max(np.abs(ev)) < 0.9                                        # contraction
    small = amg.setup(fem.assemble(8, np.ones(128)))
    assert len(small) == 1                                                 # exact coarsest solve
    b = np.random.default_rng(2).standard_normal((49, 3))
    assert np.allclose(fem.assemble(8, np.ones(128)) @ amg.vcycle(small, b), b, atol=1e-12)


# -------------------------------------------------------------- two-level (Eq. RAS_2L)

def test_two_level_cycle_equals_expanded_formula():
    """B from the three-step cycle equals M P + (I - Q A) M + Q - M P A M with
    P = I - A Q (the reading of Eq. RAS_2L), and I - B A factors as
    (I - M A)(I - Q A)(I - M A)."""
    prob = galerkin.build(8, 1, 2, 4, sigma2=0.3, bx=0.5, by=0.5)
    tl = twolevel.TwoLevel(prob, 2, 2, 1, exact_coarse=True, omega=0.7)
    n, P = prob.n, prob.P
    N = n * P
    cols = lambda f: np.stack([galerkin.to_vec(f(galerkin.from_vec(e, n, P))) for e in np.eye(N)], axis=1)
    A = galerkin.assembled(prob).toarray()
    M = cols(lambda R: tl.omega * tl.ras(R))
    Q = cols(lambda R: tl.RT @ tl.coarse_solve(tl.R @ R))
    B = cols(tl.apply)
    I = np.eye(N)
    Pm = I - A @ Q
    ref = M @ Pm + (I - Q @ A) @ M + Q - M @ Pm @ A @ M
    assert np.max(np.abs(B - ref)) < 1e-12 * np.max(np.abs(B))
    E = (I - M @ A) @ (I - Q @ A) @ (I - M @ A)
    assert np.max(np.abs((I - B @ A) - E)) < 1e-11
    # Q A is the A-orthogonal projection onto the coarse space
    assert np.max(np.abs(Q @ A @ Q @ A - Q @ A)) < 1e-11


def test_two_level_fgmres_converges():
    prob = galerkin.build(32, 2, 2, 4, sigma2=0.3, bx=0.5, by=0.5)
    tl = twolevel.TwoLevel(prob, 2, 2, 1, exact_coarse=False)
    X, its, hist = twolevel.fgmres(prob, tl, tol=1e-8)
    Xd = galerkin.solve_direct(prob)
    assert galerkin.relres(prob, X) <= 1e-8 and its < 40
    assert np.linalg.norm(X - Xd) / np.linalg.norm(Xd) < 1e-7
