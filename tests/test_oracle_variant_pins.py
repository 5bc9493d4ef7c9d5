"""Pins of the oracle's versions of the paper's own preconditioner variants
(Sec. 3 and Sec. 5): ILU(0) against its defining properties, and the
scalability the paper reports (Tab. ws_lp): one-level RAS iterations grow
with the number of subdomains at a fixed subdomain size, the two-level
variants' iterations do not."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import galerkin, twolevel, variants

pytestmark = pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")


def test_ilu0_reproduces_the_matrix_on_its_pattern():
    """(L U)_ij = a_ij for every (i, j) of A's pattern (the defining
    property of ILU(0)); entries outside the pattern are dropped fill."""
    A = sp.random(40, 40, density=0.15, random_state=3) + 6.0 * sp.eye(40)
    F, pat = variants.ilu0(A)
    L = np.tril(F, -1) + np.eye(40)
    U = np.triu(F)
    D = L @ U - A.toarray()
    assert np.max(np.abs(D[pat])) <= 1e-13 * np.max(np.abs(A.toarray()))
    assert np.any(np.abs(D[~pat]) > 1e-8)          # some fill was dropped
    assert not np.any(F[~pat])                      # nothing stored off the pattern


def test_ilu0_is_exact_without_fill():
    """A tridiagonal matrix has no fill: ILU(0) is its LU and solves exactly."""
    rng = np.random.default_rng(4)
    n = 50
    main = 4.0 + rng.random(n)
    off = -rng.random(n - 1)
    A = sp.diags([off, main, off], [-1, 0, 1], format="csr")
    F, _ = variants.ilu0(A)
    b = rng.standard_normal(n)
    x = variants.ilu0_solve(F, b)
    assert np.linalg.norm(A @ x - b) <= 1e-13 * np.linalg.norm(b)


def test_coupled_block_is_the_restricted_galerkin_matrix():
    """The node-major coupled block of one box equals the rows and columns
    of the assembled Galerkin matrix for that box's nodes, reordered."""
    prob = galerkin.build(12, 2, 2, 4, sigma2=0.3, bx=0.5, by=0.5)
    idx = np.array([3, 4, 5, 14, 15, 16, 25, 26, 27])
    B = variants.coupled_block([prob.A(k) for k in range(prob.K)], prob.G(), idx).toarray()
    M = galerkin.assembled(prob).toarray()         # mode-major
    n, P = prob.n, prob.P
    sel = (np.arange(P)[None, :] * n + idx[:, None]).reshape(-1)   # node-major selection
    assert np.allclose(B, M[np.ix_(sel, sel)], rtol=0, atol=1e-14 * np.max(np.abs(M)))


def test_two_level_iterations_do_not_grow_with_subdomains():
    """Subdomains of about 8 x 8 nodes on meshes 16^2, 32^2 and 64^2
    (2 x 2 to 8 x 8 boxes, overlap 1, L = 2, p = 2, sigma^2 = 0.3, FGMRES to
    1e-5 as in the paper): the one-level RAS with ILU(0) coupled sub-solves
    needs about twice the iterations per doubling of the boxes per
    direction, the two-level cycle with the 2GV3 coarse solve a constant
    count."""
    one, two = [], []
    for N, s in ((16, 2), (32, 4), (64, 8)):
        prob = galerkin.build(N, 2, 2, 4, sigma2=0.3, bx=0.5, by=0.5)
        _, its, _ = twolevel.fgmres(prob, variants.OneLevel(prob, s, s, 1), tol=1e-5, max_it=400)
        one.append(its)
        _, its, _ = twolevel.fgmres(prob, variants.TwoLevelPaper(prob, s, s, 1, coarse="2gv3"), tol=1e-5,
                                    max_it=400)
        two.append(its)
    print("one-level", one, "two-level 2GV3", two)
    assert all(b >= 1.7 * a for a, b in zip(one, one[1:]))
    assert max(two) - min(two) <= 1 and max(two) <= 8


@pytest.mark.parametrize("coarse", ["exact", "2gv2"])
def test_two_level_variants_converge_alike(coarse):
    """The exact and 2GV2 coarse solves give the same outer count as 2GV3
    on a 4 x 4-box problem (the coarse tolerance only matters at scale)."""
    prob = galerkin.build(32, 2, 2, 4, sigma2=0.3, bx=0.5, by=0.5)
    _, ref, _ = twolevel.fgmres(prob, variants.TwoLevelPaper(prob, 4, 4, 1, coarse="2gv3"), tol=1e-5)
    pc = variants.TwoLevelPaper(prob, 4, 4, 1, coarse=coarse)
    X, its, _ = twolevel.fgmres(prob, pc, tol=1e-5)
    assert abs(its - ref) <= 1
    assert galerkin.relres(prob, X) <= 1e-5
    if coarse == "2gv2":
        assert 0 < max(pc.inner_its) <= 100
