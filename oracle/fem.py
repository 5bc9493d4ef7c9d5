"""Structured P1 finite elements on the unit square (Sec. 2.1; the paper's
element type is unstated, FreeFEM is used there).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Mesh: nodes (i h, j h), h = 1/N, i, j = 0..N.  Each cell (i, j) is split by
the "/" diagonal (i,j)-(i+1,j+1) into a lower triangle
[(i,j), (i+1,j), (i+1,j+1)] (element id 2 (j N + i)) and an upper triangle
[(i,j), (i+1,j+1), (i,j+1)] (element id 2 (j N + i) + 1).  Interior nodes
1..N-1 are numbered r = (j-1)(N-1) + (i-1).  Dirichlet u = 0 is imposed by
elimination (the boundary rows and columns are dropped).  The coefficient is
piecewise constant, evaluated at the element centroid.
"""
import numpy as np
import scipy.sparse as sp

LOWER = ((0, 0), (1, 0), (1, 1))
UPPER = ((0, 0), (1, 1), (0, 1))


def p1_stiffness(verts):
    """Unit-coefficient P1 element matrix of a triangle given by 3 vertices.

    Plain definition: K[i, j] = area * grad(lambda_i) . grad(lambda_j), with
    grad(lambda_i) = rot90(edge opposite i) / (2 area).  In 2D this matrix
    does not depend on the size of the triangle, so integer reference
    vertices give it exactly.
    """
    v = np.asarray(verts, dtype=np.float64)
    area2 = (v[1, 0] - v[0, 0]) * (v[2, 1] - v[0, 1]) - (v[2, 0] - v[0, 0]) * (v[1, 1] - v[0, 1])
    grads = np.empty((3, 2))
    for i in range(3):
        a, b = v[(i + 1) % 3], v[(i + 2) % 3]
        grads[i] = (a[1] - b[1], b[0] - a[0])
    grads /= area2
    return 0.5 * abs(area2) * grads @ grads.T


def elements(N):
    """Element connectivity as (i, j) grid coordinates, shape [2 N^2, 3, 2]."""
    out = np.empty((2 * N * N, 3, 2), dtype=np.int64)
    for j in range(N):
        for i in range(N):
            e = 2 * (j * N + i)
            out[e] = [(i + di, j + dj) for (di, dj) in LOWER]
            out[e + 1] = [(i + di, j + dj) for (di, dj) in UPPER]
    return out


def centroids(N):
    el = elements(N)
    h = 1.0 / N
    c = el.mean(axis=1) * h
    return c[:, 0], c[:, 1]


def interior_index(N, i, j):
    """Interior number of grid node (i, j), or -1 on the boundary."""
    i = np.asarray(i)
    j = np.asarray(j)
    inside = (i >= 1) & (i <= N - 1) & (j >= 1) & (j <= N - 1)
    return np.where(inside, (j - 1) * (N - 1) + (i - 1), -1)


def element_entries(N):
    """All element-matrix entries that couple two interior nodes.

    Returns (row, col, elem, kval): the interior numbers of the two nodes, the
    element id and the unit-coefficient entry K_e[a, b].
    """
    el = elements(N)
    Ks = np.stack([p1_stiffness(LOWER), p1_stiffness(UPPER)])
    E = len(el)
    idx = interior_index(N, el[:, :, 0], el[:, :, 1])          # [E, 3]
    a, b = np.meshgrid(np.arange(3), np.arange(3), indexing="ij")
    rows = idx[:, a.ravel()]                                   # [E, 9]
    cols = idx[:, b.ravel()]
    kval = Ks[np.arange(E) % 2][:, a.ravel(), b.ravel()]       # [E, 9]
    elem = np.repeat(np.arange(E), 9).reshape(E, 9)
    keep = (rows >= 0) & (cols >= 0)
    return rows[keep], cols[keep], elem[keep], kval[keep]


def assemble(N, coef):
    """Stiffness matrix of -div(coef grad u) on interior nodes (scipy CSR):
    A = sum_e coef_e K_e, summed entry by entry."""
    rows, cols, elem, kval = element_entries(N)
    n = (N - 1) ** 2
    A = sp.coo_matrix((np.asarray(coef)[elem] * kval, (rows, cols)), shape=(n, n)).tocsr()
    A.sum_duplicates()
    return A


def load_vector(N):
    """b_r = integral of phi_r (f = 1): sum over elements of area / 3."""
    el = elements(N)
    n = (N - 1) ** 2
    b = np.zeros(n)
    area = 0.5 / (N * N)
    idx = interior_index(N, el[:, :, 0], el[:, :, 1]).ravel()
    np.add.at(b, idx[idx >= 0], area / 3.0)
    return b


def shared_pattern(N, cbar0):
    """CSR pattern rule: the pattern of A_0 after elimination with exact zeros
    dropped, columns ascending.  Returns (rowptr, colidx) as int64."""
    A0 = assemble(N, cbar0)
    A0.eliminate_zeros()
    A0.sort_indices()
    return A0.indptr.astype(np.int64), A0.indices.astype(np.int64)


def assemble_all(N, cbar, k_chunk=16):
    """A_k for every input PCE term on the shared CSR pattern.

    Returns rowptr int64 [n+1], colidx int64 [nnz], values float64 [K, nnz].
    Every element entry lands on a pattern position; the entries that do not
    (the hypotenuse couplings) are exactly zero for every coefficient.
    """
    rowptr, colidx = shared_pattern(N, cbar[0])
    n = len(rowptr) - 1
    rows, cols, elem, kval = element_entries(N)
    pos_of = {}
    for r in range(n):
        for t in range(rowptr[r], rowptr[r + 1]):
            pos_of[(r, int(colidx[t]))] = t
    pos = np.array([pos_of.get((int(r), int(c)), -1) for r, c in zip(rows, cols)])
    assert np.all(kval[pos < 0] == 0.0)
    on = pos >= 0
    S = sp.csr_matrix((np.ones(on.sum()), (pos[on], np.arange(on.sum()))),
                      shape=(len(colidx), on.sum()))
    K = cbar.shape[0]
    vals = np.empty((K, len(colidx)))
    for k0 in range(0, K, k_chunk):
        contrib = cbar[k0:k0 + k_chunk][:, elem[on]] * kval[on][None, :]
        vals[k0:k0 + k_chunk] = (S @ contrib.T).T
    return rowptr, colidx, vals


def assemble_dirichlet_x(N, coef, u_left, u_right):
    """Oracle-only variant for the appendix problem (Eq. qunlc4 with m = 0):
    u = u_left at x = 0, u = u_right at x = 1, zero Neumann at y = 0, 1.
    Unknowns: nodes with 1 <= i <= N-1, 0 <= j <= N (numbered j (N-1) + i-1).
    Returns (A, rhs, node_i, node_j)."""
    el = elements(N)
    nu = (N - 1) * (N + 1)

    def idx_of(i, j):
        return -1 if (i == 0 or i == N) else j * (N - 1) + (i - 1)

    Klow = p1_stiffness(LOWER)
    Kup = p1_stiffness(UPPER)
    rows, cols, vals = [], [], []
    rhs = np.zeros(nu)
    for e in range(len(el)):
        Ke = Klow if e % 2 == 0 else Kup
        nodes = el[e]
        for a in range(3):
            ia = idx_of(*nodes[a])
            if ia < 0:
                continue
            for b in range(3):
                ib = idx_of(*nodes[b])
                if ib >= 0:
                    rows.append(ia)
                    cols.append(ib)
                    vals.append(coef[e] * Ke[a, b])
                else:
                    ub = u_left if nodes[b][0] == 0 else u_right
                    rhs[ia] -= coef[e] * Ke[a, b] * ub
    A = sp.coo_matrix((vals, (rows, cols)), shape=(nu, nu)).tocsr()
    ii = np.array([i for j in range(N + 1) for i in range(1, N)])
    jj = np.array([j for j in range(N + 1) for i in range(1, N)])
    return A, rhs, ii, jj


def load_vector_f(N, f):
    """b_r = integral f phi_r by the 3-point edge-midpoint rule per element
    (exact for quadratics), used for the O(h^2) convergence pin."""
    el = elements(N)
    h = 1.0 / N
    n = (N - 1) ** 2
    b = np.zeros(n)
    area = 0.5 * h * h
    for e in range(len(el)):
        pts = el[e] * h
        idx = interior_index(N, el[e, :, 0], el[e, :, 1])
        mids = [(pts[0] + pts[1]) / 2, (pts[1] + pts[2]) / 2, (pts[2] + pts[0]) / 2]
        # basis values at the midpoints: phi_a = 1/2 on the two edges touching a
        for a in range(3):
            if idx[a] < 0:
                continue
            acc = 0.0
            for m, (p0, p1) in enumerate([(0, 1), (1, 2), (2, 0)]):
                phi = 0.5 if a in (p0, p1) else 0.0
                acc += f(mids[m][0], mids[m][1]) * phi
            b[idx[a]] += area * acc / 3.0
    return b
