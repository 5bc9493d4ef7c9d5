"""Setup artefacts and the Galerkin operator apply through the C ABI versus
the FP64 oracle (GPU)."""
import numpy as np
import pytest

from oracle import galerkin, pce
from sg_inputs import CONFIGS, random_block

pytestmark = pytest.mark.gpu


def setup_pair(N, L, p, q, sigma2=0.3, b=0.5, user_modes=None):
    import paper_2310_14649_gb300 as sg
    prob = sg.sg_setup(N, L, p, q, sigma2=sigma2, bx=b, by=b, user_modes=user_modes)
    ref = galerkin.build(N, L, p, q, sigma2=sigma2, bx=b, by=b, user_modes=user_modes)
    return prob, ref


def to_dev(X, dtype, ld=None):
    import torch
    n, P = X.shape
    ld = ld or n
    out = torch.zeros((P, ld), dtype=dtype, device="cuda")
    out[:, :n] = torch.from_numpy(np.ascontiguousarray(X.T)).to(dtype)
    return out


def from_dev(Y, n):
    return Y[:, :n].double().cpu().numpy().T


def bound_and_terms(ref, X):
    """|A||X| elementwise (the oracle applied to absolute values) and the
    largest number of products summed into one output entry."""
    absprob = galerkin.Problem(**{**ref.__dict__, "vals": np.abs(ref.vals), "g": np.abs(ref.g)})
    Yb = galerkin.apply(absprob, np.abs(X))
    per_a = np.bincount(ref.kab[:, 1], minlength=ref.P).max()
    row_len = np.diff(ref.rowptr).max()
    return Yb, int(per_a * row_len)


def gamma(m, u):
    """Deterministic rounding bound gamma_m = m u / (1 - m u) for a sum of m
    products whose factors carry at most 3 extra roundings (value, g, x)."""
    m = m + 3
    return m * u / (1 - m * u)


U64, U32 = 2.0 ** -53, 2.0 ** -24


# integer artefacts must match the oracle bit for bit
@pytest.mark.parametrize("N,L,p,q", [(32, 2, 2, 4), (20, 3, 2, 4), (17, 1, 3, 6), (64, 4, 3, 6)])
def test_integer_artefacts_bit_exact(gpu, N, L, p, q):
    import paper_2310_14649_gb300 as sg
    prob, ref = setup_pair(N, L, p, q)
    assert (prob.n, prob.P, prob.K, prob.nnzA, prob.T) == (ref.n, ref.P, ref.K, len(ref.colidx), len(ref.g))
    assert np.array_equal(sg.sg_get_multi_indices(prob, 0), pce.multi_indices(L, p))
    assert np.array_equal(sg.sg_get_multi_indices(prob, 1), pce.multi_indices(L, q))
    kab, num, g = sg.sg_get_triples(prob)
    assert np.array_equal(kab, ref.kab) and np.array_equal(num, ref.num)
    assert np.max(np.abs(g - ref.g) / np.abs(ref.g)) < 4 * U64
    rowptr, colidx = sg.sg_get_csr(prob)
    assert np.array_equal(rowptr, ref.rowptr) and np.array_equal(colidx, ref.colidx)


# b = 0.3 and 0.35 have exactly tied 2D eigenvalues whose order must not
# depend on the host's rounding
@pytest.mark.parametrize("N,L,p,q,s2,b", [(32, 2, 2, 4, 0.3, 0.5), (24, 3, 2, 4, 0.5, 0.2), (32, 3, 2, 4, 0.3, 0.3),
                                         (32, 2, 2, 4, 0.3, 0.35)])
def test_stiffness_values(gpu, N, L, p, q, s2, b):
    import paper_2310_14649_gb300 as sg
    prob, ref = setup_pair(N, L, p, q, s2, b)
    vals = sg.sg_get_values(prob)
    scale = np.abs(ref.vals[0]).max()
    assert np.max(np.abs(vals - ref.vals)) < 1e-13 * scale


def check_apply(prob, ref, X, dtype, ld=None, kernel=0, fp64=1):
    """fp64: 1 keeps FP64 applies on the selected kernel, 2 on the
    assembled edge blocks."""
    import torch
    import paper_2310_14649_gb300 as sg
    sg.sg_set_apply_kernel(prob, kernel)
    sg.sg_set_apply_fp64(prob, fp64)
    Xd = to_dev(X, dtype, ld)
    Yd = torch.full_like(Xd, float("nan"))
    sg.sg_apply(prob, Xd, Yd)
    torch.cuda.synchronize()
    Xq = from_dev(Xd, ref.n)           # the inputs the kernel actually saw
    Yref = galerkin.apply(ref, Xq)
    Yb, m = bound_and_terms(ref, Xq)
    u = U64 if dtype == torch.float64 else U32
    err = np.abs(from_dev(Yd, ref.n) - Yref)
    assert np.all(err <= gamma(m, u) * Yb + 1e-300), (err / np.maximum(Yb, 1e-300)).max()
    return Yd


@pytest.mark.parametrize("dt", ["f64", "f64-shared", "f64-asm", "f32", "f32-shared"])
@pytest.mark.parametrize("N,L,p,q", [(32, 2, 2, 4), (33, 3, 3, 6), (2, 2, 1, 2), (9, 0, 0, 0), (40, 1, 5, 10)])
def test_apply_vs_oracle(gpu, dt, N, L, p, q):
    """Register-specialised, shared-memory and (FP64) assembled-block
    kernels, FP64 and FP32, each against the oracle within the
    deterministic rounding bound."""
    import torch
    import paper_2310_14649_gb300 as sg
    dtype = torch.float64 if dt.startswith("f64") else torch.float32
    kernel = 1 if dt.endswith("shared") else 2
    fp64 = 2 if dt.endswith("asm") else 1
    prob, ref = setup_pair(N, L, p, q)
    X = random_block(ref.n, ref.P, seed=3)
    check_apply(prob, ref, X, dtype, kernel=kernel, fp64=fp64)
    assert sg.sg_apply_fp64_info(prob)["fine"] == (fp64 == 2)
    # ragged leading dimension and a second, different input
    check_apply(prob, ref, random_block(ref.n, ref.P, seed=4), dtype, ld=ref.n + 37, kernel=kernel, fp64=fp64)


@pytest.mark.parametrize("fp64", [1, 2])
def test_residual_in_place(gpu, fp64):
    import torch
    import paper_2310_14649_gb300 as sg
    prob, ref = setup_pair(32, 2, 2, 4)
    sg.sg_set_apply_fp64(prob, fp64)
    X = random_block(ref.n, ref.P, seed=8)
    F = random_block(ref.n, ref.P, seed=9)
    Xd, Fd = to_dev(X, torch.float64), to_dev(F, torch.float64)
    sg.sg_residual(prob, Fd, Xd, Fd)
    torch.cuda.synchronize()
    assert sg.sg_apply_fp64_info(prob)["fine"] == (fp64 == 2)
    R = from_dev(Fd, ref.n)
    Rref = F - galerkin.apply(ref, X)
    Yb, m = bound_and_terms(ref, X)
    assert np.all(np.abs(R - Rref) <= gamma(m + 1, U64) * (Yb + np.abs(F)))


@pytest.mark.parametrize("N,L,p,q", [(32, 2, 2, 4), (33, 3, 3, 6), (2, 2, 1, 2), (9, 0, 0, 0), (40, 1, 5, 10),
                                     (12, 5, 3, 2), (12, 4, 4, 2), (10, 3, 7, 2)])
def test_refine_residual_double_fp32(gpu, N, L, p, q):
    """The refinement residual over the double-FP32 edge blocks against the
    FP64 oracle: within 2^-40 of |A||X| + |F| (FP32 alone gives 2^-24),
    ragged leading dimension, F == R in place, and the policy switch back
    to the FP64 apply.  P = 56, 70 and 120 take the kernels with 8, 11 and
    16 outputs per warp (P up to 64, 88 and 128)."""
    import torch
    import paper_2310_14649_gb300 as sg
    prob, ref = setup_pair(N, L, p, q)
    sg.sg_set_refine_residual(prob, 2)
    info = sg.sg_refine_residual_info(prob)
    npair = ref.P * (ref.P + 1) // 2
    assert info["built"] == 1 and info["bytes"] >= npair * 2 * N * (N - 1) * 8
    X = random_block(ref.n, ref.P, seed=5)
    F = random_block(ref.n, ref.P, seed=6)
    Rref = F - galerkin.apply(ref, X)
    Yb, m = bound_and_terms(ref, X)
    bound = (2.0 ** -40 + gamma(m + 1, U64)) * (Yb + np.abs(F))
    for ld in (ref.n, ref.n + 37):
        Xd, Fd = to_dev(X, torch.float64, ld), to_dev(F, torch.float64, ld)
        Rd = torch.full_like(Fd, 7.0)
        sg.sg_residual_refine(prob, Fd, Xd, Rd)
        torch.cuda.synchronize()
        R = from_dev(Rd, ref.n)
        assert np.all(np.abs(R - Rref) <= bound)
        assert torch.all(Rd[:, ref.n:] == 7.0)  # padding rows untouched
        sg.sg_residual_refine(prob, Fd, Xd, Fd)
        torch.cuda.synchronize()
        assert np.array_equal(from_dev(Fd, ref.n), R)
    sg.sg_set_refine_residual(prob, 1)
    assert sg.sg_refine_residual_info(prob)["built"] == 0
    Xd, Fd = to_dev(X, torch.float64), to_dev(F, torch.float64)
    sg.sg_residual_refine(prob, Fd, Xd, Fd)
    torch.cuda.synchronize()
    assert np.all(np.abs(from_dev(Fd, ref.n) - Rref) <= gamma(m + 1, U64) * (Yb + np.abs(F)))


def test_refine_residual_full_size_sampled_rows(gpu):
    """256x256 mesh, L=4, p=3 (P=35), q=6 (K=210), the bench's launch:
    sampled rows of the double-FP32 refinement residual against the
    entrywise oracle definition, for a random iterate and for a smooth one
    (the FP64 solution of the mean problem) whose residual is small."""
    import torch
    import paper_2310_14649_gb300 as sg
    c = CONFIGS["poisson256_L4_p3"]
    prob, ref = setup_pair(c["N"], c["L"], c["p"], c["q"], c["sigma2"], c["b"])
    rows = np.unique(np.concatenate([[0, 1, ref.n - 1, ref.n // 2],
                                     np.random.default_rng(1).integers(0, ref.n, 60)]))
    absref = galerkin.Problem(**{**ref.__dict__, "vals": np.abs(ref.vals), "g": np.abs(ref.g)})
    m = int(np.bincount(ref.kab[:, 1]).max() * 5)
    import scipy.sparse.linalg as spla
    smooth = np.zeros((ref.n, ref.P))
    smooth[:, 0] = spla.spsolve(ref.A(0).tocsc(), ref.b)
    F = ref.rhs()
    for X in (random_block(ref.n, ref.P, seed=22), smooth):
        Xd, Fd = to_dev(X, torch.float64), to_dev(F, torch.float64)
        Rd = torch.empty_like(Xd)
        sg.sg_residual_refine(prob, Fd, Xd, Rd)
        torch.cuda.synchronize()
        R = from_dev(Rd, ref.n)[rows]
        Rref = F[rows] - galerkin.apply_rows(ref, X, rows)
        Yb = galerkin.apply_rows(absref, np.abs(X), rows) + np.abs(F[rows])
        assert np.all(np.abs(R - Rref) <= (2.0 ** -40 + gamma(m, U64)) * Yb)
    assert sg.sg_refine_residual_info(prob)["built"] == 1


def test_rhs(gpu):
    import torch
    import paper_2310_14649_gb300 as sg
    prob, ref = setup_pair(16, 2, 2, 4)
    F = torch.full((ref.P, ref.n + 5), 7.0, dtype=torch.float64, device="cuda")
    sg.sg_get_rhs(prob, F)
    Fh = F.cpu().numpy()
    assert np.max(np.abs(Fh[0, :ref.n] - ref.b)) <= 4 * U64 * ref.b.max()
    assert np.all(Fh[1:] == 0) and np.all(Fh[0, ref.n:] == 0)


def test_apply_full_size_sampled_rows(gpu):
    """256x256 mesh, L=4, p=3 (P=35), q=6 (K=210): sampled output rows
    against the entrywise oracle definition, FP64 and FP32."""
    import torch
    import paper_2310_14649_gb300 as sg
    c = CONFIGS["poisson256_L4_p3"]
    prob, ref = setup_pair(c["N"], c["L"], c["p"], c["q"], c["sigma2"], c["b"])
    rows = np.unique(np.concatenate([[0, 1, ref.n - 1, ref.n // 2],
                                     np.random.default_rng(0).integers(0, ref.n, 60)]))
    X = random_block(ref.n, ref.P, seed=21)
    for dtype, u, kernel, fp64 in ((torch.float64, U64, 0, 2), (torch.float64, U64, 2, 1), (torch.float32, U32, 2, 1),
                                   (torch.float32, U32, 1, 1)):
        sg.sg_set_apply_kernel(prob, kernel)
        sg.sg_set_apply_fp64(prob, fp64)
        Xd = to_dev(X, dtype)
        Yd = torch.empty_like(Xd)
        sg.sg_apply(prob, Xd, Yd)
        torch.cuda.synchronize()
        Xq = from_dev(Xd, ref.n)
        Y = from_dev(Yd, ref.n)[rows]
        Yref = galerkin.apply_rows(ref, Xq, rows)
        absref = galerkin.Problem(**{**ref.__dict__, "vals": np.abs(ref.vals), "g": np.abs(ref.g)})
        Yb = galerkin.apply_rows(absref, np.abs(Xq), rows)
        m = int(np.bincount(ref.kab[:, 1]).max() * 5)
        assert np.all(np.abs(Y - Yref) <= gamma(m, u) * Yb)


def test_bad_arguments(gpu):
    import torch
    import paper_2310_14649_gb300 as sg
    prob, ref = setup_pair(8, 1, 1, 2)
    X = torch.zeros((ref.P, ref.n), dtype=torch.float64, device="cuda")
    with pytest.raises(sg.SgError) as e:
        sg.sg_apply(prob, X, X)          # aliasing input and output
    assert e.value.status == -1
    from paper_2310_14649_gb300 import _lib
    Y = torch.zeros_like(X)
    st = _lib.lib().sg_apply(prob.handle, 0, _lib.dev_ptr(X), ref.n - 1, _lib.dev_ptr(Y), ref.n, None)
    assert st == -1


@pytest.mark.parametrize("cfg", [(1, 1, 1, 1, 8, 1), (2, 1, 1, 1, 16, 1), (1, 2, 1, 1, 0, 2), (2, 3, 2, 1, 32, 1),
                                 (1, 4, 1, 2, 4, 1), (1, 2, 2, 2, 8, 1), (1, 1, 3, 1, 8, 1), (1, 1, 1, 4, 8, 1),
                                 (2, 1, 1, 8, 8, 1), (1, 1, 1, 1, 16, 1, 3), (1, 1, 1, 1, 5, 1, 4),
                                 (1, 1, 1, 1, 1, 1, 2), (1, 1, 1, 1, 32, 2, 4), (1, 1, 1, 1, 8, 1, 0, 3),
                                 (1, 1, 1, 1, 16, 1, 0, 5), (1, 1, 1, 5, 16, 1, 0, 1, 1), (2, 1, 1, 4, 8, 1, 0, 1, 2),
                                 (1, 2, 2, 2, 8, 1, 0, 1, 1)])
@pytest.mark.parametrize("N", [20, 21])
def test_specialised_kernel_configs(gpu, cfg, N):
    """Every tile shape (rows per thread, output groups, prefetch, CTAs per
    SM, values staged through shared memory) computes the same operator,
    for even and odd row counts."""
    import torch
    import paper_2310_14649_gb300 as sg
    prob, ref = setup_pair(N, 3, 3, 6)
    sg.sg_apply_config(prob, *cfg)
    check_apply(prob, ref, random_block(ref.n, ref.P, seed=12), torch.float32, kernel=2)
    check_apply(prob, ref, random_block(ref.n, ref.P, seed=13), torch.float32, kernel=2, ld=ref.n + 3)


@pytest.mark.parametrize("cfg", [(1, 1, 1, 1, 16, 1), (1, 2, 2, 1, 8, 1), (1, 1, 1, 4, 8, 1), (1, 4, 2, 1, 4, 1),
                                 (1, 2, 4, 1, 4, 1), (1, 1, 1, 1, 8, 1, 0, 4), (1, 1, 1, 5, 8, 1, 0, 1, 1),
                                 (1, 2, 1, 2, 8, 1, 0, 1, 2)])
@pytest.mark.parametrize("N", [20, 21])
def test_specialised_fp64_configs(gpu, cfg, N):
    """The FP64 family (exact double coefficients) in several tile shapes."""
    import torch
    import paper_2310_14649_gb300 as sg
    prob, ref = setup_pair(N, 3, 3, 6)
    sg.sg_apply_config(prob, *cfg, which=2)
    check_apply(prob, ref, random_block(ref.n, ref.P, seed=15), torch.float64, kernel=2)
    check_apply(prob, ref, random_block(ref.n, ref.P, seed=16), torch.float64, kernel=2, ld=ref.n + 5)
    with pytest.raises(sg.SgError):
        sg.sg_apply_config(prob, 2, 1, 1, 1, 8, 1, which=2)   # paired rows are FP32 only
    with pytest.raises(sg.SgError):
        sg.sg_apply_config(prob, 1, 2, 1, 1, 8, 1, 3)           # staging needs one group
    with pytest.raises(sg.SgError):
        sg.sg_apply_config(prob, 1, 1, 1, 2, 8, 1, 0, 1, 3)     # 1, 2 or 4 warps per group
    with pytest.raises(sg.SgError):
        sg.sg_apply_config(prob, 1, 1, 1, 1, 8, 1, 3, 1, 1)     # narrow groups are not staged


def test_autotune_picks_a_valid_shape(gpu):
    import torch
    import paper_2310_14649_gb300 as sg
    prob, ref = setup_pair(48, 2, 2, 4)
    ms = sg.sg_apply_autotune(prob, force=True)
    info = sg.sg_apply_info(prob)
    assert ms > 0 and info["rows"] in (1, 2) and 1 <= info["groups"] <= 4
    if sg.sg_apply_flux(prob, -1):     # the tuner chose the edge-flux form
        check_flux(prob, ref, random_block(ref.n, ref.P, seed=14).astype(np.float32).astype(np.float64))
    else:
        check_apply(prob, ref, random_block(ref.n, ref.P, seed=14), torch.float32, kernel=2)
    ms64 = sg.sg_apply_autotune(prob, force=True, which=2)
    assert ms64 > 0 and sg.sg_apply_info(prob, which=2)["rows"] == 1
    check_apply(prob, ref, random_block(ref.n, ref.P, seed=17), torch.float64, kernel=2)


@pytest.mark.parametrize("dt", ["f64", "f32"])
@pytest.mark.parametrize("nv,length", [(1, 1), (7, 1000), (32, 300001)])
def test_mdot(gpu, dt, nv, length):
    """Multi-vector dot products against numpy FP64 sums."""
    import torch
    import paper_2310_14649_gb300 as sg
    prob, ref = setup_pair(8, 1, 1, 2)
    dtype = torch.float64 if dt == "f64" else torch.float32
    g = torch.Generator().manual_seed(nv * 7 + length)
    V = torch.randn((nv, length + 5), generator=g, dtype=torch.float64).to(dtype).cuda()[:, :length]
    w = torch.randn(length, generator=g, dtype=torch.float64).to(dtype).cuda()
    out = torch.zeros(nv, dtype=torch.float64, device="cuda")
    for _ in range(2):
        sg.sg_mdot(prob, V, w, out)
    torch.cuda.synchronize()
    Vh, wh = V.double().cpu().numpy(), w.double().cpu().numpy()
    refv = Vh @ wh
    bound = np.abs(Vh) @ np.abs(wh)
    u = U64 if dt == "f64" else U32
    assert np.all(np.abs(out.cpu().numpy() - refv) <= gamma(8 if dt == "f32" else 1, u) * bound + 1e-12 * bound)


def flux_bound(ref, X):
    """Rounding scale of the edge-flux form: sum over the four edges of
    sum_k |w_k| |G_k| (|x_r| + |x_neighbour|), the conductances w_k of the
    oracle's element coefficients (half the sum over the two triangles of
    each edge), and the largest number of products summed into one output."""
    N, m, n = ref.N, ref.N - 1, ref.n
    c = ref.cbar                                              # [K, E]
    lo = c[:, 0::2].reshape(ref.K, N, N)                      # [k, j, i] lower triangle of cell (i, j)
    up = c[:, 1::2].reshape(ref.K, N, N)
    i = np.tile(np.arange(1, N), m)
    j = np.repeat(np.arange(1, N), m)
    east = 0.5 * (lo[:, j, i] + up[:, j - 1, i])
    west = 0.5 * (lo[:, j, i - 1] + up[:, j - 1, i - 1])
    north = 0.5 * (up[:, j, i] + lo[:, j, i - 1])
    south = 0.5 * (up[:, j - 1, i] + lo[:, j - 1, i - 1])
    r = np.arange(n)
    Xa = np.abs(X)
    zero = np.zeros((1, ref.P))
    Xp = np.vstack([Xa, zero])
    nb = {"e": np.where(i < m, r + 1, n), "w": np.where(i > 1, r - 1, n),
          "n": np.where(j < m, r + m, n), "s": np.where(j > 1, r - m, n)}
    G = np.abs(ref.G())
    bound = np.zeros((n, ref.P))
    for key, w in (("e", east), ("w", west), ("n", north), ("s", south)):
        D = Xa + Xp[nb[key]]
        for k in range(ref.K):
            bound += np.abs(w[k])[:, None] * (D @ G[k].T)
    per_a = np.bincount(ref.kab[:, 1], minlength=ref.P).max()
    return bound, int(4 * 2 * per_a)


@pytest.mark.parametrize("N,L,p,q", [(32, 2, 2, 4), (64, 4, 3, 6), (29, 3, 2, 4)])
def test_flux_apply_matches_oracle(gpu, N, L, p, q):
    """The edge-flux form of the fine FP32 operator (conductances per edge,
    y_r = sum over edges of sum_k w_k G_k (x_r - x_neighbour)) against the
    oracle's operator, elementwise within its rounding bound; switching back
    restores the five-slot form."""
    import torch
    import paper_2310_14649_gb300 as sg
    prob, ref = setup_pair(N, L, p, q)
    X = random_block(ref.n, ref.P, seed=55).astype(np.float32).astype(np.float64)
    try:
        assert sg.sg_apply_flux(prob, 1) == 1
        check_flux(prob, ref, X)
    finally:
        assert sg.sg_apply_flux(prob, 0) == 0
    prob.close()


def check_flux(prob, ref, X):
    import torch
    import paper_2310_14649_gb300 as sg
    Yr = galerkin.apply(ref, X)
    Xd = to_dev(X, torch.float32, ref.n + 7)
    Yd = torch.full((ref.P, ref.n + 3), float("nan"), dtype=torch.float32, device="cuda")
    sg.sg_apply(prob, Xd, Yd)
    Y = from_dev(Yd, ref.n)
    bound, m = flux_bound(ref, X)
    assert np.all(np.abs(Y - Yr) <= gamma(m, U32) * bound + 1e-30)
    assert np.linalg.norm(Y - Yr) <= 1e-5 * np.linalg.norm(Yr)
