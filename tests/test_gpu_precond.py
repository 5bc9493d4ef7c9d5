"""Preconditioner pieces (Sec. 3) through the C ABI versus the FP64 oracle
(GPU): integer artefacts bit-exact, operators within rounding bounds."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import amg, coarse, galerkin, ras, twolevel
from sg_inputs import random_block

pytestmark = pytest.mark.gpu

CASES = [
    # N, L, p, q, sigma2, b, sx, sy, overlap
    (32, 2, 2, 4, 0.3, 0.5, 2, 2, 1),
    (36, 3, 2, 4, 0.5, 0.2, 3, 2, 2),
]


@pytest.fixture(scope="module", params=CASES, ids=lambda c: "N%d_L%d_p%d" % c[:3])
def pair(request, gpu):
    import paper_2310_14649_gb300 as sg
    N, L, p, q, s2, b, sx, sy, ov = request.param
    prob = sg.sg_setup(N, L, p, q, sigma2=s2, bx=b, by=b)
    sg.sg_precond_setup(prob, sx, sy, ov, inner_rtol=1e-13, inner_max=200)
    ref = galerkin.build(N, L, p, q, sigma2=s2, bx=b, by=b)
    omega = sg.sg_precond_info(prob)[0]
    tl = twolevel.TwoLevel(ref, sx, sy, ov, exact_coarse=True, omega=omega)
    return prob, ref, tl, (sx, sy, ov)


def dev(X, dtype, ld=None):
    import torch
    n, P = X.shape
    out = torch.zeros((P, ld or n), dtype=dtype, device="cuda")
    out[:, :n] = torch.from_numpy(np.ascontiguousarray(X.T)).to(dtype)
    return out


def host(Y, n):
    return Y[:, :n].double().cpu().numpy().T


def run(prob, which, X, nout, dtype):
    import torch
    import paper_2310_14649_gb300 as sg
    Xd = dev(X, dtype, X.shape[0] + 3)
    Yd = torch.full((X.shape[1], nout + 5), float("nan"), dtype=dtype, device="cuda")
    sg.sg_precond_apply(prob, which, Xd, Yd)
    torch.cuda.synchronize()
    return host(Yd, nout), host(Xd, X.shape[0])


def test_partitions_bit_exact(pair):
    import paper_2310_14649_gb300 as sg
    prob, ref, tl, (sx, sy, ov) = pair
    parts = ras.partitions(ref.A(0), ref.N, sx, sy, ov)
    for b, (idx, own) in enumerate(parts):
        gi, go = sg.sg_get_partition(prob, b)
        assert np.array_equal(gi, idx) and np.array_equal(go, own)


def test_coarse_pattern_bit_exact(pair):
    import paper_2310_14649_gb300 as sg
    prob, ref, tl, _ = pair
    RT = abs(coarse.interpolation(ref.N))
    pat = sp.csr_matrix((np.ones(len(ref.colidx)), ref.colidx, ref.rowptr), shape=(ref.n, ref.n))
    S = (RT.T @ pat @ RT).tocsr()
    S.sort_indices()
    rp, ci = sg.sg_get_coarse_csr(prob)
    assert np.array_equal(rp, S.indptr) and np.array_equal(ci, S.indices)


def test_amg_aggregates_bit_exact(pair):
    import paper_2310_14649_gb300 as sg
    prob, ref, tl, _ = pair
    levels = amg.setup(tl.Acs[0])
    nlev = sg.sg_precond_info(prob)[1]
    assert nlev == len(levels)
    A = tl.Acs[0]
    for lev in range(nlev - 1):
        n, agg = sg.sg_get_amg_level(prob, lev)
        ragg, _ = amg.aggregate(A)
        assert n == A.shape[0] and np.array_equal(agg, ragg)
        A = levels[lev + 1].A


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_transfer_and_coarse_operator(pair, dt):
    import torch
    import paper_2310_14649_gb300 as sg
    prob, ref, tl, _ = pair
    dtype = torch.float64 if dt == "f64" else torch.float32
    tol = 1e-14 if dt == "f64" else 2e-6
    nc = tl.nc
    X = random_block(ref.n, ref.P, seed=31)
    Y, Xq = run(prob, sg.PC_RESTRICT, X, nc, dtype)
    Yr = tl.R @ Xq
    assert np.max(np.abs(Y - Yr)) <= tol * np.max(np.abs(Yr))
    Xc = random_block(nc, ref.P, seed=32)
    Y, Xq = run(prob, sg.PC_INTERP, Xc, ref.n, dtype)
    Yr = tl.RT @ Xq
    assert np.max(np.abs(Y - Yr)) <= tol * np.max(np.abs(Yr))
    Y, Xq = run(prob, sg.PC_COARSE_APPLY, Xc, nc, dtype)
    Yr = coarse.coarse_apply(tl.Acs, tl.G, Xq)
    scale = np.max(np.abs(coarse.coarse_apply([abs(a) for a in tl.Acs], abs(tl.G), abs(Xq))))
    assert np.max(np.abs(Y - Yr)) <= (50 * tol) * scale


@pytest.mark.parametrize("fp64", [1, 2])
def test_coarse_apply_fp64_paths(pair, fp64):
    """The FP64 coarse operator on its generated kernel and on assembled
    edge blocks, against the oracle."""
    import torch
    import paper_2310_14649_gb300 as sg
    prob, ref, tl, _ = pair
    try:
        sg.sg_set_apply_fp64(prob, fp64)
        Xc = random_block(tl.nc, ref.P, seed=38)
        Y, Xq = run(prob, sg.PC_COARSE_APPLY, Xc, tl.nc, torch.float64)
        info = sg.sg_apply_fp64_info(prob)
        assert info["coarse"] == (fp64 == 2) and (info["bytes"] > 0) == (fp64 == 2)
        Yr = coarse.coarse_apply(tl.Acs, tl.G, Xq)
        scale = np.max(np.abs(coarse.coarse_apply([abs(a) for a in tl.Acs], abs(tl.G), abs(Xq))))
        assert np.max(np.abs(Y - Yr)) <= 5e-13 * scale
    finally:
        sg.sg_set_apply_fp64(prob, 0)


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_amg_vcycle(pair, dt):
    import torch
    import paper_2310_14649_gb300 as sg
    prob, ref, tl, _ = pair
    dtype = torch.float64 if dt == "f64" else torch.float32
    levels = amg.setup(tl.Acs[0])
    Xc = random_block(tl.nc, ref.P, seed=33)
    Y, Xq = run(prob, sg.PC_AMG, Xc, tl.nc, dtype)
    Yr = amg.vcycle(levels, Xq)
    tol = 1e-11 if dt == "f64" else 1e-4
    assert np.max(np.abs(Y - Yr)) <= tol * np.max(np.abs(Yr))


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_ras_and_smoother(pair, dt):
    import torch
    import paper_2310_14649_gb300 as sg
    prob, ref, tl, _ = pair
    dtype = torch.float64 if dt == "f64" else torch.float32
    tol = 1e-11 if dt == "f64" else 1e-4
    X = random_block(ref.n, ref.P, seed=34)
    Y, Xq = run(prob, sg.PC_RAS_LOCAL, X, ref.n, dtype)
    Yr = ras.apply_ras(tl.parts, tl.solvers, Xq)
    assert np.max(np.abs(Y - Yr)) <= tol * np.max(np.abs(Yr))
    Y, Xq = run(prob, sg.PC_SMOOTH, X, ref.n, dtype)
    Yr = tl.omega * tl.ras(Xq)
    assert np.max(np.abs(Y - Yr)) <= tol * np.max(np.abs(Yr))


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_ras_ring_depths(pair, dt):
    """The RAS local solves with 2, 3, 5 and 8 line steps' matrices in
    flight (and the automatic depth) match the oracle; a depth outside 2..8
    is rejected."""
    import torch
    import paper_2310_14649_gb300 as sg
    prob, ref, tl, (sx, sy, ov) = pair
    dtype = torch.float64 if dt == "f64" else torch.float32
    tol = 1e-11 if dt == "f64" else 1e-4
    X = random_block(ref.n, ref.P, seed=36)
    try:
        for stages in (2, 3, 5, 8, 0):
            sg.sg_precond_setup(prob, sx, sy, ov, inner_rtol=1e-13, inner_max=200, ras_stages=stages)
            Y, Xq = run(prob, sg.PC_RAS_LOCAL, X, ref.n, dtype)
            Yr = ras.apply_ras(tl.parts, tl.solvers, Xq)
            assert np.max(np.abs(Y - Yr)) <= tol * np.max(np.abs(Yr)), stages
        for bad in (1, 9):
            with pytest.raises(sg.SgError):
                sg.sg_precond_setup(prob, sx, sy, ov, ras_stages=bad)
    finally:
        sg.sg_precond_setup(prob, sx, sy, ov, inner_rtol=1e-13, inner_max=200)


def test_ras_kernel_automatic_choice(pair):
    """ras_kernel 3 keeps one of the two FP32 local-solve kernels (the
    faster on this problem) and the local solves match the oracle."""
    import torch
    import paper_2310_14649_gb300 as sg
    prob, ref, tl, (sx, sy, ov) = pair
    try:
        sg.sg_precond_setup(prob, sx, sy, ov, inner_rtol=1e-13, inner_max=200, ras_kernel=3)
        assert sg.sg_precond_ras_kernel(prob) in (0, 2)
        X = random_block(ref.n, ref.P, seed=40)
        Y, Xq = run(prob, sg.PC_RAS_LOCAL, X, ref.n, torch.float32)
        Yr = ras.apply_ras(tl.parts, tl.solvers, Xq)
        assert np.max(np.abs(Y - Yr)) <= 1e-4 * np.max(np.abs(Yr))
    finally:
        sg.sg_precond_setup(prob, sx, sy, ov, inner_rtol=1e-13, inner_max=200)


@pytest.mark.parametrize("kernel,modes", [(1, 0), (1, 3), (1, 8), (1, 10), (0, 0), (0, 4)])
def test_ras_kernels(pair, kernel, modes):
    """FP32 RAS local solves on the tensor cores (3xTF32 MMA; several mode
    chunks per box, ragged last chunk, one or two 8-mode tiles) and on the
    FMA kernel match the oracle."""
    import torch
    import paper_2310_14649_gb300 as sg
    prob, ref, tl, (sx, sy, ov) = pair
    X = random_block(ref.n, ref.P, seed=37)
    try:
        sg.sg_precond_setup(prob, sx, sy, ov, inner_rtol=1e-13, inner_max=200, ras_kernel=kernel, ras_modes=modes)
        Y, Xq = run(prob, sg.PC_RAS_LOCAL, X, ref.n, torch.float32)
        Yr = ras.apply_ras(tl.parts, tl.solvers, Xq)
        assert np.max(np.abs(Y - Yr)) <= 1e-4 * np.max(np.abs(Yr))
        assert np.linalg.norm(Y - Yr) <= 2e-6 * np.linalg.norm(Yr)
        with pytest.raises(sg.SgError):
            sg.sg_precond_setup(prob, sx, sy, ov, ras_kernel=4)
    finally:
        sg.sg_precond_setup(prob, sx, sy, ov, inner_rtol=1e-13, inner_max=200)


def test_omega_estimate_is_the_smoother_radius(pair):
    import paper_2310_14649_gb300 as sg
    prob, ref, tl, _ = pair
    omega = sg.sg_precond_info(prob)[0]
    tl1 = twolevel.TwoLevel(ref, *pair[3], exact_coarse=True, omega=None)
    # both sides run 20 power iterations (FP32 on the GPU, FP64 here)
    assert abs(omega - tl1.omega) <= 1e-3 * tl1.omega


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_coarse_correction_and_two_level(pair, dt):
    """With the inner coarse GMRES driven to 1e-13, Q and the two-level
    cycle match the oracle's exact coarse solve."""
    import torch
    import paper_2310_14649_gb300 as sg
    prob, ref, tl, _ = pair
    dtype = torch.float64 if dt == "f64" else torch.float32
    tol = 1e-9 if dt == "f64" else 2e-4
    X = random_block(ref.n, ref.P, seed=35)
    Y, Xq = run(prob, sg.PC_COARSE, X, ref.n, dtype)
    Yr = tl.RT @ tl.coarse_solve(tl.R @ Xq)
    assert np.max(np.abs(Y - Yr)) <= tol * np.max(np.abs(Yr))
    Y, Xq = run(prob, sg.PC_TWOLEVEL, X, ref.n, dtype)
    Yr = tl.apply(Xq)
    assert np.max(np.abs(Y - Yr)) <= tol * np.max(np.abs(Yr))


@pytest.mark.parametrize("cfg", [(1, 1, 1, 4, 8, 1), (1, 2, 1, 2, 16, 1), (2, 1, 1, 2, 8, 1), (1, 1, 2, 1, 8, 1),
                                 (1, 1, 1, 1, 16, 1, 3), (1, 1, 1, 7, 16, 1, 0, 1, 1), (1, 1, 2, 4, 16, 1, 0, 1, 1),
                                 (2, 1, 1, 4, 16, 1, 0, 1, 2)])
def test_coarse_apply_tile_shapes(pair, cfg):
    """The coarse family's specialised kernel in several tile shapes."""
    import torch
    import paper_2310_14649_gb300 as sg
    prob, ref, tl, _ = pair
    sg.sg_apply_config(prob, *cfg, which=1)
    Xc = random_block(tl.nc, ref.P, seed=41)
    Y, Xq = run(prob, sg.PC_COARSE_APPLY, Xc, tl.nc, torch.float32)
    Yr = coarse.coarse_apply(tl.Acs, tl.G, Xq)
    scale = np.max(np.abs(coarse.coarse_apply([abs(a) for a in tl.Acs], abs(tl.G), abs(Xq))))
    assert np.max(np.abs(Y - Yr)) <= 1e-4 * scale
    sg.sg_apply_config(prob, 1, 1, 1, 4, 32, 1, which=1)


@pytest.fixture(scope="module")
def multilevel(gpu):
    """N = 128: 3,969 coarse unknowns, a hierarchy of several levels."""
    import paper_2310_14649_gb300 as sg
    N, L, p, q, s2, b = 128, 2, 2, 4, 0.3, 0.5
    ref = galerkin.build(N, L, p, q, sigma2=s2, bx=b, by=b)
    Acs, _ = coarse.coarse_matrices(ref)
    levels = amg.setup(Acs[0])
    prob = sg.sg_setup(N, L, p, q, sigma2=s2, bx=b, by=b)
    return prob, ref, levels, Acs[0].shape[0]


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_amg_vcycle_kernels_multilevel(multilevel, dt):
    """The fused V-cycle (level 0 GPU-wide, the coarser levels in one launch
    with one CTA per mode) and one launch per level operation both match the
    oracle's V-cycle on a hierarchy of three levels."""
    import torch
    import paper_2310_14649_gb300 as sg
    prob, ref, levels, nc = multilevel
    assert len(levels) >= 3
    dtype = torch.float64 if dt == "f64" else torch.float32
    Xc = random_block(nc, ref.P, seed=35)
    tol = 1e-11 if dt == "f64" else 1e-4
    out = {}
    for cl in (0, 1):
        sg.sg_precond_setup(prob, 4, 4, 1, amg_kernel=cl)
        assert sg.sg_precond_info(prob)[1] == len(levels)
        Y, Xq = run(prob, sg.PC_AMG, Xc, nc, dtype)
        Yr = amg.vcycle(levels, Xq)
        assert np.max(np.abs(Y - Yr)) <= tol * np.max(np.abs(Yr)), cl
        # a second application on the same buffers gives the same result
        Y2, _ = run(prob, sg.PC_AMG, Xc, nc, dtype)
        assert np.array_equal(Y, Y2), cl
        out[cl] = Y
    with pytest.raises(sg.SgError) as e:
        sg.sg_precond_setup(prob, 4, 4, 1, amg_kernel=2)
    assert e.value.status == -1


def test_ras_explicit_inverses(pair):
    """RAS local solves by explicit local inverses on tcgen05 (ras_kernel 2:
    FP32 owned rows of each local inverse, TF32 products with operands split
    into high and remainder parts): the local solves, the smoother with its
    fused Kronecker factor, and the two-level cycle against the oracle; a
    wait limit of 0 is reported as SG_ERR_TIMEOUT and the next apply agrees
    with the first."""
    import torch
    import paper_2310_14649_gb300 as sg
    prob, ref, tl, (sx, sy, ov) = pair
    X = random_block(ref.n, ref.P, seed=39)
    try:
        sg.sg_precond_setup(prob, sx, sy, ov, inner_rtol=1e-13, inner_max=200, ras_kernel=2)
        Y, Xq = run(prob, sg.PC_RAS_LOCAL, X, ref.n, torch.float32)
        Yr = ras.apply_ras(tl.parts, tl.solvers, Xq)
        assert np.max(np.abs(Y - Yr)) <= 1e-4 * np.max(np.abs(Yr))
        # the inverse entries are stored in FP32: their rounding (u = 2^-24)
        # accumulates over the n_i overlapped nodes of a row, about
        # sqrt(n_i) u relative in L2 (2e-6 for 36^2 nodes), plus the TF32
        # split's 2^-22 per product
        assert np.linalg.norm(Y - Yr) <= 1e-5 * np.linalg.norm(Yr)
        omega = sg.sg_precond_info(prob)[0]
        Y, Xq = run(prob, sg.PC_SMOOTH, X, ref.n, torch.float32)
        Gt = ras.kronecker_factor(ref)
        Yr = omega * np.linalg.solve(Gt, ras.apply_ras(tl.parts, tl.solvers, Xq).T).T
        assert np.max(np.abs(Y - Yr)) <= 1e-4 * np.max(np.abs(Yr))
        try:
            sg.sg_set_wait_limit(prob, 0)
            with pytest.raises(sg.SgError) as e:
                run(prob, sg.PC_RAS_LOCAL, X, ref.n, torch.float32)
            assert e.value.status == -5
        finally:
            sg.sg_set_wait_limit(prob, -1)
        Y2, _ = run(prob, sg.PC_RAS_LOCAL, X, ref.n, torch.float32)
        Y1, _ = run(prob, sg.PC_RAS_LOCAL, X, ref.n, torch.float32)
        assert np.array_equal(Y1, Y2)
        # FP64 data keep the line kernel
        Y, Xq = run(prob, sg.PC_RAS_LOCAL, X, ref.n, torch.float64)
        Yr = ras.apply_ras(tl.parts, tl.solvers, Xq)
        assert np.max(np.abs(Y - Yr)) <= 1e-11 * np.max(np.abs(Yr))
    finally:
        sg.sg_precond_setup(prob, sx, sy, ov, inner_rtol=1e-13, inner_max=200)


@pytest.mark.parametrize("L,p", [(4, 3), (4, 4), (6, 3)], ids=["P35", "P70", "P84"])
def test_ras_explicit_inverses_wide_modes(gpu, L, p):
    """Explicit-inverse local solves and the smoother with its fused
    Kronecker factor at P = 35, 70 and 84 (48, 80 and 96 padded modes: two
    accumulation chains with two accumulators, one chain with four slots,
    one chain with two slots) against the oracle, on a 24^2 mesh whose boxes
    have a ragged 128-row tile (144 owned rows) and a ragged node chunk (168
    overlapped nodes)."""
    import torch
    import paper_2310_14649_gb300 as sg
    N, q, sx, sy, ov = 24, 2, 2, 2, 1
    prob = sg.sg_setup(N, L, p, q, sigma2=0.3, bx=0.5, by=0.5)
    try:
        sg.sg_precond_setup(prob, sx, sy, ov, inner_rtol=1e-13, inner_max=200, ras_kernel=2)
        assert sg.sg_precond_ras_kernel(prob) == 2
        ref = galerkin.build(N, L, p, q, sigma2=0.3, bx=0.5, by=0.5)
        parts = ras.partitions(ref.A(0), N, sx, sy, ov)
        solvers = ras.local_solvers(ref.A(0), parts)
        X = random_block(ref.n, ref.P, seed=43)
        Y, Xq = run(prob, sg.PC_RAS_LOCAL, X, ref.n, torch.float32)
        Yr = ras.apply_ras(parts, solvers, Xq)
        assert np.max(np.abs(Y - Yr)) <= 1e-4 * np.max(np.abs(Yr))
        assert np.linalg.norm(Y - Yr) <= 1e-5 * np.linalg.norm(Yr)
        omega = sg.sg_precond_info(prob)[0]
        Y, Xq = run(prob, sg.PC_SMOOTH, X, ref.n, torch.float32)
        Gt = ras.kronecker_factor(ref)
        Yr = omega * np.linalg.solve(Gt, ras.apply_ras(parts, solvers, Xq).T).T
        assert np.max(np.abs(Y - Yr)) <= 1e-4 * np.max(np.abs(Yr))
    finally:
        prob.close()
