"""Batched deterministic solves for Monte Carlo verification (Sec. 4.1,
Fig. mcs_verify_poisson) through the C ABI (GPU): each sample against the
oracle's sparse direct solve of the same deterministic problem, and the
paper's verification setting (10,201 vertices, three random variables,
input order 2, output order 3, sigma = 0.1, 40,000 samples) comparing the
GPU's SG solution with the GPU's Monte Carlo samples and with a
Gauss-Hermite collocation of the oracle."""
import itertools

import numpy as np
import pytest
import scipy.sparse.linalg as spla
from numpy.polynomial import hermite_e as H

from oracle import fem, galerkin

pytestmark = pytest.mark.gpu


def samples(S, L, seed):
    return np.random.default_rng(seed).standard_normal((S, L))


def chaos(mi, xi):
    """psi_a(xi_s) for the orthonormal Hermite chaos: [S, P]."""
    from math import factorial
    out = np.ones((xi.shape[0], mi.shape[0]))
    for a, alpha in enumerate(mi):
        for d, k in enumerate(alpha):
            if k:
                c = np.zeros(int(k) + 1)
                c[-1] = 1.0
                out[:, a] *= H.hermeval(xi[:, d], c) / np.sqrt(float(factorial(int(k))))
    return out


@pytest.mark.parametrize("N,L,dt", [(20, 3, "f64"), (33, 2, "f32"), (37, 4, "f32")])
def test_samples_match_direct_solves(gpu, N, L, dt):
    """Meshes whose node counts are below, equal to and above one node per
    thread of the 1024-thread CTA."""
    import torch
    import paper_2310_14649_gb300 as sg
    prob = sg.sg_setup(N, L, 1, 2, sigma2=0.5, bx=0.3, by=0.3)
    ref = galerkin.build(N, L, 1, 2, 0.5, 0.3, 0.3)
    xi = samples(7, L, 5)
    dtype = torch.float64 if dt == "f64" else torch.float32
    U = torch.full((7, ref.n + 5), float("nan"), dtype=dtype, device="cuda")
    its = sg.sg_sample_solve(prob, torch.from_numpy(xi).cuda(), U, rtol=1e-6)
    assert 0 < its < 2000
    Uh = U[:, :ref.n].double().cpu().numpy()
    for s in range(7):
        u = spla.spsolve(fem.assemble(N, np.exp(xi[s] @ ref.gfield)).tocsc(), ref.b)
        assert np.linalg.norm(Uh[s] - u) <= 2e-5 * np.linalg.norm(u), s
    prob.close()


def test_paper_verification_setting(gpu):
    """101 x 101 vertices (N = 100), L = 3, input order 2, output order 3,
    sigma = 0.1 (variance 0.01), four subdomains; 40,000 Monte Carlo
    samples on the GPU.  The SG mean and standard deviation agree with the
    Monte Carlo ones within four standard errors plus the SG truncation
    error (measured against a 6^3-point collocation of the exact lognormal
    problem), at the points (0.5, 0.5) and (0.3, 0.7) and over the mesh;
    the SG surrogate evaluated at every sample agrees with that sample's
    deterministic solve (so the pdfs at the two points agree)."""
    import torch
    import paper_2310_14649_gb300 as sg
    N, L, p, q, s2, b = 100, 3, 3, 2, 0.01, 0.5
    prob = sg.sg_setup(N, L, p, q, sigma2=s2, bx=b, by=b)
    sg.sg_precond_setup(prob, 2, 2, 1)
    X = torch.zeros((prob.P, prob.n), dtype=torch.float64, device="cuda")
    info = sg.sg_solve(prob, X, rtol=1e-10, mode=1)
    assert info["relres"] <= 1e-10
    Xh = X.cpu().numpy().T                                # [n, P]
    mean_sg = Xh[:, 0]
    std_sg = np.sqrt(np.sum(Xh[:, 1:] ** 2, axis=1))
    S = 40000
    xi = samples(S, L, 2023)
    U = torch.empty((S, prob.n), dtype=torch.float32, device="cuda")
    its = sg.sg_sample_solve(prob, torch.from_numpy(xi).cuda(), U, rtol=1e-6)
    assert its < 2000
    Ud = U.double()
    mean_mc = Ud.mean(0).cpu().numpy()
    std_mc = Ud.std(0).cpu().numpy()
    # collocation of the exact lognormal problem (oracle)
    ref = galerkin.build(N, L, p, q, s2, b, b)
    x, w = H.hermegauss(6)
    w = w / np.sqrt(2.0 * np.pi)
    m1 = np.zeros(ref.n)
    m2 = np.zeros(ref.n)
    for i, j, k in itertools.product(range(6), repeat=3):
        u = spla.spsolve(fem.assemble(N, np.exp(np.array([x[i], x[j], x[k]]) @ ref.gfield)).tocsc(), ref.b)
        m1 += w[i] * w[j] * w[k] * u
        m2 += w[i] * w[j] * w[k] * u * u
    std_c = np.sqrt(m2 - m1 ** 2)
    trunc_mean = np.abs(mean_sg - m1)
    trunc_std = np.abs(std_sg - std_c)
    assert np.linalg.norm(trunc_mean) <= 1e-6 * np.linalg.norm(m1)
    assert np.linalg.norm(trunc_std) <= 1e-3 * np.linalg.norm(std_c)
    se_mean = std_mc / np.sqrt(S)
    se_std = std_mc / np.sqrt(2.0 * S)
    m = N - 1
    for (px, py) in ((0.5, 0.5), (0.3, 0.7)):
        r = (round(py * N) - 1) * m + (round(px * N) - 1)
        assert abs(mean_sg[r] - mean_mc[r]) <= 4 * se_mean[r] + trunc_mean[r] + 1e-6 * mean_sg[r]
        assert abs(std_sg[r] - std_mc[r]) <= 4 * se_std[r] + trunc_std[r] + 1e-4 * std_sg[r]
    assert np.linalg.norm(mean_sg - mean_mc) <= 4 * np.linalg.norm(se_mean) + np.linalg.norm(trunc_mean) \
        + 1e-6 * np.linalg.norm(mean_sg)
    # the surrogate at every sample: sum_a X[r, a] psi_a(xi_s) at the two points
    mi = sg.sg_get_multi_indices(prob, 0)
    Psi = chaos(mi, xi)                                   # [S, P]
    for (px, py) in ((0.5, 0.5), (0.3, 0.7)):
        r = (round(py * N) - 1) * m + (round(px * N) - 1)
        u_sg = Psi @ Xh[r]
        u_mc = Ud[:, r].cpu().numpy()
        assert np.max(np.abs(u_sg - u_mc)) <= 2e-3 * np.max(np.abs(u_mc))
    prob.close()
