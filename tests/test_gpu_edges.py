"""Edge cases across the GPU path: empty and single-image calls, the
deterministic problem (L = 0, one mode), the smallest meshes, RAS mode
chunkings, and batches that mix them."""
import numpy as np
import pytest

from oracle import galerkin
from sg_inputs import random_block

pytestmark = pytest.mark.gpu


def zeros(prob):
    import torch
    return torch.zeros((prob.P, prob.n), dtype=torch.float64, device="cuda")


def test_network_on_zero_and_one_image(gpu):
    import torch
    import paper_2310_14649_gb300 as sg
    prob = sg.sg_setup(24, 2, 2, 4)
    sg.sg_cnn_init(prob, seed=3)
    R = torch.zeros((0, prob.n), dtype=torch.float32, device="cuda")
    sg.sg_cnn_apply(prob, R, torch.zeros_like(R))   # nothing to do
    R1 = torch.from_numpy(random_block(prob.n, 1, seed=5).T.copy()).float().cuda()
    out = []
    for kernel in (1, 0):
        sg.sg_cnn_set_kernel(prob, kernel)
        Z = torch.full_like(R1, float("nan"))
        sg.sg_cnn_apply(prob, R1, Z)
        out.append(Z)
    assert torch.isfinite(out[0]).all()
    assert (out[0] - out[1]).abs().max().item() <= 1e-2 * out[1].abs().max().item()


@pytest.mark.parametrize("mode", [0, 1])
def test_deterministic_problem_one_mode(gpu, mode):
    """L = 0: P = K = 1, the Galerkin system is the deterministic FEM
    system with the mean coefficient."""
    import paper_2310_14649_gb300 as sg
    prob = sg.sg_setup(20, 0, 0, 0)
    sg.sg_precond_setup(prob, 2, 2, 1)
    X = zeros(prob)
    info = sg.sg_solve(prob, X, rtol=1e-10, mode=mode)
    ref = galerkin.build(20, 0, 0, 0)
    Xd = galerkin.solve_direct(ref)
    Xh = X.cpu().numpy().T
    assert info["relres"] <= 1e-10
    assert np.linalg.norm(Xh - Xd) / np.linalg.norm(Xd) < 1e-9


def test_smallest_mesh_with_preconditioner(gpu):
    """N = 4: a 3 x 3 interior grid and a 1-node coarse grid."""
    import paper_2310_14649_gb300 as sg
    prob = sg.sg_setup(4, 2, 1, 2)
    sg.sg_precond_setup(prob, 1, 1, 1)
    X = zeros(prob)
    info = sg.sg_solve(prob, X, rtol=1e-10, mode=1)
    ref = galerkin.build(4, 2, 1, 2)
    Xd = galerkin.solve_direct(ref)
    assert info["relres"] <= 1e-10
    assert np.linalg.norm(X.cpu().numpy().T - Xd) / np.linalg.norm(Xd) < 1e-9


def test_ras_chunkings_agree(gpu):
    """The RAS local solve gives identical results for every number of
    modes per CTA (modes are independent; the sums run in the same order)."""
    import torch
    import paper_2310_14649_gb300 as sg
    prob = sg.sg_setup(40, 3, 2, 4)
    R = torch.from_numpy(random_block(prob.n, prob.P, seed=9).T.copy()).float().cuda()
    out = []
    for modes in (0, 1, 2, 3, 7, 10):
        sg.sg_precond_setup(prob, 3, 3, 2, ras_modes=modes)
        Z = torch.full_like(R, float("nan"))
        sg.sg_precond_apply(prob, sg.PC_RAS_LOCAL, R, Z)
        out.append(Z)
    for Z in out[1:]:
        assert torch.equal(Z, out[0])


def test_batch_mixing_tiny_and_deterministic_systems(gpu):
    import paper_2310_14649_gb300 as sg
    specs = [(4, 2, 1, 2, 1), (20, 0, 0, 0, 2), (28, 3, 2, 4, 2)]
    probs, refs = [], []
    for N, L, p, q, S in specs:
        pr = sg.sg_setup(N, L, p, q)
        sg.sg_precond_setup(pr, S, S, 1)
        probs.append(pr)
        refs.append(galerkin.build(N, L, p, q))
    Xs = [zeros(p) for p in probs]
    infos = sg.sg_solve_batch(probs, Xs, rtol=1e-9, mode=1)
    for X, ref, inf in zip(Xs, refs, infos):
        Xd = galerkin.solve_direct(ref)
        assert inf["relres"] <= 1e-9
        assert np.linalg.norm(X.cpu().numpy().T - Xd) / np.linalg.norm(Xd) < 1e-8


def test_learned_smoother_in_a_batch(gpu):
    """A recorded batch uses the smoother selected at creation: a system
    with the trained network solves inside the graph."""
    import paper_2310_14649_gb300 as sg
    pr = sg.sg_setup(32, 2, 2, 4)
    sg.sg_precond_setup(pr, 2, 2, 1)
    sg.sg_train_precond(pr, n_pairs=384, epochs=6, batch=16, seed=1)
    ref = galerkin.build(32, 2, 2, 4)
    X = zeros(pr)
    info = sg.sg_solve_batch([pr], [X], rtol=1e-8, mode=1, max_it=300)[0]
    Xd = galerkin.solve_direct(ref)
    assert info["relres"] <= 1e-8
    assert np.linalg.norm(X.cpu().numpy().T - Xd) / np.linalg.norm(Xd) < 1e-7


def test_large_p_apply_in_separate_output_cta_groups(gpu):
    """The shape used for P > 48 (output groups in separate CTAs), forced on
    two small problems (P = 35 in 3 groups, P = 28 in 4), FP32 and FP64,
    against the oracle apply."""
    import torch
    import paper_2310_14649_gb300 as sg
    for (N, L, p, q, cg) in [(16, 3, 4, 8, 3), (12, 6, 2, 4, 4)]:
        prob = sg.sg_setup(N, L, p, q)
        ref = galerkin.build(N, L, p, q)
        X = random_block(ref.n, ref.P, seed=21)
        Yr = galerkin.apply(ref, X)
        for which, dt, tol in ((0, torch.float32, 2e-5), (2, torch.float64, 1e-12)):
            sg.sg_apply_config(prob, 1, 1, 1, 1, 8, 1, 0, cg, which=which)
            sg.sg_set_apply_kernel(prob, 2)
            Xd = torch.from_numpy(np.ascontiguousarray(X.T)).to(dt).cuda()
            Yd = torch.full_like(Xd, float("nan"))
            sg.sg_apply(prob, Xd, Yd)
            Y = Yd.double().cpu().numpy().T
            assert np.max(np.abs(Y - Yr)) <= tol * np.max(np.abs(Yr)), (N, L, which)
        prob.close()
