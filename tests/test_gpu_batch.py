"""Graph-captured and batched solves through the C ABI (GPU): every system of
a batch reaches relres 1e-8 and the FP64 oracle's solution to 1e-7, a batch
of one agrees with sg_solve, and relaunching a recorded batch reproduces
its result bit for bit."""
import numpy as np
import pytest

from oracle import galerkin
from sg_inputs import batch_system

pytestmark = pytest.mark.gpu

# small systems of different sizes (mesh, KL modes, orders, boxes)
SMALL = [
    dict(N=24, L=2, p=2, q=4, sigma2=0.3, b=0.5, sx=2, sy=2, overlap=1),
    dict(N=32, L=3, p=2, q=4, sigma2=0.3, b=0.3, sx=2, sy=2, overlap=2),
    dict(N=40, L=2, p=3, q=6, sigma2=0.5, b=0.7, sx=3, sy=2, overlap=1),
]


def make(c):
    import paper_2310_14649_gb300 as sg
    prob = sg.sg_setup(c["N"], c["L"], c["p"], c["q"], sigma2=c["sigma2"], bx=c["b"], by=c["b"])
    sg.sg_precond_setup(prob, c["sx"], c["sy"], c["overlap"])
    return prob


def zeros(prob):
    import torch
    return torch.zeros((prob.P, prob.n), dtype=torch.float64, device="cuda")


@pytest.fixture(scope="module")
def small(gpu):
    probs = [make(c) for c in SMALL]
    refs = [galerkin.build(c["N"], c["L"], c["p"], c["q"], c["sigma2"], c["b"], c["b"]) for c in SMALL]
    sols = [galerkin.solve_direct(r) for r in refs]
    return probs, refs, sols


@pytest.mark.parametrize("mode,passes", [(1, 0), (0, 0), (1, 2)])
def test_batch_matches_oracle(small, mode, passes):
    import paper_2310_14649_gb300 as sg
    probs, refs, sols = small
    Xs = [zeros(p) for p in probs]
    infos = sg.sg_solve_batch(probs, Xs, rtol=1e-8, mode=mode, orth_passes=passes)
    for X, ref, Xd, inf in zip(Xs, refs, sols, infos):
        Xh = X.cpu().numpy().T
        assert inf["relres"] <= 1e-8
        assert galerkin.relres(ref, Xh) <= 1.01e-8
        assert np.linalg.norm(Xh - Xd) / np.linalg.norm(Xd) <= 1e-7
        assert 0 < inf["outer_it"] < 100 and inf["inner_it"] > 0
        if mode == 1:
            assert inf["ir_steps"] >= 1


def test_batch_of_one_agrees_with_sg_solve(small):
    import paper_2310_14649_gb300 as sg
    probs, refs, sols = small
    p = probs[1]
    X1 = zeros(p)
    i1 = sg.sg_solve(p, X1, rtol=1e-8, mode=1)
    X2 = zeros(p)
    i2 = sg.sg_solve_batch([p], [X2], rtol=1e-8, mode=1)[0]
    assert i2["relres"] <= 1e-8
    assert abs(i2["outer_it"] - i1["outer_it"]) <= 2
    d = (X1 - X2).norm().item() / X1.norm().item()
    assert d < 1e-7, d


def test_relaunch_is_reproducible_and_guess_is_used(small):
    import torch
    import paper_2310_14649_gb300 as sg
    probs, refs, sols = small
    B = sg.sg_batch_create(probs, rtol=1e-8, mode=1)
    Xa = [zeros(p) for p in probs]
    Xb = [zeros(p) for p in probs]
    ia = sg.sg_batch_solve(B, Xa)
    ib = sg.sg_batch_solve(B, Xb)
    for a, b, x, y in zip(ia, ib, Xa, Xb):
        assert a["outer_it"] == b["outer_it"] and a["inner_it"] == b["inner_it"]
        assert torch.equal(x, y)
    # warm start from the solution: no refinement step is needed
    ic = sg.sg_batch_solve(B, Xa)
    for inf in ic:
        assert inf["ir_steps"] == 0 and inf["outer_it"] == 0 and inf["relres"] <= 1e-8
    # manufactured right-hand sides through the recorded graph
    rng = np.random.default_rng(5)
    Fs, Xs_true = [], []
    for p, ref in zip(probs, refs):
        Xt = rng.standard_normal((ref.n, ref.P))
        Xs_true.append(Xt)
        Fs.append(torch.from_numpy(np.ascontiguousarray(galerkin.apply(ref, Xt).T)).cuda())
    Xm = [zeros(p) for p in probs]
    sg.sg_batch_solve(B, Xm, Fs=Fs)
    for X, Xt in zip(Xm, Xs_true):
        Xh = X.cpu().numpy().T
        assert np.linalg.norm(Xh - Xt) / np.linalg.norm(Xt) < 1e-5
    B.close()


def test_batch_rejects_changed_problem(gpu):
    import paper_2310_14649_gb300 as sg
    p = make(SMALL[0])
    B = sg.sg_batch_create([p], rtol=1e-8)
    sg.sg_precond_setup(p, 2, 2, 1)
    with pytest.raises(sg.SgError) as e:
        sg.sg_batch_solve(B, [zeros(p)])
    assert e.value.status == -1
    B.close()
    with pytest.raises(sg.SgError):
        sg.sg_batch_create([p, p])


@pytest.mark.parametrize("change", ["config", "kernel"])
def test_batch_rejects_reconfigured_apply(gpu, change):
    """A change of apply kernel frees the solver workspaces the batch was
    recorded with; a solve then re-creates them, possibly at the same
    addresses.  The recorded batch must refuse to run (SG_ERR_ARG) without
    launching its graph."""
    import paper_2310_14649_gb300 as sg
    p = make(SMALL[0])
    B = sg.sg_batch_create([p], rtol=1e-8)
    if change == "config":
        sg.sg_apply_config(p, rows=1, groups=1, prefetch=4)
    else:
        sg.sg_set_apply_kernel(p, 1)
    X = zeros(p)
    assert sg.sg_solve(p, X, rtol=1e-8, mode=1)["relres"] <= 1e-8
    l0 = sg.sg_launch_count()
    with pytest.raises(sg.SgError) as e:
        sg.sg_batch_solve(B, [zeros(p)])
    assert e.value.status == -1
    assert sg.sg_launch_count() == l0
    B.close()
    p.close()


def test_twelve_uneven_systems(gpu):
    """The batch of twelve seeded systems (meshes 64^2..384^2, L 2..5,
    p 2..4) in one recorded graph: every system reaches relres 1e-8, and
    the solutions agree with one-at-a-time sg_solve."""
    import paper_2310_14649_gb300 as sg
    cfgs = [batch_system(s) for s in range(12)]
    probs = [make(c) for c in cfgs]
    Xs = [zeros(p) for p in probs]
    infos = sg.sg_solve_batch(probs, Xs, rtol=1e-8, mode=1)
    for p, X, inf in zip(probs, Xs, infos):
        assert inf["relres"] <= 1e-8
        Y = zeros(p)
        sg.sg_solve(p, Y, rtol=1e-8, mode=1)
        assert (X - Y).norm().item() <= 1e-6 * Y.norm().item()
