"""Pins of the oracle's CNN smoother (CPU): the convolution against a
direct 2D correlation, gradients against central differences, the Adam step
against its closed form on a quadratic."""
import numpy as np
import pytest
import scipy.signal

from oracle import cnn


def test_conv_matches_direct_correlation():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 7, 9, 3))
    W = rng.standard_normal((3, 3, 3, 4))
    b = rng.standard_normal(4)
    y = cnn.conv3x3(x, W, b)
    for n in range(2):
        for co in range(4):
            ref = b[co] + sum(scipy.signal.correlate2d(x[n, :, :, ci], W[:, :, ci, co], mode="same")
                              for ci in range(3))
            assert np.max(np.abs(y[n, :, :, co] - ref)) < 1e-12


def test_gradients_by_central_differences():
    rng = np.random.default_rng(1)
    params = [(rng.standard_normal((3, 3, ci, co)) * 0.4, rng.standard_normal(co) * 0.1)
              for ci, co in [(2, 3), (3, 3), (3, 1)]]
    x = rng.standard_normal((2, 5, 6, 2))
    zs = rng.standard_normal((2, 5, 6, 1))

    def L(p, xx):
        y, _ = cnn.forward(p, xx)
        return cnn.loss(y, zs)[0]
    y, acts = cnn.forward(params, x)
    _, dy = cnn.loss(y, zs)
    grads, dx = cnn.backward(params, acts, dy)
    h = 1e-6
    checks = [(0, 0, (1, 2, 0, 1)), (1, 0, (0, 0, 2, 2)), (2, 0, (2, 1, 1, 0)), (0, 1, (2,)), (2, 1, (0,))]
    for l, which, idx in checks:
        pp = [(W.copy(), b.copy()) for W, b in params]
        pm = [(W.copy(), b.copy()) for W, b in params]
        pp[l][which][idx] += h
        pm[l][which][idx] -= h
        num = (L(pp, x) - L(pm, x)) / (2 * h)
        ana = grads[l][which][idx]
        assert abs(num - ana) <= 1e-6 * max(1.0, abs(num)), (l, which, idx, num, ana)
    for idx in [(0, 1, 2, 0), (1, 4, 5, 1)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        num = (L(params, xp) - L(params, xm)) / (2 * h)
        assert abs(num - dx[idx]) <= 1e-6 * max(1.0, abs(num))


def test_adam_first_step_closed_form():
    """After one step from zero moments, every parameter moves by
    lr * sign(g) (up to eps)."""
    params = [(np.ones((3, 3, 1, 1)), np.zeros(1))]
    g = [(np.full((3, 3, 1, 1), 0.3), np.array([-2.0]))]
    new, state = cnn.adam_step(params, g, cnn.adam_init(params), lr=1e-2)
    assert np.allclose(new[0][0], 1.0 - 1e-2, atol=1e-9)
    assert np.allclose(new[0][1], 1e-2, atol=1e-9)


@pytest.mark.parametrize("b1,b2", [(0.9, 0.999), (0.5, 0.75)])
def test_adam_several_steps_closed_form(b1, b2):
    """Steps t = 1..5 with gradients that change from step to step: the
    moments are the bias-corrected exponentially weighted sums
    m_t = (1-b1) sum_s b1^(t-s) g_s / (1-b1^t) and
    v_t = (1-b2) sum_s b2^(t-s) g_s^2 / (1-b2^t) (Kingma and Ba, Alg. 1 in
    closed form), and the parameter after t steps is
    theta_0 - lr sum_{s<=t} m_s / (sqrt(v_s) + eps).  With two different
    (b1, b2) pairs a swapped decay rate, a wrong bias-correction power or a
    missing correction fails."""
    lr, eps = 1e-2, 1e-8
    theta0 = np.array([0.7, -1.3, 2.0])
    gs = [np.array([0.3, -2.0, 0.05]) * (1 + 0.5 * s) * (-1) ** s for s in range(5)]
    gs = [gs[s] + np.array([0.1, 0.2, -0.3]) * s * s for s in range(5)]
    params = [(theta0.reshape(3, 1, 1, 1), np.array([0.25]))]
    state = cnn.adam_init(params)
    expect = theta0.copy()
    expect_b = 0.25
    for t in range(1, 6):
        grads = [(gs[t - 1].reshape(3, 1, 1, 1), np.array([gs[t - 1][0] - 1.0]))]
        params, state = cnn.adam_step(params, grads, state, lr=lr, b1=b1, b2=b2, eps=eps)
        w1 = np.array([(1 - b1) * b1 ** (t - s) for s in range(1, t + 1)]) / (1 - b1 ** t)
        w2 = np.array([(1 - b2) * b2 ** (t - s) for s in range(1, t + 1)]) / (1 - b2 ** t)
        G = np.array(gs[:t])
        mh = w1 @ G
        vh = w2 @ (G * G)
        expect = expect - lr * mh / (np.sqrt(vh) + eps)
        gb = G[:, 0] - 1.0
        expect_b = expect_b - lr * (w1 @ gb) / (np.sqrt(w2 @ (gb * gb)) + eps)
        assert state[0] == t
        np.testing.assert_allclose(params[0][0].ravel(), expect, rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(params[0][1], [expect_b], rtol=1e-13, atol=1e-15)


def test_adam_minimises_a_quadratic():
    """On f(theta) = 0.5 sum a_i theta_i^2 Adam with a small step reaches
    the minimiser: after 3000 steps of lr 1e-2 every |theta_i| is below
    a few lr (its steps are about lr in size near the optimum)."""
    a = np.array([1.0, 10.0, 0.1])
    params = [(np.array([1.0, -2.0, 3.0]).reshape(3, 1, 1, 1), np.zeros(1))]
    state = cnn.adam_init(params)
    for _ in range(3000):
        th = params[0][0].ravel()
        params, state = cnn.adam_step(params, [((a * th).reshape(3, 1, 1, 1), np.zeros(1))], state, lr=1e-2)
    assert np.all(np.abs(params[0][0]) < 5e-2)


def test_he_init_scale():
    p = cnn.he_init(np.random.default_rng(0))
    W = p[1][0]
    assert W.shape == (3, 3, 32, 32)
    assert abs(W.std() - np.sqrt(2.0 / 288)) < 0.05 * np.sqrt(2.0 / 288)


def test_energy_loss_gradient_and_special_cases():
    """The energy-norm loss: its gradient by central differences through the
    network, the value for A_0 = I equals the plain relative squared error,
    and it is zero at the target."""
    import scipy.sparse as sp
    rng = np.random.default_rng(3)
    m = 5
    T = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(m, m))
    A0 = (sp.kron(sp.identity(m), T) + sp.kron(T, sp.identity(m))).tocsr()
    params = [(rng.standard_normal((3, 3, ci, co)) * 0.4, rng.standard_normal(co) * 0.1)
              for ci, co in [(2, 3), (3, 1)]]
    x = rng.standard_normal((2, m, m, 2))
    zs = rng.standard_normal((2, m, m, 1))

    def L(p):
        y, _ = cnn.forward(p, x)
        return cnn.loss_energy(y, zs, A0)[0]
    y, acts = cnn.forward(params, x)
    _, dy = cnn.loss_energy(y, zs, A0)
    grads, _ = cnn.backward(params, acts, dy)
    h = 1e-6
    for l, which, idx in [(0, 0, (2, 1, 1, 2)), (1, 0, (0, 2, 1, 0)), (0, 1, (1,)), (1, 1, (0,))]:
        pp = [(W.copy(), b.copy()) for W, b in params]
        pm = [(W.copy(), b.copy()) for W, b in params]
        pp[l][which][idx] += h
        pm[l][which][idx] -= h
        num = (L(pp) - L(pm)) / (2 * h)
        assert abs(num - grads[l][which][idx]) <= 1e-6 * max(1.0, abs(num))
    eye = sp.identity(m * m, format="csr")
    assert abs(cnn.loss_energy(y, zs, eye)[0] - cnn.loss(y, zs)[0]) <= 1e-12 * cnn.loss(y, zs)[0]
    L0, g0 = cnn.loss_energy(zs, zs, A0)
    assert L0 == 0.0 and np.all(g0 == 0.0)
