"""Pins of the oracle's CNN smoother (CPU): the convolution against a
direct 2D correlation, gradients against central differences, the Adam step
against its closed form on a quadratic."""
import numpy as np
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
