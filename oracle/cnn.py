"""FP64 reference of the learned smoother: a 5-layer 3x3 convolutional
network applied to every PCE mode image of a residual.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Not in the paper (the method statement adds it in place of the mean-based
block solve): parity with the paper is unpinned; the gradients below are
pinned by central differences.  Two training losses: the relative squared
error ||zhat - z*||^2 / ||z*||^2, and the same error in the energy norm of
A_0 (weights the oscillatory error a smoother must remove).

Network: channels 2 -> 32 -> 32 -> 32 -> 32 -> 1, 3x3 kernels, zero padding
1, bias, ReLU after the first four layers.  Input channel 0 is the residual
mode image divided by its RMS, channel 1 is log(a_rr / 4) with a_rr the
diagonal of A_0 (the mean coefficient seen by node r); the output is
multiplied back by the RMS.  Weights are stored [layer]: W [3, 3, Cin, Cout]
(tap-major), b [Cout].  Images are [batch, H, W, C] (channels last).
"""
import numpy as np

CHANNELS = (2, 32, 32, 32, 32, 1)


def conv3x3(x, W, b):
    """y[n,i,j,co] = b[co] + sum_{dy,dx,ci} W[dy,dx,ci,co] x[n,i+dy-1,j+dx-1,ci]
    with zero padding (plain definition, loop over the 9 taps)."""
    n, H, Wd, ci = x.shape
    co = W.shape[3]
    xp = np.zeros((n, H + 2, Wd + 2, ci))
    xp[:, 1:-1, 1:-1, :] = x
    y = np.broadcast_to(b, (n, H, Wd, co)).copy()
    for dy in range(3):
        for dx in range(3):
            y += xp[:, dy:dy + H, dx:dx + Wd, :] @ W[dy, dx]
    return y


def forward(params, x):
    """Returns the output and the list of layer inputs (for backward)."""
    acts = [x]
    h = x
    for l, (W, b) in enumerate(params):
        h = conv3x3(h, W, b)
        if l < len(params) - 1:
            h = np.maximum(h, 0.0)
        acts.append(h)
    return h, acts


def backward(params, acts, dy):
    """Gradients of a scalar loss given dL/d(output) = dy.  Returns
    [(dW, db)] per layer and dL/dx."""
    grads = [None] * len(params)
    g = dy
    for l in range(len(params) - 1, -1, -1):
        W, b = params[l]
        x = acts[l]
        if l < len(params) - 1:
            g = g * (acts[l + 1] > 0.0)          # ReLU of layer l's output
        n, H, Wd, ci = x.shape
        xp = np.zeros((n, H + 2, Wd + 2, ci))
        xp[:, 1:-1, 1:-1, :] = x
        dW = np.zeros_like(W)
        for dy_ in range(3):
            for dx_ in range(3):
                dW[dy_, dx_] = np.einsum("nhwi,nhwo->io", xp[:, dy_:dy_ + H, dx_:dx_ + Wd, :], g)
        db = g.sum(axis=(0, 1, 2))
        # dL/dx: correlation of g with the flipped kernel
        gp = np.zeros((n, H + 2, Wd + 2, g.shape[3]))
        gp[:, 1:-1, 1:-1, :] = g
        dx = np.zeros_like(x)
        for dy_ in range(3):
            for dx_ in range(3):
                dx += gp[:, 2 - dy_:2 - dy_ + H, 2 - dx_:2 - dx_ + Wd, :] @ W[dy_, dx_].T
        grads[l] = (dW, db)
        g = dx
    return grads, g


def loss(zhat, zstar):
    """sum over images of ||zhat - z*||^2 / ||z*||^2, and its gradient."""
    num = np.sum((zhat - zstar) ** 2, axis=(1, 2, 3))
    den = np.sum(zstar ** 2, axis=(1, 2, 3))
    L = np.sum(num / den)
    return L, 2.0 * (zhat - zstar) / den[:, None, None, None]


def loss_energy(zhat, zstar, A0):
    """sum over images of (e^T A_0 e) / (z*^T A_0 z*), e = zhat - z*: the
    squared error in the energy norm of the SPD mean matrix A_0 (images
    [batch, m, m, 1] in node order), and its gradient 2 A_0 e / (z*^T A_0 z*)."""
    nb = zhat.shape[0]
    e = (zhat - zstar).reshape(nb, -1)
    z = zstar.reshape(nb, -1)
    Ae = (A0 @ e.T).T
    Az = (A0 @ z.T).T
    num = np.sum(e * Ae, axis=1)
    den = np.sum(z * Az, axis=1)
    L = np.sum(num / den)
    return L, (2.0 * Ae / den[:, None]).reshape(zhat.shape)


def he_init(rng):
    """He-normal weights (std sqrt(2 / fan_in)), zero biases."""
    params = []
    for l in range(5):
        ci, co = CHANNELS[l], CHANNELS[l + 1]
        W = rng.standard_normal((3, 3, ci, co)) * np.sqrt(2.0 / (9 * ci))
        params.append((W, np.zeros(co)))
    return params


def features(R, diag, N):
    """Network input of a residual block R [n, P] (mode-major columns) on the
    (N-1) x (N-1) grid: channel 0 = r_a / rms(r_a), channel 1 = log(diag/4).
    Returns x [P, m, m, 2] and the per-mode RMS."""
    m = N - 1
    P = R.shape[1]
    rms = np.sqrt(np.mean(R ** 2, axis=0))
    safe = np.where(rms > 0, rms, 1.0)
    x = np.zeros((P, m, m, 2))
    x[..., 0] = (R / safe).T.reshape(P, m, m)
    x[..., 1] = np.log(diag / 4.0).reshape(m, m)[None]
    return x, rms


def smoother_apply(params, R, diag, N):
    """z_a = rms(r_a) * CNN(x_a) for every mode (the learned local solve)."""
    x, rms = features(R, diag, N)
    y, _ = forward(params, x)
    P = R.shape[1]
    return (y[..., 0].reshape(P, -1) * rms[:, None]).T


def adam_step(params, grads, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """Adam (Kingma and Ba) on every weight and bias; state holds (t, m, v)."""
    t, ms, vs = state
    t += 1
    out, new_m, new_v = [], [], []
    for (W, b), (dW, db), (mW, mb), (vW, vb) in zip(params, grads, ms, vs):
        p_new = []
        m_pair, v_pair = [], []
        for p, g, m_, v_ in ((W, dW, mW, vW), (b, db, mb, vb)):
            m_ = b1 * m_ + (1 - b1) * g
            v_ = b2 * v_ + (1 - b2) * g * g
            mhat = m_ / (1 - b1 ** t)
            vhat = v_ / (1 - b2 ** t)
            p_new.append(p - lr * mhat / (np.sqrt(vhat) + eps))
            m_pair.append(m_)
            v_pair.append(v_)
        out.append(tuple(p_new))
        new_m.append(tuple(m_pair))
        new_v.append(tuple(v_pair))
    return out, (t, new_m, new_v)


def adam_init(params):
    zeros = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
    return (0, zeros, [(np.zeros_like(W), np.zeros_like(b)) for W, b in params])
