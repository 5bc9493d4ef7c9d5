"""Karhunen-Loeve expansion of the Gaussian field g (Sec. 2.1, Eqs. KLE and
CovarKer2DNLP).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper cites an analytic eigen-solution of the separable exponential
kernel sigma^2 exp(-|x1-x2|/b_x - |y1-y2|/b_y) but the formula itself is
missing from the text.  This module writes out the standard one-dimensional
solution on [-a, a] (a = 1/2, coordinates shifted by 1/2, c = 1/b):

  even modes: theta tan(theta) = a c,  theta in (k pi, k pi + pi/2),
              phi(s) = cos(w s) / sqrt(a + sin(2 w a) / (2 w)),
  odd modes:  theta cot(theta) = -a c, theta in (k pi + pi/2, (k+1) pi),
              phi(s) = sin(w s) / sqrt(a - sin(2 w a) / (2 w)),
  w = theta / a,  lambda_1D = 2 b / (1 + b^2 w^2).

2D pairs: lambda_mn = sigma^2 lambda^x_m lambda^y_n, phi_mn = phi^x_m phi^y_n;
the L largest are kept, ties broken by (m, n) ascending.  Roots are found by
bisection down to a bracket of adjacent doubles.
"""
import math

import numpy as np

HALF = 0.5


def _bisect(f, lo, hi, increasing):
    """Bisection until lo and hi are adjacent doubles; returns the midpoint
    rule's last lower end (the largest x with f(x) on the 'below' side)."""
    while True:
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            return lo
        v = f(mid)
        if (v < 0.0) == increasing:
            lo = mid
        else:
            hi = mid


def eigen_1d(b, count, a=HALF):
    """First `count` 1D eigenpairs of exp(-|s-t|/b) on [-a, a].

    Returns list of (lambda, omega, parity) with parity 0 = cosine (even),
    1 = sine (odd), ordered by lambda descending (omega ascending).
    """
    c = 1.0 / b
    out = []
    for m in range(count):
        k = m // 2
        if m % 2 == 0:
            lo, hi = k * math.pi, k * math.pi + 0.5 * math.pi
            theta = _bisect(lambda t: t * math.tan(t) - a * c, lo, hi, True)
        else:
            lo, hi = k * math.pi + 0.5 * math.pi, (k + 1) * math.pi
            theta = _bisect(lambda t: t / math.tan(t) + a * c, lo, hi, False)
        w = theta / a
        lam = 2.0 * b / (1.0 + b * b * w * w)
        out.append((lam, w, m % 2))
    return out


def phi_1d(mode, s, a=HALF):
    lam, w, parity = mode
    s = np.asarray(s, dtype=np.float64)
    if parity == 0:
        return np.cos(w * s) / math.sqrt(a + math.sin(2.0 * w * a) / (2.0 * w))
    return np.sin(w * s) / math.sqrt(a - math.sin(2.0 * w * a) / (2.0 * w))


def modes_2d(sigma2, bx, by, L):
    """The L leading 2D modes as a list of (lambda, m, n, mode_x, mode_y)."""
    ex = eigen_1d(bx, L)
    ey = eigen_1d(by, L)
    cand = []
    for m in range(L):
        for n in range(L):
            # sigma^2 (lambda_m lambda_n): the 1D product is commutative, so
            # the equal pairs (m, n), (n, m) of b_x = b_y stay exact ties
            lam = sigma2 * (ex[m][0] * ey[n][0])
            cand.append((-lam, m, n))
    cand.sort()
    return [(-nl, m, n, ex[m], ey[n]) for (nl, m, n) in cand[:L]]


def field_modes(sigma2, bx, by, L, x, y):
    """g_i(x, y) = sqrt(lambda_i) phi_i(x, y) for i < L, shape [L, len(x)]."""
    out = np.empty((L, len(x)))
    for i, (lam, m, n, mx, my) in enumerate(modes_2d(sigma2, bx, by, L)):
        out[i] = math.sqrt(lam) * phi_1d(mx, np.asarray(x) - HALF) * phi_1d(my, np.asarray(y) - HALF)
    return out


def nystrom_1d(b, npts=2000, a=HALF):
    """Eigenvalues of exp(-|s-t|/b) on [-a, a] by Gauss-Legendre Nystrom
    (an independent discretisation used only to pin eigen_1d)."""
    xg, wg = np.polynomial.legendre.leggauss(npts)
    s = a * xg
    w = a * wg
    Kmat = np.exp(-np.abs(s[:, None] - s[None, :]) / b)
    sw = np.sqrt(w)
    ev, evec = np.linalg.eigh(sw[:, None] * Kmat * sw[None, :])
    order = np.argsort(ev)[::-1]
    return ev[order], s, evec[:, order] / sw[:, None]
