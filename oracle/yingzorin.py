"""Near-singular evaluation of the single layer by the scheme of Ying and Zorin (Sec. 2.2.2, the caption of
Fig. fig:near-singular: the numerical near-singular integration of the paper's BIEM ground truth). Test
infrastructure only.

For a target x within the near zone of a source vesicle (distance to its points at most h = L/N):
1. the closest point x0 = X(alpha0) of the curve's trigonometric interpolant: Newton's method on
   g(alpha) = (X(alpha) - x) . X'(alpha) = 0 from the nearest of the N points;
2. the single layer at x0: the on-curve values S[X, f] at the N points (the self rule, oracle.stokes)
   evaluated at alpha0 by their trigonometric interpolant (the caption's interpolation along the membrane);
3. the single layer at x_i = x0 + s i beta h n(alpha0), i = 1..m, on the side of x (s the sign of
   (x - x0) . n), by the trapezoid rule on the curve upsampled by ceil(sqrt(N)) (N^{3/2} points);
4. the interpolating polynomial through (i beta h, u_i), i = 0..m, evaluated at t = |x - x0|.
Readings: the paper gives neither m nor beta, and its caption places the interpolation points outside the
near zone. We take m = 6 and beta = 1/4 (points from a quarter to one and a half spacings): with N^{3/2}
upsampling the trapezoid rule is already accurate a quarter spacing from the curve (its error falls like
exp(-2 pi rho t / h)), and a short span keeps the polynomial accurate where the vesicle bends on the scale of
a few spacings. On the curve of App. A (density (sin t, cos t)), at targets within one spacing, the largest
error relative to the largest velocity is 2.1e-4 (N = 32), 4.3e-6 (N = 64) and 7.4e-6 (N = 128); with points
at h, 2h, ..., 5h it was 4.5e-3, 1.4e-3 and 1.0e-3 (tests/test_oracle_yingzorin.py).

Pins (tests/test_oracle_yingzorin.py): circle closed forms inside and outside, the App. A accuracy above,
the closest point against brute force on a fine sampling, linearity in the density.
"""
import math

import numpy as np

from .spectral import Geometry, eval_interpolant, upsample
from .stokes import self_single_layer_matrix, single_layer_trapezoid

YZ_M = 6
YZ_BETA = 0.25


def _curve_at(cx, cy, alpha):
    """X, X', X'' of the trigonometric interpolant with coefficients (np.fft / N) at alpha."""
    N = len(cx)
    k = np.fft.fftfreq(N, d=1.0 / N)
    k[N // 2] = 0.0  # the Nyquist mode is dropped from derivatives (its value term is kept below)
    e = np.exp(1j * k * alpha)
    out = []
    for c in (cx, cy):
        # the value: all modes, the Nyquist coefficient as a cosine (k[N//2] = 0 puts it in the sum as a
        # constant, which the correction below replaces)
        v = np.real(np.sum(c * e)) - np.real(c[N // 2]) + np.real(c[N // 2]) * math.cos(N // 2 * alpha)
        d1 = np.real(np.sum(1j * k * c * e))
        d2 = np.real(np.sum(-(k ** 2) * c * e))
        out.append((v, d1, d2))
    return out


def closest_point(x, y, px, py, iters=30):
    """alpha0 of the point of the interpolant of (x, y) closest to (px, py)."""
    N = len(x)
    cx, cy = np.fft.fft(x) / N, np.fft.fft(y) / N
    j = int(np.argmin((x - px) ** 2 + (y - py) ** 2))
    a = 2.0 * np.pi * j / N
    for _ in range(iters):
        (X, X1, X2), (Y, Y1, Y2) = _curve_at(cx, cy, a)
        g = (X - px) * X1 + (Y - py) * Y1
        gp = X1 * X1 + Y1 * Y1 + (X - px) * X2 + (Y - py) * Y2
        step = g / gp
        a -= step
        if abs(step) < 1e-15:
            break
    return a


def single_layer_near(x, y, fx, fy, mu, tx, ty, m=YZ_M, beta=YZ_BETA):
    """S[X, f] at the targets (tx, ty), all within the near zone of the curve (x, y) (module header)."""
    N = len(x)
    g = Geometry(x, y)
    h = g.h
    u0 = self_single_layer_matrix(x, y, mu) @ np.concatenate([fx, fy])
    rho = int(math.ceil(math.sqrt(N)))
    xu, yu, fxu, fyu = upsample(x, rho), upsample(y, rho), upsample(fx, rho), upsample(fy, rho)
    cx, cy = np.fft.fft(x) / N, np.fft.fft(y) / N
    nodes = beta * h * np.arange(m + 1)
    ox, oy = np.zeros(len(tx)), np.zeros(len(tx))
    for q, (px, py) in enumerate(zip(tx, ty)):
        a = closest_point(x, y, px, py)
        (X, X1, _), (Y, Y1, _) = _curve_at(cx, cy, a)
        sp = math.hypot(X1, Y1)
        nx, ny = Y1 / sp, -X1 / sp
        s = 1.0 if (px - X) * nx + (py - Y) * ny >= 0 else -1.0
        t = math.hypot(px - X, py - Y)
        vx = [eval_interpolant(u0[:N], np.array([a]))[0]]
        vy = [eval_interpolant(u0[N:], np.array([a]))[0]]
        lx = X + s * nodes[1:] * nx
        ly = Y + s * nodes[1:] * ny
        ax, ay = single_layer_trapezoid(xu, yu, fxu, fyu, lx, ly, mu)
        vx += list(ax)
        vy += list(ay)
        # Lagrange form of the interpolating polynomial at t
        for i in range(m + 1):
            w = 1.0
            for j in range(m + 1):
                if j != i:
                    w *= (t - nodes[j]) / (nodes[i] - nodes[j])
            ox[q] += w * vx[i]
            oy[q] += w * vy[i]
    return ox, oy


def near_correction_yz(xs, ys, fxs, fys, mu, near_pairs, m=YZ_M, beta=YZ_BETA):
    """As oracle.nearfield.near_correction, with the single layer of each near (target, source vesicle) pair
    evaluated by this scheme."""
    P = sum(len(x) for x in xs)
    X = np.concatenate(xs)
    Y = np.concatenate(ys)
    cx = np.zeros(P)
    cy = np.zeros(P)
    by_src = {}
    for t, v in near_pairs:
        by_src.setdefault(v, []).append(t)
    for v, targets in sorted(by_src.items()):
        t = np.array(targets)
        ax, ay = single_layer_near(xs[v], ys[v], fxs[v], fys[v], mu, X[t], Y[t], m, beta)
        np.add.at(cx, t, ax)
        np.add.at(cy, t, ay)
    return cx, cy
