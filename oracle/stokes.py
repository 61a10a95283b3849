"""2D Stokeslet and single-layer quadratures (Eqs. single_layer, Stokeslet; Sec. 2.2.2).

Test infrastructure only.

Readings:
* Stokeslet sign. Eq. Stokeslet prints (1/4 pi mu)(log|r| + r r^T/|r|^2) with no identity on
  the log term. We use the standard free-space kernel (1/4 pi mu)(-log|r| I + r r^T/|r|^2);
  the printed sign would make a point force drive the nearby fluid against itself.
* Self (log-singular) rule. The paper uses Alpert's hybrid Gauss-trapezoid rule whose node
  tables it does not print. We use Kress's spectrally accurate product rule for the
  logarithmic kernel: with N = 2n and t_j = 2 pi j / N,
      int_0^{2pi} log(4 sin^2((t - tau)/2)) phi(tau) dtau ~ sum_j R(t - t_j) phi(t_j),
      R(d) = -(2 pi/n) sum_{m=1}^{n-1} cos(m d)/m - (pi/n^2) cos(n d),
  obtained from log(4 sin^2(s/2)) = -2 sum_{m>=1} cos(m s)/m applied to the interpolant.
  -log|r| is split as -1/2 log(4 sin^2((t-tau)/2)) - 1/2 log(|r|^2 / (4 sin^2((t-tau)/2)));
  the second part is smooth (diagonal limit -log|X_alpha|) and takes trapezoid weights, as
  does r r^T/|r|^2 (diagonal limit X_s X_s^T).

Pins (tests/test_oracle_stokes.py): closed-form single layer of every Fourier mode on a
circle (on-curve), closed form outside a circle for constant density, S[n] = 0 on any
closed curve, zero net flux of the single-layer velocity through the curve.
"""
import numpy as np

from .spectral import Geometry


def stokeslet(rx, ry, mu):
    """Components (Gxx, Gxy, Gyy) of (1/4 pi mu)(-log|r| I + r r^T/|r|^2)."""
    r2 = rx * rx + ry * ry
    c = 1.0 / (4.0 * np.pi * mu)
    lg = -0.5 * np.log(r2)
    return c * (lg + rx * rx / r2), c * (rx * ry / r2), c * (lg + ry * ry / r2)


def kress_weights(N):
    """R(2 pi d / N) for d = 0..N-1 (Kress product rule for the log kernel, N = 2n)."""
    n = N // 2
    d = np.arange(N)
    t = 2.0 * np.pi * d / N
    R = np.zeros(N)
    for m in range(1, n):
        R -= (2.0 * np.pi / n) * np.cos(m * t) / m
    R -= (np.pi / n ** 2) * np.cos(n * t)
    return R


def self_single_layer_matrix(x, y, mu):
    """Dense 2N x 2N matrix S with [u_x; u_y] = S @ [f_x; f_y] on the curve itself.

    u(X_i) = int G(X_i - X(tau)) f(tau) |X_alpha(tau)| dtau (Eq. single_layer) with the
    Kress rule for the log part and trapezoid weights for the rest (module header).
    """
    g = Geometry(x, y)
    N = g.N
    i = np.arange(N)[:, None]
    j = np.arange(N)[None, :]
    d = (i - j) % N
    R = kress_weights(N)[d]
    rx = g.x[:, None] - g.x[None, :]
    ry = g.y[:, None] - g.y[None, :]
    r2 = rx * rx + ry * ry
    off = d != 0
    sin2 = 4.0 * np.sin(np.pi * d / N) ** 2
    dal = 2.0 * np.pi / N
    logpart = np.empty((N, N))
    rxx = np.empty((N, N))
    rxy = np.empty((N, N))
    ryy = np.empty((N, N))
    logpart[off] = -0.5 * R[off] - 0.5 * dal * np.log(r2[off] / sin2[off])
    rxx[off] = rx[off] ** 2 / r2[off]
    rxy[off] = rx[off] * ry[off] / r2[off]
    ryy[off] = ry[off] ** 2 / r2[off]
    diag = np.arange(N)
    logpart[diag, diag] = -0.5 * R[diag, diag] - dal * np.log(g.sa)
    rxx[diag, diag] = g.tx ** 2
    rxy[diag, diag] = g.tx * g.ty
    ryy[diag, diag] = g.ty ** 2
    c = 1.0 / (4.0 * np.pi * mu)
    w = g.sa[None, :]
    S = np.zeros((2 * N, 2 * N))
    S[:N, :N] = c * w * (logpart + dal * rxx)
    S[:N, N:] = c * w * (dal * rxy)
    S[N:, :N] = c * w * (dal * rxy)
    S[N:, N:] = c * w * (logpart + dal * ryy)
    return S


def single_layer_trapezoid(xs, ys, fx, fy, tx, ty, mu):
    """Trapezoid-rule single layer of one closed curve at target points (Sec. 2.2.2).

    u(t) = sum_j G(t - X_j) f_j |X_alpha|_j (2 pi / N), the far-field rule of the paper.
    """
    g = Geometry(xs, ys)
    w = g.sa * 2.0 * np.pi / g.N
    tx = np.atleast_1d(np.asarray(tx, dtype=np.float64))
    ty = np.atleast_1d(np.asarray(ty, dtype=np.float64))
    rx = tx[:, None] - g.x[None, :]
    ry = ty[:, None] - g.y[None, :]
    gxx, gxy, gyy = stokeslet(rx, ry, mu)
    ux = (gxx * (fx * w)[None, :] + gxy * (fy * w)[None, :]).sum(axis=1)
    uy = (gxy * (fx * w)[None, :] + gyy * (fy * w)[None, :]).sum(axis=1)
    return ux, uy
