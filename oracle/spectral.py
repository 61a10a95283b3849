"""Spectral discretisation of one closed curve (Sec. 2.2.1). Test infrastructure only.

A vesicle is N points X_j = (x_j, y_j) at alpha_j = 2*pi*j/N, j = 0..N-1, counter-clockwise.
Its parametrisation is the trigonometric interpolant with modes -N/2+1..N/2 (Sec. 2.2.1).

Readings (the paper is silent on these):
* the Nyquist mode N/2 is dropped from every first derivative, so d/dalpha is a real skew
  circulant; higher derivatives are repeated first derivatives with the 1/|X_alpha| metric
  applied each time, as d/ds = |X_alpha|^{-1} d/dalpha prescribes (Sec. 2.2.1);
* evaluated between grid points, the interpolant carries half the Nyquist coefficient on
  cos(N alpha/2), which keeps it real.

Pins (tests/test_oracle_geometry.py): exact derivatives of trigonometric polynomials, ellipse
curvature and area closed forms, Frenet identity for X_ssss, length against a fine reference.
"""
import numpy as np


def wavenumbers(N):
    """Integer wavenumbers in FFT order with the Nyquist entry set to zero."""
    k = np.fft.fftfreq(N, d=1.0 / N)
    k[N // 2] = 0.0
    return k


def d_alpha(v):
    """d/dalpha of real periodic samples along the last axis (Sec. 2.2.1)."""
    v = np.asarray(v, dtype=np.float64)
    N = v.shape[-1]
    return np.fft.ifft(1j * wavenumbers(N) * np.fft.fft(v, axis=-1), axis=-1).real


def d_alpha_matrix(N):
    """Dense N x N real matrix D with D @ v == d_alpha(v)."""
    return d_alpha(np.eye(N)).T


def d_s(v, sa):
    """Arclength derivative d/ds = |X_alpha|^{-1} d/dalpha (Sec. 2.2.1)."""
    return d_alpha(v) / sa


class Geometry:
    """Per-vesicle geometric quantities at the N material points.

    sa = |X_alpha|, (tx, ty) = X_s, outward normal n = (ty, -tx) for a counter-clockwise
    curve, curvature c = x_s y_ss - y_s x_ss, area by the discrete Green formula, length
    by the periodic trapezoid rule of |X_alpha|, arclength spacing h = L / N (Sec. 2.2).
    """

    def __init__(self, x, y):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        N = x.shape[-1]
        self.N = N
        self.x, self.y = x, y
        self.xa, self.ya = d_alpha(x), d_alpha(y)
        self.sa = np.sqrt(self.xa ** 2 + self.ya ** 2)
        self.tx, self.ty = self.xa / self.sa, self.ya / self.sa
        self.nx, self.ny = self.ty, -self.tx
        self.xss, self.yss = d_s(self.tx, self.sa), d_s(self.ty, self.sa)
        self.curv = self.tx * self.yss - self.ty * self.xss
        dal = 2.0 * np.pi / N
        self.area = dal * np.sum(0.5 * (x * self.ya - y * self.xa))
        self.length = dal * np.sum(self.sa)
        self.h = self.length / N


def x_ssss(x, y):
    """Fourth arclength derivative of each coordinate, D_s applied four times (Eq. elastic_force)."""
    g = Geometry(x, y)
    out = []
    for v in (x, y):
        w = v
        for _ in range(4):
            w = d_s(w, g.sa)
        out.append(w)
    return out[0], out[1]


def force(x, y, sigma, kappa):
    """Membrane force f = -kappa X_ssss + (sigma X_s)_s (Eq. elastic_force).

    (sigma X_s)_s is read literally: D_s applied to the product sigma * X_s.
    """
    g = Geometry(x, y)
    bx, by = x_ssss(x, y)
    fx = -kappa * bx + d_s(sigma * g.tx, g.sa)
    fy = -kappa * by + d_s(sigma * g.ty, g.sa)
    return fx, fy


def bending_energy(x, y, kappa):
    """E_b = kappa/2 * int c^2 ds (Sec. 5.2), periodic trapezoid rule."""
    g = Geometry(x, y)
    return 0.5 * kappa * np.sum(g.curv ** 2 * g.sa) * 2.0 * np.pi / g.N


def interpolant_coeffs(v):
    """Fourier coefficients of the real trigonometric interpolant of samples v (length N)."""
    return np.fft.fft(np.asarray(v, dtype=np.float64)) / v.shape[-1]


def eval_interpolant(v, alpha):
    """Evaluate the trigonometric interpolant of samples v at arbitrary parameters alpha.

    Modes -N/2+1..N/2-1 plus half the Nyquist coefficient on each of +-N/2 (real-valued).
    Direct O(N * len(alpha)) sum.
    """
    v = np.asarray(v, dtype=np.float64)
    N = v.shape[-1]
    c = interpolant_coeffs(v)
    alpha = np.asarray(alpha, dtype=np.float64)
    out = np.full(alpha.shape, c[0].real)
    for k in range(1, N // 2):
        ck = c[k]
        out = out + 2.0 * (ck.real * np.cos(k * alpha) - ck.imag * np.sin(k * alpha))
    out = out + c[N // 2].real * np.cos((N // 2) * alpha)
    return out


def upsample(v, factor):
    """Samples of the trigonometric interpolant of v on a grid `factor` times finer (zero padding)."""
    v = np.asarray(v, dtype=np.float64)
    N = v.shape[-1]
    Nu = N * factor
    c = np.fft.fft(v)
    cu = np.zeros(Nu, dtype=np.complex128)
    cu[: N // 2] = c[: N // 2]
    cu[Nu - N // 2 + 1:] = c[N // 2 + 1:]
    cu[N // 2] = 0.5 * c[N // 2]
    cu[Nu - N // 2] = 0.5 * c[N // 2]
    return np.fft.ifft(cu).real * factor
