"""Standardisation of a vesicle for the networks (Sec. 3.4.1; Algorithms 2-4). Test infrastructure only.

standardize(X) -> (X^o, params):
1. centre: the area centroid. The paper prints c = int X (X.n) ds / int X.n ds; by the divergence
   theorem the numerator is 3 A xbar and the denominator 2 A, so the printed ratio is 1.5 xbar and
   not translation invariant. Reading: c = (2/3) int X (X.n) ds / int X.n ds = xbar.
2. inertia tensor J = 1/4 int (r.n)(|r|^2 I - r r^T) ds, r = X - c (the paper's boundary form of the
   area integral); principal axis = eigenvector of the smallest eigenvalue, sign chosen so that its
   y component is >= 0 (x > 0 when it is 0); rotate by theta so that the axis lies along +y.
3. scale to unit length (s = 1/L).
4. reorder: the first point is the right-most of the points j with y_{j-1} < 0 <= y_j (an upward
   crossing of the x axis, i.e. on or just above it, points counter-clockwise) -- reading of
   "the first point lies on or just above the x-axis".
The networks see the Fourier-filtered standardised shape: modes |k| > kmax and the Nyquist mode
zeroed (reading; the paper names no cut-off, the library takes kmax as a parameter). Displacements map back with destandardize_disp.
The network input and output are the Fourier coefficients of the standardised shape and of the
relaxation displacement (fourier_features / features_to_samples): a_k = (1/N) sum_j v_j cos(2 pi k j/N),
b_k = -(1/N) sum_j v_j sin(2 pi k j/N), k = 0..K, laid out as [a_0..a_K, b_1..b_K] for x, then for y
(reading: the paper feeds point coordinates to its convolutional networks; coefficients normalised per
mode let a fully connected network resolve the small high modes that the bending force amplifies).

Pins (tests/test_oracle_standardize.py): invariance of X^o to translation, rotation and scaling of
the input; J of an ellipse in closed form; the centroid against the polygon centroid; exact
round trip of points and displacements; the features of single cosine and sine modes in closed
form and the synthesis of features against the FFT low-pass.
"""
import numpy as np

from .spectral import Geometry


def centroid(x, y):
    g = Geometry(x, y)
    w = g.sa * 2.0 * np.pi / g.N
    xn = x * g.nx + y * g.ny
    den = np.sum(xn * w)
    return np.array([np.sum(x * xn * w), np.sum(y * xn * w)]) / (1.5 * den)


def inertia(x, y, c):
    g = Geometry(x, y)
    w = g.sa * 2.0 * np.pi / g.N
    rx, ry = x - c[0], y - c[1]
    rn = rx * g.nx + ry * g.ny
    r2 = rx * rx + ry * ry
    Jxx = 0.25 * np.sum(rn * (r2 - rx * rx) * w)
    Jxy = 0.25 * np.sum(rn * (-rx * ry) * w)
    Jyy = 0.25 * np.sum(rn * (r2 - ry * ry) * w)
    return np.array([[Jxx, Jxy], [Jxy, Jyy]])


def principal_axis(J):
    w, V = np.linalg.eigh(J)
    p = V[:, 0]
    if p[1] < 0 or (p[1] == 0 and p[0] < 0):
        p = -p
    return p


class Params:
    def __init__(self, c, cos_t, sin_t, s, j0):
        self.c, self.cos_t, self.sin_t, self.s, self.j0 = c, cos_t, sin_t, s, j0


def standardize(x, y):
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    c = centroid(x, y)
    p = principal_axis(inertia(x, y, c))
    # rotation R(theta) with R p = e_y: cos t = p_y, sin t = p_x  (R = [[c, -s], [s, c]])
    ct, st = p[1], p[0]
    rx, ry = x - c[0], y - c[1]
    xr, yr = ct * rx - st * ry, st * rx + ct * ry
    s = 1.0 / Geometry(x, y).length
    xr, yr = s * xr, s * yr
    N = len(x)
    cand = [j for j in range(N) if yr[j - 1] < 0 <= yr[j]]
    j0 = max(cand, key=lambda j: xr[j]) if cand else 0
    return np.roll(xr, -j0), np.roll(yr, -j0), Params(c, ct, st, s, j0)


def destandardize_disp(dx, dy, p):
    """Map a displacement field from the standardised frame back to the original points."""
    dx, dy = np.roll(dx, p.j0) / p.s, np.roll(dy, p.j0) / p.s
    return p.cos_t * dx + p.sin_t * dy, -p.sin_t * dx + p.cos_t * dy


def destandardize_points(xo, yo, p):
    ux, uy = destandardize_disp(xo, yo, p)
    return ux + p.c[0], uy + p.c[1]


def to_frame_disp(dx, dy, p):
    """A displacement field of the original points expressed in the standardised frame."""
    rx, ry = p.cos_t * dx - p.sin_t * dy, p.sin_t * dx + p.cos_t * dy
    return np.roll(p.s * rx, -p.j0), np.roll(p.s * ry, -p.j0)


def fourier_filter(v, kmax=None):
    """Zero the modes |k| > kmax (default N/4) and the Nyquist mode of real samples v."""
    N = len(v)
    kmax = N // 4 if kmax is None else min(kmax, N // 2 - 1)
    c = np.fft.fft(v)
    k = np.abs(np.fft.fftfreq(N, d=1.0 / N))
    c[k > kmax] = 0.0
    return np.fft.ifft(c).real


def feature_count(K):
    return 4 * K + 2


def fourier_features(vx, vy, K):
    """[a_0..a_K, b_1..b_K] of vx, then of vy (module header), written out as the DFT sums."""
    N = len(vx)
    j = np.arange(N)
    out = []
    for v in (np.asarray(vx, float), np.asarray(vy, float)):
        a = [np.sum(v * np.cos(2.0 * np.pi * k * j / N)) / N for k in range(K + 1)]
        b = [-np.sum(v * np.sin(2.0 * np.pi * k * j / N)) / N for k in range(1, K + 1)]
        out += a + b
    return np.array(out)


def features_to_samples(f, K, N):
    """The samples v_j = a_0 + 2 sum_{k=1..K} (a_k cos(2 pi k j/N) - b_k sin(2 pi k j/N)) of x and y."""
    j = np.arange(N)
    res = []
    for c in range(2):
        g = f[c * (2 * K + 1):(c + 1) * (2 * K + 1)]
        v = np.full(N, g[0])
        for k in range(1, K + 1):
            v = v + 2.0 * (g[k] * np.cos(2.0 * np.pi * k * j / N) - g[K + k] * np.sin(2.0 * np.pi * k * j / N))
        res.append(v)
    return res[0], res[1]
