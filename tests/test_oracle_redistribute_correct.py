"""Pins for oracle.redistribute (Sec. 4.2) and oracle.correct (Sec. 4.3)."""
import numpy as np
import pytest

from oracle.correct import area_length, correct
from oracle.redistribute import redistribute
from oracle.spectral import Geometry, d_alpha, upsample


def _noisy(N, seed=0):
    t = 2 * np.pi * np.arange(N) / N
    rng = np.random.default_rng(seed)
    # uneven parametrisation of a smooth curve
    s = t + 0.3 * np.sin(t) + 0.1 * np.sin(2 * t + rng.uniform())
    return 1.2 * np.cos(s) + 0.05 * np.cos(3 * s), 0.7 * np.sin(s) + 0.03 * np.sin(4 * s)


def test_circle_is_fixed_point():
    N = 32
    t = 2 * np.pi * np.arange(N) / N
    x, y = 0.4 * np.cos(t) + 1, 0.4 * np.sin(t) - 2
    xr, yr, a = redistribute(x, y)
    assert np.max(np.abs(a - t)) < 1e-13
    assert np.max(np.abs(xr - x)) + np.max(np.abs(yr - y)) < 1e-13


@pytest.mark.parametrize("N", [32, 64])
def test_equal_arclength_spacing(N):
    x, y = _noisy(N)
    xr, yr, a = redistribute(x, y)
    # arclength of the ORIGINAL curve at the new parameters, from a 256x finer resampling:
    # the targets must be equally spaced up to the linear-interpolation error
    f = 256
    xu, yu = upsample(x, f), upsample(y, f)
    sp = np.hypot(d_alpha(xu), d_alpha(yu)) * 2 * np.pi / (N * f)
    lf = np.concatenate([[0.0], np.cumsum(0.5 * (sp + np.roll(sp, -1)))])
    af = 2 * np.pi * np.arange(N * f + 1) / (N * f)
    la = np.interp(np.concatenate([a, [2 * np.pi]]), af, lf)
    seg = np.diff(la)
    assert np.max(np.abs(seg / seg.mean() - 1)) < 2e-3  # linear interpolation on the 6N grid
    g0, g1 = Geometry(x, y), Geometry(xr, yr)
    assert abs(g1.length / g0.length - 1) < 5e-4
    assert abs(g1.area / g0.area - 1) < 5e-4
    # before: strongly uneven
    sp0 = sp.reshape(N, f).sum(axis=1)
    assert np.max(np.abs(sp0 / sp0.mean() - 1)) > 0.1


def test_scaled_circle_corrected_back():
    N = 32
    t = 2 * np.pi * np.arange(N) / N
    R = 0.7
    x, y = 1.04 * R * np.cos(t) + 3, 1.04 * R * np.sin(t) - 1
    xc, yc, fired, _ = correct(x, y, np.pi * R * R, 2 * np.pi * R)
    assert fired
    assert np.max(np.abs(np.hypot(xc - 3, yc + 1) - R)) < 1e-13


def test_correction_constraints_and_kkt():
    N = 64
    x, y = _noisy(N, 4)
    A0, L0 = area_length(x, y)
    xp = x * 1.03 + 0.004 * np.sin(5 * 2 * np.pi * np.arange(N) / N)
    yp = y * 0.995
    xc, yc, fired, it = correct(xp, yp, A0, L0)
    assert fired
    A, L = area_length(xc, yc)
    assert abs(A / A0 - 1) < 1e-12 and abs(L / L0 - 1) < 1e-12
    # stationarity: X~ - X lies in span(grad A, grad L) at X~
    dal = 2 * np.pi / N
    xa, ya = d_alpha(xc), d_alpha(yc)
    s = np.hypot(xa, ya)
    gA = dal * np.concatenate([ya, -xa])
    gL = -dal * np.concatenate([d_alpha(xa / s), d_alpha(ya / s)])
    J = np.vstack([gA, gL]).T
    d = np.concatenate([xc - xp, yc - yp])
    lam = np.linalg.lstsq(J, d, rcond=None)[0]
    assert np.linalg.norm(J @ lam - d) < 1e-10 * np.linalg.norm(d)


def test_no_correction_below_trigger():
    N = 32
    x, y = _noisy(N, 5)
    A0, L0 = area_length(x, y)
    xc, yc, fired, _ = correct(x * 1.001, y * 1.001, A0, L0, tol=0.01)
    assert not fired and np.array_equal(xc, x * 1.001)
