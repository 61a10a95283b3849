"""Pins for oracle.spectral (Sec. 2.2.1): exact spectral derivatives, ellipse closed forms,
Frenet identity, circle bending force balanced by tension."""
import numpy as np
import pytest

from oracle.spectral import Geometry, d_alpha, d_alpha_matrix, eval_interpolant, force, upsample, x_ssss


def _alpha(N):
    return 2.0 * np.pi * np.arange(N) / N


@pytest.mark.parametrize("N", [16, 32, 64, 128])
def test_derivative_exact_on_trig_polynomials(N):
    a = _alpha(N)
    rng = np.random.default_rng(0)
    v = np.zeros(N)
    dv = np.zeros(N)
    for k in range(N // 2):
        c, s = rng.standard_normal(2)
        v += c * np.cos(k * a) + s * np.sin(k * a)
        dv += k * (-c * np.sin(k * a) + s * np.cos(k * a))
    assert np.max(np.abs(d_alpha(v) - dv)) < 1e-11 * N


def test_nyquist_mode_dropped_and_matrix_skew():
    N = 16
    a = _alpha(N)
    assert np.max(np.abs(d_alpha(np.cos(N // 2 * a)))) < 1e-13
    D = d_alpha_matrix(N)
    assert np.max(np.abs(D + D.T)) < 1e-13


@pytest.mark.parametrize("a_ax,b_ax", [(2.0, 1.0), (1.3, 0.4)])
def test_ellipse_curvature_area(a_ax, b_ax):
    N = 128
    t = _alpha(N)
    g = Geometry(a_ax * np.cos(t), b_ax * np.sin(t))
    exact = a_ax * b_ax / (a_ax ** 2 * np.sin(t) ** 2 + b_ax ** 2 * np.cos(t) ** 2) ** 1.5
    assert np.max(np.abs(g.curv - exact)) < 1e-7 * exact.max()
    assert abs(g.area - np.pi * a_ax * b_ax) < 1e-13 * np.pi * a_ax * b_ax


def test_length_against_fine_polygon():
    N = 64
    t = _alpha(N)
    g = Geometry(2.0 * np.cos(t), 1.0 * np.sin(t))
    tt = np.linspace(0, 2 * np.pi, 400001)
    ref = np.sum(np.hypot(np.diff(2 * np.cos(tt)), np.diff(np.sin(tt))))
    assert abs(g.length - ref) < 1e-9 * ref


def test_frenet_identity_fourth_derivative():
    # X_ssss = (c_ss - c^3) N_in - 3 c c_s T, N_in the inward normal
    N = 128
    t = _alpha(N)
    x, y = 1.5 * np.cos(t), 0.8 * np.sin(t)
    g = Geometry(x, y)
    bx, by = x_ssss(x, y)
    cs = d_alpha(g.curv) / g.sa
    css = d_alpha(cs) / g.sa
    nin_x, nin_y = -g.ty, g.tx
    ex = (css - g.curv ** 3) * nin_x - 3 * g.curv * cs * g.tx
    ey = (css - g.curv ** 3) * nin_y - 3 * g.curv * cs * g.ty
    scale = np.max(np.abs(ex))
    assert np.max(np.abs(bx - ex)) < 1e-7 * scale
    assert np.max(np.abs(by - ey)) < 1e-7 * scale


@pytest.mark.parametrize("R", [0.5, 2.0])
def test_circle_bending_balanced_by_tension(R):
    N = 32
    t = _alpha(N)
    x, y = R * np.cos(t) + 0.3, R * np.sin(t) - 1.0
    bx, by = x_ssss(x, y)
    # X_ssss = n / R^3 on a circle
    assert np.max(np.abs(bx - np.cos(t) / R ** 3)) < 1e-11 / R ** 3
    kappa = 1.7
    fx, fy = force(x, y, np.full(N, -kappa / R ** 2), kappa)
    assert np.max(np.abs(fx)) + np.max(np.abs(fy)) < 1e-10 * kappa / R ** 3


def test_interpolant_and_upsampling_reproduce_trig_polynomial():
    N = 16
    t = _alpha(N)
    v = 1.0 + np.cos(3 * t) - 0.5 * np.sin(5 * t) + 0.25 * np.cos(8 * t)
    fine = 2 * np.pi * np.arange(6 * N) / (6 * N)
    expect = 1.0 + np.cos(3 * fine) - 0.5 * np.sin(5 * fine) + 0.25 * np.cos(8 * fine)
    assert np.max(np.abs(upsample(v, 6) - expect)) < 1e-13
    assert np.max(np.abs(eval_interpolant(v, fine) - expect)) < 1e-13
