"""Pins for oracle.nearfield (Sec. 3.3, Algorithm 4, App. A)."""
import numpy as np
import pytest

from oracle.farfield import far_field
from oracle.nearfield import (LAYERS, layer_points, layer_velocities, near_correction, rbf_eval,
                              rbf_weights)
from oracle.spectral import Geometry, upsample
from oracle.stokes import single_layer_trapezoid


@pytest.mark.parametrize("R", [0.5, 2.0])
def test_circle_layers_constant_density(R):
    # inside a circle the single layer of a constant density is constant, (R/4mu)(1 - 2 log R) F;
    # outside it is (1/4 pi mu)[-2 pi R log rho F + pi R F + pi R (1 - R^2/rho^2) e^{2 i psi} conj F]
    N = 32
    t = 2 * np.pi * np.arange(N) / N
    x, y = R * np.cos(t), R * np.sin(t)
    F = 0.7 - 0.4j
    UX, UY = layer_velocities(x, y, np.full(N, F.real), np.full(N, F.imag), 1.0)
    LX, LY, h = layer_points(x, y)
    U = UX + 1j * UY
    inside = R / 4 * (1 - 2 * np.log(R)) * F
    for k, d in enumerate(LAYERS):
        seg = U[k * N:(k + 1) * N]
        if d <= 0:
            # N^{3/2}-point trapezoid at distance h/2: converges like exp(-pi sqrt(N))
            assert np.max(np.abs(seg - inside)) < 1e-8 * abs(inside)
        else:
            z = LX[k * N:(k + 1) * N] + 1j * LY[k * N:(k + 1) * N]
            rho, psi = np.abs(z), np.angle(z)
            ex = (-2 * np.pi * R * np.log(rho) * F + np.pi * R * F
                  + np.pi * R * (1 - R ** 2 / rho ** 2) * np.exp(2j * psi) * np.conj(F)) / (4 * np.pi)
            assert np.max(np.abs(seg - ex)) < 1e-8 * abs(inside)


def _appendix_shape(N):
    t = 2 * np.pi * np.arange(N) / N
    return 1.0 * np.cos(t) + 0.25 * np.cos(2 * t), 0.55 * np.sin(t) - 0.1 * np.sin(3 * t)


def test_normal_density_gives_zero_layer_velocity():
    # S[n] = 0 for any closed curve; the off-curve layers see the upsampled (interpolated) normal
    x, y = _appendix_shape(128)
    g = Geometry(x, y)
    UX, UY = layer_velocities(x, y, g.nx, g.ny, 1.0)
    # residual = interpolation error of the normal itself (about 1e-7 at N = 128)
    assert np.max(np.abs(UX)) + np.max(np.abs(UY)) < 1e-6


@pytest.mark.parametrize("N,tol", [(32, 4e-2), (64, 1e-2), (128, 1e-2)])
def test_appendix_a_accuracy(N, tol):
    # App. A: density (sin t, cos t), targets on normal lines within one spacing of the curve
    x, y = _appendix_shape(N)
    g = Geometry(x, y)
    t = 2 * np.pi * np.arange(N) / N
    fx, fy = np.sin(t), np.cos(t)
    LX, LY, h = layer_points(x, y)
    WX, WY = rbf_weights(LX, LY, *layer_velocities(x, y, fx, fy, 1.0), h)
    dq = np.linspace(-1, 1, 40) * h
    idx = [3, N // 3, 2 * N // 3 + 1]
    TX = np.concatenate([x[i] + dq * g.nx[i] for i in idx])
    TY = np.concatenate([y[i] + dq * g.ny[i] for i in idx])
    rx, ry = rbf_eval(LX, LY, WX, WY, h, TX, TY)
    up = 128
    ex, ey = single_layer_trapezoid(upsample(x, up), upsample(y, up), upsample(fx, up), upsample(fy, up), TX, TY, 1.0)
    px, py = single_layer_trapezoid(x, y, fx, fy, TX, TY, 1.0)
    scale = np.max(np.hypot(ex, ey))
    err_rbf = np.max(np.hypot(rx - ex, ry - ey)) / scale
    err_trap = np.max(np.hypot(px - ex, py - ey)) / scale
    assert err_rbf < tol
    assert err_trap > 5 * err_rbf


def test_correction_is_linear_in_density_and_matches_mask():
    N = 32
    x0, y0 = _appendix_shape(N)
    g0 = Geometry(x0, y0)
    t = 2 * np.pi * np.arange(N) / N
    x1, y1 = 0.3 * np.cos(t) + x0.max() + 0.3 + 0.6 * g0.h, 0.3 * np.sin(t)
    rng = np.random.default_rng(1)
    f = [rng.standard_normal(N) for _ in range(4)]
    _, _, near = far_field([x0, x1], [y0, y1], [f[0], f[1]], [f[2], f[3]], 1.0)
    assert near
    a = near_correction([x0, x1], [y0, y1], [f[0], f[1]], [f[2], f[3]], 1.0, near)
    b = near_correction([x0, x1], [y0, y1], [2 * f[0], 2 * f[1]], [2 * f[2], 2 * f[3]], 1.0, near)
    assert np.allclose(2 * a[0], b[0], rtol=1e-12, atol=0) and np.allclose(2 * a[1], b[1], rtol=1e-12, atol=0)
    masked = np.zeros(2 * N, dtype=bool)
    masked[[tt for tt, _ in near]] = True
    assert np.all(a[0][~masked] == 0.0) and np.all(np.abs(a[0][masked]) > 0)
