"""Pins for oracle.yingzorin (Sec. 2.2.2, Fig. fig:near-singular: the near-singular scheme of the paper's
BIEM ground truth): closed forms of a circle on both sides of the curve, the App. A accuracy against the
exact integral (far better than the five-layer RBF), the closest point against brute force, linearity."""
import numpy as np
import pytest

from oracle.nearfield import layer_points, layer_velocities, rbf_eval, rbf_weights
from oracle.spectral import Geometry, eval_interpolant, upsample
from oracle.stokes import single_layer_trapezoid
from oracle.yingzorin import closest_point, single_layer_near


@pytest.mark.parametrize("R", [0.5, 2.0])
def test_circle_constant_density_both_sides(R):
    # inside: (R/4mu)(1 - 2 log R) F; outside: (1/4 pi mu)[-2 pi R log rho F + pi R F + pi R (1 - R^2/rho^2)
    # e^{2 i psi} conj F], at targets within one spacing of the circle
    N = 32
    t = 2 * np.pi * np.arange(N) / N
    x, y = R * np.cos(t), R * np.sin(t)
    F = 0.7 - 0.4j
    h = 2 * np.pi * R / N
    rng = np.random.default_rng(1)
    psi = rng.uniform(0, 2 * np.pi, 24)
    rho = R + rng.uniform(-1, 1, 24) * h
    z = rho * np.exp(1j * psi)
    ux, uy = single_layer_near(x, y, np.full(N, F.real), np.full(N, F.imag), 1.0, z.real, z.imag)
    U = ux + 1j * uy
    inside = R / 4 * (1 - 2 * np.log(R)) * F
    outside = (-2 * np.pi * R * np.log(rho) * F + np.pi * R * F
               + np.pi * R * (1 - R ** 2 / rho ** 2) * np.exp(2j * psi) * np.conj(F)) / (4 * np.pi)
    ex = np.where(rho < R, inside, outside)
    # N = 32: the interpolation points a quarter spacing off the curve see the 192-point trapezoid rule to
    # about 1e-5 (exp(-2 pi rho / 4), rho = 6)
    assert np.max(np.abs(U - ex)) <= 5e-5 * np.max(np.abs(ex))


def _appendix_shape(N):
    t = 2 * np.pi * np.arange(N) / N
    return 1.0 * np.cos(t) + 0.25 * np.cos(2 * t), 0.55 * np.sin(t) - 0.1 * np.sin(3 * t)


@pytest.mark.parametrize("N,tol", [(32, 5e-4), (64, 1e-5), (128, 2e-5)])
def test_appendix_a_accuracy(N, tol):
    # App. A: density (sin t, cos t), targets on normal lines within one spacing of the curve, against the
    # trapezoid rule on the curve upsampled 128 times; the five-layer RBF scheme is far less accurate
    x, y = _appendix_shape(N)
    g = Geometry(x, y)
    t = 2 * np.pi * np.arange(N) / N
    fx, fy = np.sin(t), np.cos(t)
    dq = np.linspace(-1, 1, 40) * g.h
    idx = [3, N // 3, 2 * N // 3 + 1]
    TX = np.concatenate([x[i] + dq * g.nx[i] for i in idx])
    TY = np.concatenate([y[i] + dq * g.ny[i] for i in idx])
    up = 128
    ex, ey = single_layer_trapezoid(upsample(x, up), upsample(y, up), upsample(fx, up), upsample(fy, up), TX, TY, 1.0)
    scale = np.max(np.hypot(ex, ey))
    yx, yy = single_layer_near(x, y, fx, fy, 1.0, TX, TY)
    err = np.max(np.hypot(yx - ex, yy - ey)) / scale
    LX, LY, h = layer_points(x, y)
    WX, WY = rbf_weights(LX, LY, *layer_velocities(x, y, fx, fy, 1.0), h)
    rx, ry = rbf_eval(LX, LY, WX, WY, h, TX, TY)
    err_rbf = np.max(np.hypot(rx - ex, ry - ey)) / scale
    print("App. A, N=%d: Ying-Zorin %.2e, five-layer RBF %.2e" % (N, err, err_rbf))
    assert err <= tol
    assert err_rbf >= 20 * err


def test_closest_point_against_brute_force():
    x, y = _appendix_shape(48)
    g = Geometry(x, y)
    rng = np.random.default_rng(2)
    fine = np.linspace(0, 2 * np.pi, 200001)[:-1]
    fx, fy = eval_interpolant(x, fine), eval_interpolant(y, fine)
    for _ in range(8):
        j = int(rng.integers(48))
        d = rng.uniform(-1, 1) * g.h
        px, py = x[j] + d * g.nx[j] + 0.3 * g.h * g.tx[j], y[j] + d * g.ny[j] + 0.3 * g.h * g.ty[j]
        a = closest_point(x, y, px, py)
        b = fine[np.argmin((fx - px) ** 2 + (fy - py) ** 2)]
        assert abs((a - b + np.pi) % (2 * np.pi) - np.pi) <= 2 * np.pi / 200000
        # the closest point: the gradient of the distance vanishes there
        xa, ya = eval_interpolant(x, np.array([a]))[0], eval_interpolant(y, np.array([a]))[0]
        assert np.hypot(xa - px, ya - py) <= np.min(np.hypot(fx - px, fy - py)) + 1e-12


def test_linear_in_density():
    x, y = _appendix_shape(32)
    g = Geometry(x, y)
    rng = np.random.default_rng(3)
    f1 = rng.standard_normal((2, 32))
    f2 = rng.standard_normal((2, 32))
    TX = x[[2, 9, 20]] + 0.4 * g.h * g.nx[[2, 9, 20]]
    TY = y[[2, 9, 20]] + 0.4 * g.h * g.ny[[2, 9, 20]]
    a = np.array(single_layer_near(x, y, *(0.3 * f1 - 1.7 * f2), 1.0, TX, TY))
    b = 0.3 * np.array(single_layer_near(x, y, *f1, 1.0, TX, TY)) - 1.7 * np.array(single_layer_near(x, y, *f2, 1.0, TX, TY))
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))
