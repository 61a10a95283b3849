"""Pins for oracle.flows (Sec. 5.3, 5.4, Eq. tayGreenFlow): what each background flow must satisfy,
checked by finite differences and at special points rather than by re-evaluating its formula."""
import numpy as np

from oracle.flows import POISEUILLE, SHEAR, TAYLOR_GREEN, background


def _grad(kind, p, x, y, h=1e-6):
    ux1, uy1 = background(kind, p, x + h, y)
    ux0, uy0 = background(kind, p, x - h, y)
    vx1, vy1 = background(kind, p, x, y + h)
    vx0, vy0 = background(kind, p, x, y - h)
    return (ux1 - ux0) / (2 * h), (uy1 - uy0) / (2 * h), (vx1 - vx0) / (2 * h), (vy1 - vy0) / (2 * h)


def test_every_flow_is_divergence_free():
    rng = np.random.default_rng(0)
    x, y = rng.uniform(-2, 2, 50), rng.uniform(-0.4, 0.4, 50)
    for kind, p in ((SHEAR, (0.7,)), (TAYLOR_GREEN, (1.3, 2.0)), (POISEUILLE, (5.0, 0.5))):
        dux_dx, _, _, duy_dy = _grad(kind, p, x, y)
        assert np.max(np.abs(dux_dx + duy_dy)) <= 1e-6 * max(1.0, p[0])


def test_shear_rate_and_poiseuille_profile():
    # shear: du_x/dy equals the rate everywhere; Poiseuille: no slip at y = +-W, u_max on the axis,
    # wall shear rate 2 u_max / W
    _, _, dux_dy, _ = _grad(SHEAR, (0.7,), np.array([0.3]), np.array([-1.1]))
    assert abs(dux_dy[0] - 0.7) <= 1e-8
    umax, W = 5.0, 0.5
    ux, uy = background(POISEUILLE, (umax, W), np.array([1.0, 1.0, 1.0]), np.array([-W, 0.0, W]))
    assert np.allclose(ux, [0.0, umax, 0.0], atol=1e-14) and np.all(uy == 0.0)
    _, _, dux_dy, _ = _grad(POISEUILLE, (umax, W), np.array([0.0]), np.array([-W]))
    assert abs(dux_dy[0] - 2 * umax / W) <= 1e-6 * umax / W


def test_taylor_green_cell_structure():
    # stagnation points at the cell corners, the centre of a cell at (W/2, W/2) is a vortex centre with
    # zero velocity, and the speed is U at (W/2, 0)
    U, W = 1.3, 2.0
    ux, uy = background(TAYLOR_GREEN, (U, W), np.array([0.0, W, W / 2]), np.array([0.0, W, W / 2]))
    assert np.max(np.abs(ux)) <= 1e-14 and np.max(np.abs(uy)) <= 1e-14
    ux, uy = background(TAYLOR_GREEN, (U, W), np.array([W / 2]), np.array([0.0]))
    assert abs(ux[0] - U) <= 1e-14 and abs(uy[0]) <= 1e-14
