"""Pins for oracle.step (Algorithm 1, Eqs. advection_disc, relaxation_disc, tension_disc)."""
import numpy as np
import pytest

from oracle.correct import area_length
from oracle.spectral import bending_energy
from oracle.step import Params, Suspension
from paper_2606_25569_b300.workloads import vesicle_outline


def _ves(N, seed, cx=0.0, cy=0.0, R=1.0, nu=0.7, theta=0.3):
    rng = np.random.default_rng(seed)
    x, y = vesicle_outline(N, nu, R, 5e-2, rng, theta)
    return x + cx, y + cy


def test_relaxation_energy_decreases():
    # Sec. 5.2: a vesicle in a quiescent fluid relaxes and its bending energy decays
    x, y = _ves(32, 0)
    s = Suspension([x], [y], Params(kappa=1.0, dt=1e-3, corr_tol=1.0))
    E = [bending_energy(s.xs[0], s.ys[0], 1.0)]
    for _ in range(20):
        s.step()
        E.append(bending_energy(s.xs[0], s.ys[0], 1.0))
    assert np.all(np.diff(E) < 0)


def test_area_length_drift_first_order():
    x, y = _ves(32, 1)
    drift = []
    for dt in (2e-3, 1e-3):
        s = Suspension([x], [y], Params(kappa=1.0, dt=dt, flow_kind=1, flow_p=(1.0, 0, 0, 0), corr_tol=1.0))
        for _ in range(int(round(0.02 / dt))):
            s.step()
        A, L = area_length(s.xs[0], s.ys[0])
        drift.append(abs(L / s.L0[0] - 1))
    assert drift[1] < 0.7 * drift[0]
    assert drift[0] < 1e-3


def test_translation_rotation_equivariance():
    xa, ya = _ves(32, 2, -1.4, 0.1)
    xb, yb = _ves(32, 3, 1.5, -0.2, theta=1.2)
    p = Params(kappa=1.0, dt=1e-3, corr_tol=1.0)
    s1 = Suspension([xa, xb], [ya, yb], p)
    th = 0.7
    c, sn = np.cos(th), np.sin(th)
    rot = lambda x, y: (c * x - sn * y + 3.0, sn * x + c * y - 1.0)
    ra, rb = rot(xa, ya), rot(xb, yb)
    s2 = Suspension([ra[0], rb[0]], [ra[1], rb[1]], p)
    for _ in range(3):
        s1.step()
        s2.step()
    for v in range(2):
        ex, ey = rot(s1.xs[v], s1.ys[v])
        assert np.max(np.abs(ex - s2.xs[v])) + np.max(np.abs(ey - s2.ys[v])) < 1e-11
        assert np.max(np.abs(s1.sig[v] - s2.sig[v])) < 1e-9 * np.max(np.abs(s1.sig[v]))


def test_first_order_in_time():
    x, y = _ves(32, 4)
    T = 0.016
    finals = []
    for dt in (4e-3, 2e-3, 1e-3, 2.5e-4):
        s = Suspension([x], [y], Params(kappa=1.0, dt=dt, flow_kind=1, flow_p=(1.0, 0, 0, 0), corr_tol=1.0))
        for _ in range(int(round(T / dt))):
            s.step()
        finals.append(np.concatenate([s.xs[0], s.ys[0]]))
    ref = finals[-1]
    e = [np.linalg.norm(f - ref) for f in finals[:-1]]
    r1, r2 = e[0] / e[1], e[1] / e[2]
    assert 1.5 < r1 < 3.0 and 1.5 < r2 < 3.5


def test_advection_moves_with_uniform_background():
    # a uniform background velocity is inextensible: the vesicle translates rigidly by dt*U
    x, y = _ves(32, 5)
    s = Suspension([x], [y], Params(kappa=1.0, dt=1e-3, flow_kind=3, flow_p=(2.0, 1e9, 0, 0), corr_tol=1.0))
    s0 = Suspension([x], [y], Params(kappa=1.0, dt=1e-3, corr_tol=1.0))
    s.step()
    s0.step()
    assert np.max(np.abs(s.xs[0] - s0.xs[0] - 2e-3)) < 1e-10
    assert np.max(np.abs(s.ys[0] - s0.ys[0])) < 1e-10


def test_close_vesicles_against_circles_at_known_gaps():
    # two unit circles whose nearest points (angles 0 and pi, both sampled) are `gap` apart; h = 2 pi / N
    from oracle.step import close_vesicles
    N = 32
    t = 2 * np.pi * np.arange(N) / N
    h = 2 * np.pi / N
    far = (np.cos(t) + 40.0, np.sin(t))
    for gap, expect in ((2.9 * h, {0, 1}), (3.1 * h, set())):
        xs = [np.cos(t), np.cos(t) + 2.0 + gap, far[0]]
        ys = [np.sin(t), np.sin(t), far[1]]
        assert close_vesicles(xs, ys, 3.0) == expect


def _inextensibility_residual(x, y, sig, ux, uy, kappa, mu):
    """Surface divergence X_s . d/ds of the total membrane velocity u + S[f(sigma)], relative to the
    divergence of the velocity without tension. f is built by spectral.force (the force's definition,
    Eq. elastic_force), S by the self-quadrature: neither goes through the Operators matrices that the
    tension update solves with."""
    from oracle.spectral import Geometry, d_s, force
    from oracle.stokes import self_single_layer_matrix
    g = Geometry(x, y)
    N = len(x)
    S = self_single_layer_matrix(x, y, mu)

    def div(sigma):
        fx, fy = force(x, y, sigma, kappa)
        w = S @ np.concatenate([fx, fy]) + np.concatenate([ux, uy])
        return g.tx * d_s(w[:N], g.sa) + g.ty * d_s(w[N:], g.sa)

    return np.max(np.abs(div(sig))) / np.max(np.abs(div(np.zeros(N))))


@pytest.mark.parametrize("flow", [(1, (1.0, 0.0, 0.0, 0.0)), (2, (1.0, 1.7, 0.0, 0.0))])
def test_tension_makes_the_total_velocity_inextensible(flow):
    # Eq. tension_disc: sigma is the Lagrange multiplier of inextensibility, so the velocity of the
    # membrane under bending, the tension's own force and the background flow has zero surface
    # divergence (Eq. inextensib). A sign error or a dropped background term in the update fails it.
    from oracle.flows import background
    from oracle.operators import Operators
    from oracle.step import _tension
    for N, seed in ((32, 6), (64, 7)):
        x, y = _ves(N, seed, 0.3, -0.2, R=0.8)
        ub = background(flow[0], flow[1], x, y)
        sig = _tension(Operators(x, y, 1.3, 0.9), x, y, ub[0], ub[1], 1.3)
        assert _inextensibility_residual(x, y, sig, ub[0], ub[1], 1.3, 0.9) < 1e-10


@pytest.mark.parametrize("flow", [(1, (1.0, 0.0, 0.0, 0.0)), (2, (1.0, 1.7, 0.0, 0.0))])
def test_initial_and_stepped_tension_keep_the_membrane_inextensible(flow):
    # The suspension's sigma^0 (background velocity at X^0) and, for a single vesicle in a quiescent
    # fluid, sigma^1 (velocity u^0 = 0) each make the total velocity inextensible at their own points.
    from oracle.flows import background
    x, y = _ves(32, 8)
    s = Suspension([x], [y], Params(kappa=1.0, mu=1.0, dt=1e-3, flow_kind=flow[0], flow_p=flow[1],
                                    corr_tol=1.0))
    ub = background(flow[0], flow[1], s.xs[0], s.ys[0])
    assert _inextensibility_residual(s.xs[0], s.ys[0], s.sig[0], ub[0], ub[1], 1.0, 1.0) < 1e-10
    q = Suspension([x], [y], Params(kappa=1.0, mu=1.0, dt=1e-3, corr_tol=1.0))
    q.step()
    z = np.zeros(32)
    assert _inextensibility_residual(q.xs[0], q.ys[0], q.sig[0], z, z, 1.0, 1.0) < 1e-10
