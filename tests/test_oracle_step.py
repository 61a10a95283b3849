"""Pins for oracle.step (Algorithm 1, Eqs. advection_disc, relaxation_disc, tension_disc)."""
import numpy as np

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
