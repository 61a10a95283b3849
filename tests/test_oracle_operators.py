"""Pins for oracle.operators (Eqs. bending_op, tension_op, PTop, inextensib, Sec. 3.1)."""
import numpy as np

from oracle.operators import Operators
from oracle.spectral import Geometry


def _shape(N, seed=0):
    t = 2 * np.pi * np.arange(N) / N
    rng = np.random.default_rng(seed)
    x = 1.3 * np.cos(t) + 0.06 * np.cos(3 * t + rng.uniform()) + 0.5
    y = 0.6 * np.sin(t) + 0.05 * np.sin(2 * t + rng.uniform()) - 0.2
    return x, y


def test_projector_identities():
    N = 32
    x, y = _shape(N)
    ops = Operators(x, y, 1.0, 1.0)
    M = ops.M()
    I = np.eye(2 * N)
    assert np.max(np.abs(ops.P @ (I - M))) < 1e-8 * np.max(np.abs(ops.P))
    Q = I - M
    assert np.max(np.abs(Q @ Q - Q)) < 1e-8 * np.max(np.abs(Q))


def test_projected_velocity_is_inextensible():
    N = 64
    x, y = _shape(N, 1)
    ops = Operators(x, y, 1.0, 1.0)
    rng = np.random.default_rng(3)
    u = rng.standard_normal(2 * N)
    w = ops.project(u)
    g = Geometry(x, y)
    # surface divergence X_s . u_s computed independently from the geometry
    from oracle.spectral import d_s
    div = g.tx * d_s(w[:N], g.sa) + g.ty * d_s(w[N:], g.sa)
    assert np.max(np.abs(div)) < 1e-8 * np.max(np.abs(d_s(u[:N], g.sa)))


def test_bending_velocity_vanishes_on_circle():
    # X_ssss = n/R^3 on a circle and S[n] = 0, so B X = 0
    N = 32
    t = 2 * np.pi * np.arange(N) / N
    R = 0.5
    x, y = R * np.cos(t), R * np.sin(t)
    ops = Operators(x, y, 1.0, 1.0)
    assert np.max(np.abs(ops.B @ np.concatenate([x, y]))) < 1e-9 / R ** 3


def test_tension_operator_matches_force_definition():
    # T sigma must equal S applied to (sigma X_s)_s built from the geometry
    N = 32
    x, y = _shape(N, 2)
    ops = Operators(x, y, 2.0, 1.5)
    g = Geometry(x, y)
    from oracle.spectral import d_s
    sig = np.cos(2 * np.pi * np.arange(N) / N) + 0.3
    f = np.concatenate([d_s(sig * g.tx, g.sa), d_s(sig * g.ty, g.sa)])
    assert np.max(np.abs(ops.T @ sig - ops.S @ f)) < 1e-12 * np.max(np.abs(ops.S @ f))
