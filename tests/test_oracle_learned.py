"""Pins for oracle.learned (Sec. 3.2: Eqs. advectionMap, advTenMap and S_sigma): with the exact columns the
learned advection and tension reproduce the exact operators for velocities of modes <= K_f, the basis
reproduces band-limited velocities, the columns do not depend on the vesicle's position, orientation,
size or point labelling, and every advection column is inextensible."""
import numpy as np
import pytest

from oracle.learned import (advect_learned, basis_count, basis_field, exact_columns, tension_learned,
                            velocity_from_frame, velocity_to_frame)
from oracle.operators import Operators
from oracle.spectral import Geometry, d_s
from oracle.standardize import features_to_samples, fourier_features, standardize
from oracle.step import _tension
from paper_2606_25569_b300.workloads import vesicle_outline


def _vesicle(N, seed):
    rng = np.random.default_rng(seed)
    x, y = vesicle_outline(N, 0.7, 0.8, 2e-2, rng, rng.uniform(0, 2 * np.pi))
    return x + 0.3, y - 1.1


def _band_limited(N, K, seed):
    rng = np.random.default_rng(seed)
    al = 2 * np.pi * np.arange(N) / N
    return [sum(rng.standard_normal() * np.cos(k * al) + rng.standard_normal() * np.sin(k * al)
                for k in range(K + 1)) for _ in range(2)]


def _no_nyquist(v):
    c = np.fft.fft(v)
    c[len(v) // 2] = 0.0
    return np.fft.ifft(c).real


def test_basis_reproduces_band_limited_velocities():
    N, Kf = 32, 6
    ux, uy = _band_limited(N, Kf, 1)
    f = fourier_features(ux, uy, Kf)
    u = sum(f[i] * basis_field(i, Kf, N) for i in range(basis_count(Kf)))
    assert np.max(np.abs(u - np.concatenate([ux, uy]))) < 1e-13 * np.max(np.abs(u))


def test_frame_round_trip_of_velocities():
    x, y = _vesicle(48, 2)
    _, _, fr = standardize(x, y)
    ux, uy = _band_limited(48, 20, 3)
    bx, by = velocity_from_frame(*velocity_to_frame(ux, uy, fr), fr)
    assert np.max(np.abs(bx - ux)) + np.max(np.abs(by - uy)) < 1e-13


@pytest.mark.parametrize("N", [32, 64])
def test_exact_columns_reproduce_the_advection(N):
    # Eq. advection_disc: X* = X + dt (I - M) u; columns kept to mode N/2 - 1 (the Nyquist mode is the only
    # one they cannot carry)
    x, y = _vesicle(N, 4)
    Kf, Kout = 8, N // 2 - 1
    adv, _ = exact_columns(x, y, Kf, Kout)
    ux, uy = _band_limited(N, Kf, 5)
    dt = 1e-3
    q = Operators(x, y, 1.0, 1.0).project(np.concatenate([ux, uy]))
    lx, ly = advect_learned(x, y, ux, uy, dt, adv, Kf, Kout)
    for got, ref in ((lx, x + dt * q[:N]), (ly, y + dt * q[N:])):
        assert np.max(np.abs(_no_nyquist(got - ref))) < 1e-10 * dt * np.max(np.abs(q))


@pytest.mark.parametrize("N", [32, 64])
def test_exact_columns_reproduce_the_tension(N):
    # Eq. tension_disc: sigma = -L^{-1} P (B X + u), both parts through the learned form
    x, y = _vesicle(N, 6)
    Kf, Kout = 8, N // 2 - 1
    _, ten = exact_columns(x, y, Kf, Kout, kappa=1.0, mu=1.0)
    ux, uy = _band_limited(N, Kf, 7)
    ref = _tension(Operators(x, y, 1.0, 1.0), x, y, ux, uy, 1.0)
    got = tension_learned(x, y, ux, uy, ten, Kf, Kout)
    assert np.max(np.abs(_no_nyquist(got - ref))) < 1e-10 * np.max(np.abs(ref))


def test_columns_do_not_depend_on_position_orientation_size_or_labels():
    N = 32
    x, y = _vesicle(N, 8)
    a0, t0 = exact_columns(x, y, 4, 10)
    # a rotation small enough to keep the sign choice of the principal axis (oracle.standardize)
    c, s, lam = np.cos(0.2), np.sin(0.2), 0.37
    x1, y1 = lam * (c * x - s * y) + 5.0, lam * (s * x + c * y) - 2.0
    a1, t1 = exact_columns(np.roll(x1, 5), np.roll(y1, 5), 4, 10)
    assert np.max(np.abs(a1 - a0)) < 1e-10 * np.max(np.abs(a0))
    assert np.max(np.abs(t1 - t0)) < 1e-10 * np.max(np.abs(t0))


def test_advection_columns_are_inextensible():
    # (I - M) maps any velocity to an inextensible one (Eq. inextensib): zero surface divergence at the
    # standardised shape, for every column
    N = 64
    x, y = _vesicle(N, 9)
    Kf, Kout = 6, N // 2 - 1
    adv, _ = exact_columns(x, y, Kf, Kout)
    xo, yo, _ = standardize(x, y)
    g = Geometry(xo, yo)
    cw = 2 * (2 * Kout + 1)
    for i in range(basis_count(Kf)):
        vx, vy = features_to_samples(adv[i * cw:(i + 1) * cw], Kout, N)
        div = g.tx * d_s(vx, g.sa) + g.ty * d_s(vy, g.sa)
        psi = basis_field(i, Kf, N)
        scale = np.max(np.abs(g.tx * d_s(psi[:N], g.sa) + g.ty * d_s(psi[N:], g.sa))) + 1.0
        assert np.max(np.abs(div)) < 1e-6 * scale, i


def test_step_with_exact_columns_equals_the_plain_step():
    # oracle.step with the flow "networks" replaced by the exact columns (Kf = Kout = N/2 - 1): the learned
    # advection and tension are then the exact ones except for the Nyquist mode, which the Fourier-feature
    # representation does not carry; with the exact relaxation on every step (exact_every = 1) the hybrid
    # step follows the plain step. sigma is compared without its Nyquist mode (L^{-1} leaves it weakly
    # determined: 0.2% of sigma on this shape).
    from oracle.step import Params, Suspension
    N = 64
    rng = np.random.default_rng(10)
    x, y = vesicle_outline(N, 0.7, 0.8, 1e-3, rng, 0.7)
    K = N // 2 - 1
    adv = lambda a, b: exact_columns(a, b, K, K)[0]
    ten = lambda a, b: exact_columns(a, b, K, K, kappa=1.0, mu=1.0)[1]
    kw = dict(kappa=1.0, mu=1.0, dt=1e-3, flow_kind=1, flow_p=(1.0, 0, 0, 0), corr_tol=1.0)
    plain = Suspension([x], [y], Params(**kw))
    relax_net = ([16, 16], None, 1.0, 4)  # never evaluated: every step relaxes exactly
    hyb = Suspension([x], [y], Params(relax_net=relax_net, exact_every=1, flow_net=(adv, ten, K, K), **kw))
    for _ in range(3):
        plain.step()
        hyb.step()
    d = np.concatenate([hyb.xs[0] - plain.xs[0], hyb.ys[0] - plain.ys[0]])
    assert np.max(np.abs(d)) < 1e-7 * np.max(np.abs(plain.xs[0]))
    ds = _no_nyquist(hyb.sig[0] - plain.sig[0])
    assert np.max(np.abs(ds)) < 1e-5 * np.max(np.abs(plain.sig[0]))
