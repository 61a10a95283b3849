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


# ---- learned near field (Sec. 3.3, Eq. NearFieldMap)

def _layers_no_nyquist(UX, UY, N):
    return (np.concatenate([_no_nyquist(UX[d * N:(d + 1) * N]) for d in range(5)]),
            np.concatenate([_no_nyquist(UY[d * N:(d + 1) * N]) for d in range(5)]))


@pytest.mark.parametrize("N,L_scale,mu", [(32, 1.0, 1.0), (32, 2.7, 0.6), (48, 0.35, 1.9)])
def test_near_columns_reproduce_the_layer_velocities(N, L_scale, mu):
    # all modes but the Nyquist one (K_f = K_out = N/2 - 1): the learned layers equal the exact ones for any
    # position, orientation, size and viscosity, including the density's net force (its log L term)
    from oracle.learned import near_columns, near_layers_learned
    from oracle.nearfield import layer_velocities
    x, y = _vesicle(N, 11)
    x, y = L_scale * x + 0.4, L_scale * y - 0.9
    K = N // 2 - 1
    fx, fy = _band_limited(N, K, 12)
    fx = fx + 0.7  # a net force: the integral of f over the curve is not zero
    rows = near_columns(x, y, K, K)
    UX, UY = near_layers_learned(x, y, fx, fy, rows, K, K, mu)
    RX, RY = _layers_no_nyquist(*layer_velocities(x, y, fx, fy, mu), N)
    scale = max(np.max(np.abs(RX)), np.max(np.abs(RY)))
    assert np.max(np.abs(UX - RX)) <= 1e-11 * scale, np.max(np.abs(UX - RX)) / scale
    assert np.max(np.abs(UY - RY)) <= 1e-11 * scale, np.max(np.abs(UY - RY)) / scale


def test_near_columns_do_not_depend_on_position_orientation_size_or_labels():
    from oracle.learned import near_columns
    x, y = _vesicle(32, 13)
    a = near_columns(x, y, 4, 8)
    th = 0.2  # small enough to keep the principal axis's sign (the standard frame's choice)
    xr = 2.2 * (np.cos(th) * x - np.sin(th) * y) + 5.0
    yr = 2.2 * (np.sin(th) * x + np.cos(th) * y) - 3.0
    b = near_columns(np.roll(xr, 7), np.roll(yr, 7), 4, 8)
    for ra, rb in zip(a, b):
        assert np.max(np.abs(ra - rb)) <= 1e-11 * np.max(np.abs(ra))


def test_near_correction_with_near_columns_follows_the_exact_one():
    # through the RBF: a band-limited density (modes <= K_f) gives the exact correction up to the layers'
    # Nyquist mode, which the columns cannot carry
    from oracle.farfield import far_field
    from oracle.learned import near_columns, near_layers_learned
    from oracle.nearfield import near_correction
    N, K = 32, 15
    rng = np.random.default_rng(14)
    xa, ya = vesicle_outline(N, 0.7, 0.5, 2e-2, rng, 1.5)
    xb, yb = vesicle_outline(N, 0.7, 0.5, 2e-2, rng, 1.5)
    xs, ys = [xa - 0.33, xb + 0.33], [ya, yb + 0.05]
    fs = [_band_limited(N, K, 15 + v) for v in range(2)]
    fxs, fys = [f[0] for f in fs], [f[1] for f in fs]
    _, _, near = far_field(xs, ys, fxs, fys, 1.0, near_mask=True)
    assert near
    from oracle.nearfield import layer_velocities
    rows = {v: near_columns(xs[v], ys[v], K, K) for v in range(2)}
    learned = lambda v: near_layers_learned(xs[v], ys[v], fxs[v], fys[v], rows[v], K, K, 1.0)
    filtered = lambda v: _layers_no_nyquist(*layer_velocities(xs[v], ys[v], fxs[v], fys[v], 1.0), N)
    cx, cy = near_correction(xs, ys, fxs, fys, 1.0, near, layers=learned)
    fx_, fy_ = near_correction(xs, ys, fxs, fys, 1.0, near, layers=filtered)
    ex, ey = near_correction(xs, ys, fxs, fys, 1.0, near)
    scale = np.sqrt(np.sum(ex ** 2 + ey ** 2))
    same = np.sqrt(np.sum((cx - fx_) ** 2 + (cy - fy_) ** 2)) / scale
    nyq = np.sqrt(np.sum((cx - ex) ** 2 + (cy - ey) ** 2)) / scale
    print("near correction, learned layers with exact columns: %.2e from the Nyquist-filtered exact layers, "
          "%.2e from the exact ones" % (same, nyq))
    assert same <= 1e-10
    assert nyq <= 2e-2


def test_step_velocity_with_exact_near_columns_uses_the_learned_layers():
    # the hybrid step's interaction velocity with the near-field networks replaced by the exact columns:
    # the near correction is that of the exact layers with their Nyquist mode removed, for every source
    from oracle.farfield import far_field
    from oracle.learned import near_columns
    from oracle.nearfield import layer_velocities, near_correction
    from oracle.spectral import force
    from oracle.step import Params, Suspension
    N, K = 32, 15
    rng = np.random.default_rng(16)
    xa, ya = vesicle_outline(N, 0.7, 0.5, 2e-2, rng, 1.5)
    xb, yb = vesicle_outline(N, 0.7, 0.5, 2e-2, rng, 1.5)
    xc, yc = vesicle_outline(N, 0.7, 0.5, 2e-2, rng, 0.2)
    xs, ys = [xa - 0.33, xb + 0.33, xc], [ya, yb + 0.05, yc + 1.4]
    nets = [(lambda d: (lambda x, y: near_columns(x, y, K, K)[d]))(d) for d in range(5)]
    relax = (None, None, 1.0, 12)  # only its filter kmax is read by the interaction velocity
    kw = dict(kappa=1.0, mu=0.8, dt=1e-3, flow_kind=1, flow_p=(1.0, 0, 0, 0), near_field=True)
    s = Suspension(xs, ys, Params(relax_net=relax, near_net=(nets, K, K), **kw))
    u = s.interaction_velocity()
    assert s.near_pairs
    fx, fy = zip(*[force(x, y, sg, 1.0) for x, y, sg in zip(s.xs, s.ys, s.sig)])
    ux, uy, near = far_field(s.xs, s.ys, fx, fy, 0.8, near_mask=True)
    # the learned layers see the density's modes below the Nyquist one and give layers without it
    filt = lambda v: _layers_no_nyquist(*layer_velocities(s.xs[v], s.ys[v], _no_nyquist(fx[v]), _no_nyquist(fy[v]),
                                                          0.8), N)
    cx, cy = near_correction(s.xs, s.ys, fx, fy, 0.8, near, layers=filt)
    o = 0
    for v in range(3):
        bx = ux[o:o + N] + cx[o:o + N] + s.xs[v] * 0.0 + 1.0 * s.ys[v]  # shear (y, 0)
        by = uy[o:o + N] + cy[o:o + N]
        assert np.max(np.abs(u[v][0] - bx)) + np.max(np.abs(u[v][1] - by)) <= 1e-10 * np.max(np.abs(bx))
        o += N
