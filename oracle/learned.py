"""Learned advection and tension maps of the hybrid step (Sec. 3.2: Eqs. advectionMap, advTenMap and the
self-tension map S_sigma; Table tab:networks). Test infrastructure only.

The paper removes the dependence on the interaction velocity u = U_near + U_far + u_inf by expanding u in
Fourier modes along the vesicle and learning, per mode, the action of the linear operators on it:
    X_u^k : X -> (I - M) e^{ik alpha}            (advection, Eq. advection_disc)
    S_u^k : X -> L^{-1} P e^{ik alpha}            (velocity part of the tension, Eq. tension_disc)
    S_sigma: X -> L^{-1} P B X                    (self part of the tension)
All of them act in the standard frame of the vesicle (oracle.standardize: centred, principal axis along y,
unit length, first point on the positive x axis). (I - M) and L^{-1} P do not change when the vesicle is
scaled (a velocity keeps its size), and S_sigma of a vesicle of length L is S_sigma of its unit-length
copy divided by L^2 (B carries four arclength derivatives and S one length, P and L^{-1} cancel).

Readings (the paper gives neither the basis nor the output representation):
* the velocity basis is the real form of the modes k = 0..K_f of each component: with
  f = fourier_features(u_x, u_y, K_f) (oracle.standardize), a velocity whose modes are all <= K_f equals
  sum_i f_i psi_i, psi_i the field of component c equal to 1 (a_0), 2 cos(k alpha) (a_k) or
  -2 sin(k alpha) (b_k) at the points alpha_j = 2 pi j / N; modes above K_f of u are dropped;
* each learned column (a velocity field for X_u, a scalar field for S_u and S_sigma) is represented by its
  Fourier features up to K_out: fourier_features for a velocity field, the first 2 K_out + 1 of them for
  a scalar field (scalar_features);
* network outputs (one network per family): X_u row = the nb = 4 K_f + 2 columns' velocity features,
  2 (2 K_out + 1) each, in basis order; S row = S_sigma's scalar features, then the nb columns' scalar
  features, 2 K_out + 1 each.
Learned advection: X* = X^n + dt R^T roll((sum_i f_i Q_i)(alpha), j0), f the features of roll(R u, -j0);
learned tension: sigma = -roll(S_sigma(alpha), j0) / L^2 - roll((sum_i f_i S_i)(alpha), j0).

exact_columns() computes the same outputs with the exact operators (oracle.operators) at the standardised
shape: the targets the networks are trained to, and with them the learned maps reproduce the exact ones
for velocities of modes <= K_f (pins in tests/test_oracle_learned.py).

Learned near field (Sec. 3.3, Eq. NearFieldMap): N_X^k maps a shape to the single layer of the density
e^{ik alpha} at the five layer points (oracle.nearfield), so that S[X, f] there is the sum over the density's
Fourier modes. Readings: the same real basis psi_i (modes 0..K_f of each component) for the density; the
layer velocities of each psi_i at the layers of the unit-length standardised shape, with mu = 1, as
velocity features up to K_out per layer; one network per layer (row d = the nb columns of layer d,
2 (2 K_out + 1) each). For a vesicle X = c + L R^T X^o the single layer transforms as
    S[X, f](x) = L R^T S[X^o, R f](x^o) / mu - (L log L / (4 pi mu)) (integral of f over the unit curve),
(the Stokeslet's -log|r| gains -log L under the scaling; the layer spacing h = L/N scales with the shape),
so the learned layers are L R^T roll(sum_i c_i Q_d,i, j0) / mu plus that constant, c the features of
roll(R f, -j0). The learned layers are those of the density's modes 0..K_f (f_K, the basis's span): the
integral is that of f_K, by the quadrature each layer takes (the trapezoid rule on the N points for the
layer on the curve, the smooth part of the self rule; on the upsampled curve for the others).
"""
import numpy as np

from .operators import Operators
from .spectral import Geometry, upsample
from .standardize import features_to_samples, fourier_features, fourier_filter, standardize


def basis_count(Kf):
    return 4 * Kf + 2


def basis_field(i, Kf, N):
    """psi_i at the N points (x then y)."""
    per = 2 * Kf + 1
    c, r = divmod(i, per)
    j = np.arange(N)
    if r == 0:
        v = np.ones(N)
    elif r <= Kf:
        v = 2.0 * np.cos(2.0 * np.pi * r * j / N)
    else:
        v = -2.0 * np.sin(2.0 * np.pi * (r - Kf) * j / N)
    z = np.zeros(N)
    return np.concatenate([v, z]) if c == 0 else np.concatenate([z, v])


def scalar_features(v, K):
    """[a_0..a_K, b_1..b_K] of a scalar field v (the x half of fourier_features)."""
    return fourier_features(v, np.zeros_like(v), K)[:2 * K + 1]


def scalar_samples(g, K, N):
    """The scalar field with features g (inverse of scalar_features for modes <= K)."""
    f = np.concatenate([g, np.zeros(2 * K + 1)])
    return features_to_samples(f, K, N)[0]


def velocity_to_frame(ux, uy, fr):
    """A velocity field expressed in the standard frame: rotated and re-indexed, not scaled."""
    rx, ry = fr.cos_t * ux - fr.sin_t * uy, fr.sin_t * ux + fr.cos_t * uy
    return np.roll(rx, -fr.j0), np.roll(ry, -fr.j0)


def velocity_from_frame(vx, vy, fr):
    vx, vy = np.roll(vx, fr.j0), np.roll(vy, fr.j0)
    return fr.cos_t * vx + fr.sin_t * vy, -fr.sin_t * vx + fr.cos_t * vy


def exact_columns(x, y, Kf, Kout, kappa=1.0, mu=1.0):
    """(X_u row, S row) of the vesicle (x, y) from the exact operators at its standardised shape."""
    xo, yo, _ = standardize(x, y)
    N = len(x)
    ops = Operators(xo, yo, kappa, mu)
    Q = np.eye(2 * N) - ops.M()
    LP = np.linalg.solve(ops.L, ops.P)
    ss = np.linalg.solve(ops.L, ops.P @ (ops.B @ np.concatenate([xo, yo])))
    adv, ten = [], [scalar_features(ss, Kout)]
    for i in range(basis_count(Kf)):
        psi = basis_field(i, Kf, N)
        q = Q @ psi
        adv.append(fourier_features(q[:N], q[N:], Kout))
        ten.append(scalar_features(LP @ psi, Kout))
    return np.concatenate(adv), np.concatenate(ten)


def advect_learned(x, y, ux, uy, dt, adv_row, Kf, Kout):
    """X* = X^n + dt (I - M) u with the learned X_u row (module header)."""
    N = len(x)
    _, _, fr = standardize(x, y)
    vx, vy = velocity_to_frame(ux, uy, fr)
    f = fourier_features(vx, vy, Kf)
    cw = 2 * (2 * Kout + 1)
    g = np.zeros(cw)
    for i in range(basis_count(Kf)):
        g = g + f[i] * adv_row[i * cw:(i + 1) * cw]
    qx, qy = features_to_samples(g, Kout, N)
    px, py = velocity_from_frame(qx, qy, fr)
    return x + dt * px, y + dt * py


def tension_learned(x, y, ux, uy, ten_row, Kf, Kout):
    """sigma = -L^{-1} P (B X + u) with the learned S row (module header)."""
    N = len(x)
    _, _, fr = standardize(x, y)
    vx, vy = velocity_to_frame(ux, uy, fr)
    f = fourier_features(vx, vy, Kf)
    sw = 2 * Kout + 1
    g = -ten_row[:sw] / Geometry(x, y).length ** 2
    for i in range(basis_count(Kf)):
        g = g - f[i] * ten_row[(i + 1) * sw:(i + 2) * sw]
    return np.roll(scalar_samples(g, Kout, N), fr.j0)


def near_columns(x, y, Kf, Kout):
    """The N_X rows (one per layer) of the vesicle (x, y): exact layer velocities (oracle.nearfield, mu = 1)
    of every basis density psi_i at the layers of its standardised shape, as velocity features up to Kout."""
    from .nearfield import LAYERS, layer_velocities
    xo, yo, _ = standardize(x, y)
    N = len(x)
    rows = [[] for _ in LAYERS]
    for i in range(basis_count(Kf)):
        psi = basis_field(i, Kf, N)
        UX, UY = layer_velocities(xo, yo, psi[:N], psi[N:], 1.0)
        for d in range(len(LAYERS)):
            rows[d].append(fourier_features(UX[d * N:(d + 1) * N], UY[d * N:(d + 1) * N], Kout))
    return [np.concatenate(r) for r in rows]


def near_layers_learned(x, y, fx, fy, rows, Kf, Kout, mu):
    """S[X, f] at the 5N layer points of (x, y) (layer-major, as oracle.nearfield.layer_velocities) from the
    N_X rows (module header)."""
    N = len(x)
    _, _, fr = standardize(x, y)
    g = Geometry(x, y)
    L = g.length
    vx, vy = velocity_to_frame(fx, fy, fr)
    c = fourier_features(vx, vy, Kf)
    cw = 2 * (2 * Kout + 1)
    # integral of f over the unit-length curve, (1/L) times the quadrature of f ds: on the N points for the
    # layer on the curve, on the curve upsampled as in oracle.nearfield for the others
    from .nearfield import LAYERS, upsample_factor
    rho = upsample_factor(N)
    gu = Geometry(upsample(x, rho), upsample(y, rho))
    fxk, fyk = fourier_filter(fx, Kf), fourier_filter(fy, Kf)
    fxu, fyu = upsample(fxk, rho), upsample(fyk, rho)
    tot = {True: (np.sum(fxk * g.sa) * 2.0 * np.pi / N / L, np.sum(fyk * g.sa) * 2.0 * np.pi / N / L),
           False: (np.sum(fxu * gu.sa) * 2.0 * np.pi / (rho * N) / L, np.sum(fyu * gu.sa) * 2.0 * np.pi / (rho * N) / L)}
    k0 = -L * np.log(L) / (4.0 * np.pi * mu)
    UX, UY = [], []
    for d, row in zip(LAYERS, rows):
        tot_x, tot_y = tot[d == 0.0]
        acc = np.zeros(cw)
        for i in range(basis_count(Kf)):
            acc = acc + c[i] * row[i * cw:(i + 1) * cw]
        qx, qy = features_to_samples(acc, Kout, N)
        px, py = velocity_from_frame(qx, qy, fr)
        UX.append(L * px / mu + k0 * tot_x)
        UY.append(L * py / mu + k0 * tot_y)
    return np.concatenate(UX), np.concatenate(UY)
