"""Pins for oracle.farfield (Sec. 2.2.2, Sec. 4.1)."""
import numpy as np

from oracle.farfield import far_field
from oracle.spectral import Geometry


def _circle(N, R, cx, cy):
    t = 2 * np.pi * np.arange(N) / N
    return R * np.cos(t) + cx, R * np.sin(t) + cy


def test_exterior_closed_form_through_far_field():
    N = 64
    R = 0.5
    xs0, ys0 = _circle(N, R, 0.0, 0.0)
    xs1, ys1 = _circle(8, 0.05, 1.7, 0.4)
    F = 0.8 + 0.25j
    ux, uy, near = far_field([xs0, xs1], [ys0, ys1], [np.full(N, F.real), np.zeros(8)],
                             [np.full(N, F.imag), np.zeros(8)], 1.0)
    assert near == []
    rho = np.hypot(xs1, ys1)
    psi = np.arctan2(ys1, xs1)
    ex = (-2 * np.pi * R * np.log(rho) * F + np.pi * R * F
          + np.pi * R * (1 - R ** 2 / rho ** 2) * np.exp(2j * psi) * np.conj(F)) / (4 * np.pi)
    got = ux[N:] + 1j * uy[N:]
    assert np.max(np.abs(got - ex)) < 1e-12


def test_brute_force_tiny():
    rng = np.random.default_rng(7)
    M, N = 3, 8
    xs, ys, fxs, fys = [], [], [], []
    for v in range(M):
        x, y = _circle(N, 0.3 + 0.1 * v, 2.0 * v, 0.5 * v)
        xs.append(x + 0.01 * rng.standard_normal(N))
        ys.append(y + 0.01 * rng.standard_normal(N))
        fxs.append(rng.standard_normal(N))
        fys.append(rng.standard_normal(N))
    ux, uy, near = far_field(xs, ys, fxs, fys, 0.9)
    assert near == []
    k = 0
    for i in range(M):
        for a in range(N):
            sx = sy = 0.0
            for v in range(M):
                if v == i:
                    continue
                g = Geometry(xs[v], ys[v])
                for b in range(N):
                    rx = xs[i][a] - xs[v][b]
                    ry = ys[i][a] - ys[v][b]
                    r = (rx * rx + ry * ry) ** 0.5
                    w = g.sa[b] * 2 * np.pi / N
                    fr = rx * fxs[v][b] + ry * fys[v][b]
                    sx += (-np.log(r) * fxs[v][b] + fr * rx / r ** 2) * w
                    sy += (-np.log(r) * fys[v][b] + fr * ry / r ** 2) * w
            assert abs(ux[k] - sx / (4 * np.pi * 0.9)) < 1e-12 * (1 + abs(sx))
            assert abs(uy[k] - sy / (4 * np.pi * 0.9)) < 1e-12 * (1 + abs(sy))
            k += 1


def test_near_mask_semantics():
    N = 32
    x0, y0 = _circle(N, 1.0, 0.0, 0.0)
    g0 = Geometry(x0, y0)
    # second vesicle whose leftmost point sits 0.5 h from the first vesicle's rightmost point
    x1, y1 = _circle(N, 0.5, 1.0 + 0.5 * g0.h + 0.5, 0.0)
    rng = np.random.default_rng(0)
    f = [rng.standard_normal(N) for _ in range(4)]
    ux, uy, near = far_field([x0, x1], [y0, y1], [f[0], f[1]], [f[2], f[3]], 1.0)
    uxa, uya, _ = far_field([x0, x1], [y0, y1], [f[0], f[1]], [f[2], f[3]], 1.0, near_mask=False)
    g1 = Geometry(x1, y1)
    expect = []
    for i in range(N):
        if np.min(np.hypot(x1 - x0[i], y1 - y0[i])) <= g1.h:
            expect.append((i, 1))
    for i in range(N):
        if np.min(np.hypot(x0 - x1[i], y0 - y1[i])) <= g0.h:
            expect.append((N + i, 0))
    assert near == sorted(expect) and len(near) > 0
    masked = {t for t, _ in near}
    for t in range(2 * N):
        if t in masked:
            assert ux[t] == 0.0 and uy[t] == 0.0
        else:
            assert ux[t] == uxa[t] and uy[t] == uya[t]
