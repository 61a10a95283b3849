"""Pins for oracle.implicit (Sec. 2.2.3, Eq. time_step_sc1: the fully implicit step)."""
import numpy as np

from oracle.correct import area_length
from oracle.farfield import far_field
from oracle.flows import background
from oracle.implicit import ImplicitSuspension, force_matrix, implicit_solve
from oracle.operators import Operators
from oracle.spectral import bending_energy, force
from oracle.step import Params
from paper_2606_25569_b300.workloads import vesicle_outline

KAPPA, MU = 1.0, 1.0


def _ves(N, seed, cx=0.0, cy=0.0, R=1.0, nu=0.7, theta=0.3):
    rng = np.random.default_rng(seed)
    x, y = vesicle_outline(N, nu, R, 5e-2, rng, theta)
    return x + cx, y + cy


def test_force_matrix_is_the_membrane_force():
    # F [x; y; sigma] at the geometry of X itself: the spectral force -kappa X_ssss + (sigma X_s)_s (Eq. elastic_force)
    x, y = _ves(48, 0)
    sig = np.random.default_rng(1).standard_normal(48)
    F = force_matrix(Operators(x, y, KAPPA, MU), KAPPA)
    fx, fy = force(x, y, sig, KAPPA)
    got = F @ np.concatenate([x, y, sig])
    assert np.max(np.abs(got - np.concatenate([fx, fy]))) <= 1e-9 * np.max(np.abs(got))


def test_single_vesicle_equals_advection_then_relaxation_at_the_old_operators():
    # one vesicle: eliminating sigma from Eq. time_step_sc1 gives (I - dt (I - M) B) X^{n+1} = X^n + dt (I - M) u_inf
    # with every operator at X^n, and sigma^{n+1} = -L^{-1} P (B X^{n+1} + u_inf)
    for kind, fp in ((1, (1.5, 0, 0, 0)), (2, (1.0, 2.0, 0, 0))):
        x, y = _ves(32, 2, 0.3, -0.2)
        dt = 2e-3
        (x1, y1, s1), = implicit_solve([x], [y], KAPPA, MU, dt, kind, fp)
        ops = Operators(x, y, KAPPA, MU)
        ub = np.concatenate(background(kind, fp, x, y))
        IM = np.eye(64) - ops.M()
        z = np.linalg.solve(np.eye(64) - dt * IM @ ops.B, np.concatenate([x, y]) + dt * IM @ ub)
        sig = -np.linalg.solve(ops.L, ops.P @ (ops.B @ z + ub))
        assert np.max(np.abs(np.concatenate([x1, y1]) - z)) <= 1e-12 * np.max(np.abs(z))
        assert np.max(np.abs(s1 - sig)) <= 1e-9 * np.max(np.abs(sig))


def test_solution_satisfies_both_lines_with_the_far_field_sum():
    # the solved state, with densities from the operators at X^n, satisfies Eq. time_step_sc1 when the
    # interactions are evaluated by the far-field sum (Sec. 4.1) instead of the assembled blocks
    xs, ys = [], []
    for v, (cx, cy, N) in enumerate(((-1.3, 0.1, 32), (1.2, 0.4, 24), (0.0, -1.9, 32))):
        x, y = _ves(N, 10 + v, cx, cy, R=0.5)
        xs.append(x)
        ys.append(y)
    dt, kind, fp = 1e-3, 3, (1.0, 3.0, 0, 0)
    sol = implicit_solve(xs, ys, KAPPA, MU, dt, kind, fp)
    ops = [Operators(x, y, KAPPA, MU) for x, y in zip(xs, ys)]
    fx, fy = [], []
    for o, (x1, y1, s1) in zip(ops, sol):
        N = o.N
        D4 = o.Ds @ o.Ds @ o.Ds @ o.Ds
        ten = o.Ten @ s1
        fx.append(-KAPPA * D4 @ x1 + ten[:N])
        fy.append(-KAPPA * D4 @ y1 + ten[N:])
    ux, uy, _ = far_field(xs, ys, fx, fy, MU, near_mask=False)
    off = 0
    for v, (o, (x1, y1, s1)) in enumerate(zip(ops, sol)):
        N = o.N
        ub = np.concatenate(background(kind, fp, xs[v], ys[v]))
        U = o.S @ np.concatenate([fx[v], fy[v]]) + np.concatenate([ux[off:off + N], uy[off:off + N]]) + ub
        off += N
        r1 = np.concatenate([x1, y1]) - np.concatenate([xs[v], ys[v]]) - dt * U
        r2 = o.P @ U
        # rounding floor: the bending term's partial products (|S| |F| |z|) are 1e3..1e8 times the residual's terms
        z = np.concatenate([x1, y1, s1])
        mag = np.abs(o.S) @ (np.abs(force_matrix(o, KAPPA)) @ np.abs(z))
        assert np.max(np.abs(r1)) <= 1e-12 * dt * np.max(mag), np.max(np.abs(r1))
        assert np.max(np.abs(r2)) <= 1e-15 * np.max(np.abs(o.P) @ mag), np.max(np.abs(r2))


def test_mirror_symmetric_pair_stays_mirrored():
    # Poiseuille flow is even in y: a pair mirrored across y = 0 (orientation kept) stays mirrored
    x, y = _ves(32, 4, 0.2, 0.8, R=0.5)
    xm, ym = x[::-1].copy(), -y[::-1]
    sol = implicit_solve([x, xm], [y, ym], KAPPA, MU, 1e-3, 3, (1.0, 2.0, 0, 0))
    (xa, ya, sa), (xb, yb, sb) = sol
    # the stiff system amplifies rounding: a 1e-16 relative change of one input coordinate moves X^{n+1} by
    # 1.3e-10 and sigma by 5e-9 of its size, so the mirror images are held to 1e-8 and 1e-6
    s = np.max(np.abs(xa))
    assert np.max(np.abs(xb - xa[::-1])) <= 1e-8 * s
    assert np.max(np.abs(yb + ya[::-1])) <= 1e-8 * s
    assert np.max(np.abs(sb - sa[::-1])) <= 1e-6 * np.max(np.abs(sa))


def test_implicit_suspension_relaxes_and_keeps_area_and_length():
    # Sec. 5.2 in a quiescent fluid: the bending energy decays; the correction (Sec. 4.3) holds A and L
    xa, ya = _ves(32, 5, -0.9, 0.0, R=0.5)
    xb, yb = _ves(32, 6, 0.9, 0.1, R=0.5, theta=1.3)
    s = ImplicitSuspension([xa, xb], [ya, yb], Params(kappa=KAPPA, mu=MU, dt=1e-3, corr_tol=1e-3))
    E = [sum(bending_energy(x, y, KAPPA) for x, y in zip(s.xs, s.ys))]
    for _ in range(6):
        s.step()
        E.append(sum(bending_energy(x, y, KAPPA) for x, y in zip(s.xs, s.ys)))
    assert np.all(np.diff(E) < 0)
    for v in range(2):
        A, L = area_length(s.xs[v], s.ys[v])
        assert abs(A / s.A0[v] - 1) <= 1e-3 and abs(L / s.L0[v] - 1) <= 1e-3


def test_near_field_solution_satisfies_both_lines():
    # with the near field, the interactions are the masked far-field sum plus the near-field correction of the
    # same density (Sec. 3.3) at the targets the mask removed
    from oracle.nearfield import near_correction
    xs, ys = [], []
    for v, (cx, cy) in enumerate(((-0.36, 0.0), (0.36, 0.05), (0.0, 1.4))):
        x, y = _ves(32, 20 + v, cx, cy, R=0.5, theta=1.5 if v < 2 else 0.2)
        xs.append(x)
        ys.append(y)
    dt, kind, fp = 1e-3, 1, (1.0, 0, 0, 0)
    sol = implicit_solve(xs, ys, KAPPA, MU, dt, kind, fp, near_field=True)
    ops = [Operators(x, y, KAPPA, MU) for x, y in zip(xs, ys)]
    fx, fy = [], []
    for o, (x1, y1, s1) in zip(ops, sol):
        f = force_matrix(o, KAPPA) @ np.concatenate([x1, y1, s1])
        fx.append(f[:o.N])
        fy.append(f[o.N:])
    ux, uy, near = far_field(xs, ys, fx, fy, MU, near_mask=True)
    assert len(near) > 0
    cx, cy = near_correction(xs, ys, fx, fy, MU, near)
    ux, uy = ux + cx, uy + cy
    off = 0
    for v, (o, (x1, y1, s1)) in enumerate(zip(ops, sol)):
        N = o.N
        ub = np.concatenate(background(kind, fp, xs[v], ys[v]))
        U = o.S @ np.concatenate([fx[v], fy[v]]) + np.concatenate([ux[off:off + N], uy[off:off + N]]) + ub
        off += N
        r1 = np.concatenate([x1, y1]) - np.concatenate([xs[v], ys[v]]) - dt * U
        r2 = o.P @ U
        z = np.concatenate([x1, y1, s1])
        mag = np.abs(o.S) @ (np.abs(force_matrix(o, KAPPA)) @ np.abs(z))
        assert np.max(np.abs(r1)) <= 1e-12 * dt * np.max(mag), np.max(np.abs(r1))
        assert np.max(np.abs(r2)) <= 1e-15 * np.max(np.abs(o.P) @ mag), np.max(np.abs(r2))
    # and differs from the solution without the near field
    plain = implicit_solve(xs, ys, KAPPA, MU, dt, kind, fp)
    assert max(np.max(np.abs(a[2] - b[2])) for a, b in zip(sol, plain)) > 1e-6


def test_near_field_ying_zorin_solution_satisfies_both_lines():
    # as above with the Ying-Zorin evaluation as U_near^{n+1} (the ground truth's near-singular scheme)
    from oracle.yingzorin import near_correction_yz
    xs, ys = [], []
    for v, (cx, cy) in enumerate(((-0.36, 0.0), (0.36, 0.05), (0.0, 1.4))):
        x, y = _ves(32, 20 + v, cx, cy, R=0.5, theta=1.5 if v < 2 else 0.2)
        xs.append(x)
        ys.append(y)
    dt, kind, fp = 1e-3, 1, (1.0, 0, 0, 0)
    sol = implicit_solve(xs, ys, KAPPA, MU, dt, kind, fp, near_field=True, near_yz=True)
    ops = [Operators(x, y, KAPPA, MU) for x, y in zip(xs, ys)]
    fx, fy = [], []
    for o, (x1, y1, s1) in zip(ops, sol):
        f = force_matrix(o, KAPPA) @ np.concatenate([x1, y1, s1])
        fx.append(f[:o.N])
        fy.append(f[o.N:])
    ux, uy, near = far_field(xs, ys, fx, fy, MU, near_mask=True)
    assert near
    cx, cy = near_correction_yz(xs, ys, fx, fy, MU, near)
    ux, uy = ux + cx, uy + cy
    off = 0
    for v, (o, (x1, y1, s1)) in enumerate(zip(ops, sol)):
        N = o.N
        ub = np.concatenate(background(kind, fp, xs[v], ys[v]))
        U = o.S @ np.concatenate([fx[v], fy[v]]) + np.concatenate([ux[off:off + N], uy[off:off + N]]) + ub
        off += N
        r1 = np.concatenate([x1, y1]) - np.concatenate([xs[v], ys[v]]) - dt * U
        z = np.concatenate([x1, y1, s1])
        mag = np.abs(o.S) @ (np.abs(force_matrix(o, KAPPA)) @ np.abs(z))
        assert np.max(np.abs(r1)) <= 1e-12 * dt * np.max(mag), np.max(np.abs(r1))
        assert np.max(np.abs(o.P @ U)) <= 1e-15 * np.max(np.abs(o.P) @ mag)
