"""Fully implicit boundary-integral time step (Sec. 2.2.3, Eq. time_step_sc1): the paper's ground-truth
scheme. Test infrastructure only.

Operators are taken at X^n; bending, tension and the vesicle-vesicle interactions act on the new state.
Unknowns per vesicle a: X_a^{n+1} (2N_a) and sigma_a^{n+1} (N_a). With the force density
f_a = -kappa X_a,ssss + (sigma_a X_a,s)_s (linear in the unknowns, D_s and X_s of X^n) and the velocity
    U_a = S_a f_a + sum_{b != a} G_ab f_b        (self single layer + trapezoid rule of the others, Eq. single_layer)
the equations read
    X_a^{n+1} - dt U_a = X_a^n + dt u_inf(X_a^n)                         (first line of Eq. time_step_sc1)
    P_a U_a = -P_a u_inf(X_a^n)                                          (second line: L sigma + P (B X + U_far) = -P u_inf)
since L sigma + P B X = P S (Ten sigma - kappa D_s^4 X) = P S f. Readings: the first line of the printed
equation omits the background flow, which is read as part of the velocity (the vesicles move with the
flow); the near-field correction is left out (the oracle compares separated vesicles); the coupled dense
system is solved directly here (numpy), where the paper uses preconditioned GMRES, whose solution it is.
After the solve the step continues as the plain one: redistribution (Sec. 4.2) with sigma carried to the
new points by its trigonometric interpolant, then the area/length correction (Sec. 4.3).

With the near field on, the far-field sum excludes the (target, source vesicle) pairs of the near rule
(oracle.farfield) and the near-field correction of the density (oracle.nearfield, linear in it) is added
to U, as U_near^{n+1} of the printed equation (with Params.near_yz the Ying-Zorin evaluation, the ground
truth's own near-singular scheme); its matrix is assembled column by column from unit densities.

Pins (tests/test_oracle_implicit.py): for one vesicle the implicit step equals the advection with the
operators at X^n followed by the relaxation with the operators at X^n (an algebraic identity of the two
schemes); two vesicles mirrored across an axis of a symmetric background flow stay mirrored; the velocity
of the solved state satisfies both lines of the equation.
"""
import numpy as np

from . import correct as _corr
from .farfield import far_field
from .flows import background
from .operators import Operators
from .redistribute import redistribute
from .spectral import Geometry, eval_interpolant
from .stokes import stokeslet


def interaction_matrix(xa, ya, xb, yb, mu):
    """G_ab: velocity at the points of a from a force density on b by the trapezoid rule (2N_a x 2N_b)."""
    g = Geometry(xb, yb)
    w = g.sa * 2.0 * np.pi / g.N
    rx = xa[:, None] - xb[None, :]
    ry = ya[:, None] - yb[None, :]
    gxx, gxy, gyy = stokeslet(rx, ry, mu)
    return np.block([[gxx * w[None, :], gxy * w[None, :]], [gxy * w[None, :], gyy * w[None, :]]])


def force_matrix(ops, kappa):
    """F_a with f_a = F_a [x; y; sigma]: -kappa D_s^4 on each coordinate and Ten on sigma."""
    N = ops.N
    D4 = ops.Ds @ ops.Ds @ ops.Ds @ ops.Ds
    Z = np.zeros((N, N))
    return np.block([[-kappa * D4, Z, ops.Ten[:N]], [Z, -kappa * D4, ops.Ten[N:]]])


def near_blocks(xs, ys, mu, yz=False):
    """Near pairs of the far-field rule and, per source vesicle b with near targets, the dense map from
    f_b = [f_x; f_y] (2 N_b) to the near-field correction at every point ([u_x over all points; u_y]); yz: by
    the Ying-Zorin evaluation (oracle.yingzorin) instead of the layers and the RBF."""
    from .nearfield import near_correction
    from .yingzorin import near_correction_yz
    correction = near_correction_yz if yz else near_correction
    zero = [np.zeros(len(x)) for x in xs]
    _, _, near = far_field(xs, ys, zero, zero, mu, near_mask=True)
    P = sum(len(x) for x in xs)
    blocks = {}
    for b in sorted({v for _, v in near}):
        pairs = [(t, v) for t, v in near if v == b]
        Nb = len(xs[b])
        Nmat = np.zeros((2 * P, 2 * Nb))
        for c in range(2 * Nb):
            fx = [np.zeros(len(x)) for x in xs]
            fy = [np.zeros(len(x)) for x in xs]
            (fx if c < Nb else fy)[b][c % Nb] = 1.0
            cx, cy = correction(xs, ys, fx, fy, mu, pairs)
            Nmat[:, c] = np.concatenate([cx, cy])
        blocks[b] = Nmat
    return near, blocks


def implicit_solve(xs, ys, kappa, mu, dt, flow_kind, flow_p, near_field=False, near_yz=False):
    """X^{n+1}, sigma^{n+1} of Eq. time_step_sc1 for every vesicle (before redistribution)."""
    M = len(xs)
    Ns = [len(x) for x in xs]
    off = np.concatenate([[0], np.cumsum([3 * n for n in Ns])])
    poff = np.concatenate([[0], np.cumsum(Ns)])
    P = poff[-1]
    n_all = off[-1]
    ops = [Operators(x, y, kappa, mu) for x, y in zip(xs, ys)]
    F = [force_matrix(o, kappa) for o in ops]
    near, blocks = near_blocks(xs, ys, mu, near_yz) if near_field else ([], {})
    near_set = set(near)
    A = np.zeros((n_all, n_all))
    b = np.zeros(n_all)
    for a in range(M):
        Na = Ns[a]
        ra = slice(off[a], off[a + 1])
        ub = np.concatenate(background(flow_kind, flow_p, xs[a], ys[a]))
        # U_a = sum_b V_ab z_b with V_ab = G_ab F_b (G_aa = S_a)
        V = []
        for bb in range(M):
            if bb == a:
                G = ops[a].S
            else:
                G = interaction_matrix(xs[a], ys[a], xs[bb], ys[bb], mu)
                # targets of a near b: the trapezoid rule is replaced by the near-field correction
                for i in range(Na):
                    if (poff[a] + i, bb) in near_set:
                        G[i, :] = 0.0
                        G[Na + i, :] = 0.0
                if bb in blocks:
                    rows = np.concatenate([np.arange(poff[a], poff[a + 1]), P + np.arange(poff[a], poff[a + 1])])
                    G = G + blocks[bb][rows]
            V.append(G @ F[bb])
        rows_x = np.zeros((2 * Na, n_all))
        rows_s = np.zeros((Na, n_all))
        for bb in range(M):
            cb = slice(off[bb], off[bb + 1])
            rows_x[:, cb] -= dt * V[bb]
            rows_s[:, cb] += ops[a].P @ V[bb]
        rows_x[:, off[a]:off[a] + 2 * Na] += np.eye(2 * Na)
        A[off[a]:off[a] + 2 * Na] = rows_x
        A[off[a] + 2 * Na:off[a + 1]] = rows_s
        b[off[a]:off[a] + 2 * Na] = np.concatenate([xs[a], ys[a]]) + dt * ub
        b[off[a] + 2 * Na:off[a + 1]] = -ops[a].P @ ub
    z = np.linalg.solve(A, b)
    out = []
    for a in range(M):
        Na = Ns[a]
        za = z[off[a]:off[a + 1]]
        out.append((za[:Na], za[Na:2 * Na], za[2 * Na:]))
    return out


class ImplicitSuspension:
    """State (X, sigma, A_0, L_0) advanced by the implicit step (module header); created like
    oracle.step.Suspension (redistributed X^0, sigma^0 of the plain step's reading)."""

    def __init__(self, xs, ys, params):
        from .step import Suspension
        s = Suspension(xs, ys, params)
        self.p = params
        self.xs, self.ys, self.sig, self.A0, self.L0 = s.xs, s.ys, s.sig, s.A0, s.L0
        self.corrections = 0

    def step(self):
        p = self.p
        sol = implicit_solve(self.xs, self.ys, p.kappa, p.mu, p.dt, p.flow_kind, p.flow_p, near_field=p.near_field,
                             near_yz=p.near_yz)
        nxs, nys, nsig = [], [], []
        for v, (x1, y1, s1) in enumerate(sol):
            xr, yr, alpha = redistribute(x1, y1)
            sr = eval_interpolant(s1, alpha)
            xc, yc, fired, _ = _corr.correct(xr, yr, self.A0[v], self.L0[v], tol=p.corr_tol)
            self.corrections += int(fired)
            nxs.append(xc)
            nys.append(yc)
            nsig.append(sr)
        self.xs, self.ys, self.sig = nxs, nys, nsig
