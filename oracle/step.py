"""One plain boundary-integral time step for a suspension (Algorithm 1 with exact operators).

Test infrastructure only.

Per step, in this order (Sec. 3.1, Algorithm 1, Sec. 4.2-4.3):
1. force f^n = -kappa X_ssss + (sigma^n X_s)_s at X^n                         (Eq. elastic_force)
2. u^n = U_far + U_near + u_inf at X^n                                       (Algorithm 4)
3. advection  X* = X^n + dt (I - M^n) u^n                                    (Eq. advection_disc)
4. relaxation (I - dt (I - M*) B*) X^{n+1} = X*                              (Eq. relaxation_disc)
5. redistribution of X^{n+1} to equal arclength                               (Sec. 4.2)
6. tension sigma^{n+1} = -L^{-1} P (B X^{n+1} + u^n), operators at the
   redistributed X^{n+1}, u^n resampled at the new parameters                (Eq. tension_disc)
7. area/length correction when either relative error exceeds corr_tol         (Sec. 4.3)

Pins (tests/test_oracle_step.py): relaxation lowers the bending energy, area and length drift first
order in dt, translation/rotation equivariance, first-order convergence in time, a uniform background
translates a vesicle rigidly, the proximity rule on circles at known gaps; the tension update makes the
total membrane velocity u + S[f(sigma)] inextensible (surface divergence below 1e-10 of that without
tension, under shear and Taylor-Green, for sigma^0 and after a step), with f from the force's own
definition rather than the operator matrices.

Readings: Eq. tension_disc writes L^n, P^n while Algorithm 1-2 evaluate them at X^{n+1}; we
use X^{n+1} after redistribution (step 6), and since redistribution re-indexes the material
points, u^n is carried to the new points by its trigonometric interpolant. Algorithm 1
computes the tension before the correction and so do we. One far-field evaluation per step
(Algorithm 1 needs u^n once). With Params.relax_net set, step 4 is the learned relaxation of the
hybrid step (relax_learned), except for vesicles in a near pair this step (the target's owner or the
source vesicle) or within exact_gap (default HYBRID_EXACT_GAP) spacings of another vesicle, and, with exact_every = m > 0,
on every m-th step: those relax exactly, the plain step serving as the fallback of the learned one (reading: the paper's VesNet learns the near interactions
too; here they keep the exact relaxation). With Params.flow_net set as well, steps 3 and 6 of every step
take the learned advection and tension of oracle.learned (Eqs. advectionMap, advTenMap), except for the
vesicles of that fallback set, which keep the exact ones. With Params.near_net set as well (and the near
field on), step 2's near-field layer velocities of every source vesicle come from the learned near field
(oracle.learned.near_layers_learned, Sec. 3.3) in every step; otherwise, with Params.near_yz, step 2's near
field is the Ying-Zorin evaluation (oracle.yingzorin) instead of the layers and the RBF. Initial tension (not given in the paper):
sigma^0 = -L^{-1} P (B X^0 + u_inf(X^0)) after redistributing X^0, which also fixes A_0, L_0.
"""
import numpy as np

from . import correct as _corr
from .farfield import far_field
from .flows import background
from .operators import Operators
from .redistribute import redistribute
from .spectral import Geometry, eval_interpolant, force


HYBRID_EXACT_GAP = 4.0


class Params:
    def __init__(self, kappa=1.0, mu=1.0, dt=1e-4, flow_kind=0, flow_p=(0.0, 0.0, 0.0, 0.0),
                 near_field=False, corr_tol=0.01, relax_net=None, exact_every=0, exact_gap=HYBRID_EXACT_GAP,
                 flow_net=None, near_net=None, near_yz=False):
        self.kappa, self.mu, self.dt = float(kappa), float(mu), float(dt)
        self.flow_kind, self.flow_p = int(flow_kind), tuple(float(v) for v in flow_p)
        self.near_field, self.corr_tol = bool(near_field), float(corr_tol)
        # (dims, flat parameters, output scale, filter kmax[, affine]): the learned relaxation of the hybrid
        # step; with exact_every = m > 0 every m-th step (counting from 1) relaxes exactly instead
        self.relax_net = relax_net
        self.exact_every = int(exact_every)
        # in a learned step, vesicles within exact_gap spacings h of another vesicle relax exactly
        self.exact_gap = float(exact_gap)
        # (adv, ten, Kf, Kout), each network (dims, flat parameters, affine or None) or a function of the
        # vesicle (x, y) giving its output row: with relax_net set, the
        # advection and the tension of every step come from them (oracle.learned), for every vesicle
        self.flow_net = flow_net
        # (nets, Kf, Kout), nets the five layer networks (as flow_net's entries), layer order -h .. h: with
        # relax_net set and the near field on, the near-field layer velocities come from them
        self.near_net = near_net
        # the near field by the Ying-Zorin scheme (oracle.yingzorin) instead of the layers and the RBF
        self.near_yz = bool(near_yz)


def relax_learned(x, y, net):
    """Hybrid relaxation (VesNet's X_X map, Sec. 3.2, 3.4.1): redistribute X* (Sec. 4.2),
    standardise, evaluate the network on the Fourier features of the standardised shape (modes
    k <= K = min(kmax, N/2 - 1), zero-padded to the width 16 ceil((4K + 2)/16); bfloat16 operands as on
    the tensor cores, input first rounded to float32), synthesise the displacement from the scaled
    output's features, map it back to the original frame, add it to X*_r and remove the modes |k| > K
    of the result (the network represents only those modes). net = (dims, params, scale, kmax[, affine]),
    affine the network's per-feature input and output maps (oracle.mlp)."""
    from .mlp import forward
    from .standardize import (destandardize_disp, feature_count, features_to_samples, fourier_features,
                              fourier_filter, standardize)
    dims, params, scale, kmax = net[:4]
    affine = net[4] if len(net) > 4 else None
    N = len(x)
    K = min(kmax, N // 2 - 1)
    xr, yr, _ = redistribute(x, y)
    xo, yo, fr = standardize(xr, yr)
    inp = np.zeros((1, dims[0]))
    inp[0, :feature_count(K)] = fourier_features(xo, yo, K)
    out, _ = forward(params, dims, inp, bf16=True, affine=affine)
    ddx, ddy = features_to_samples(scale * out[0, :feature_count(K)], K, N)
    dx, dy = destandardize_disp(ddx, ddy, fr)
    return np.concatenate([fourier_filter(xr + dx, kmax), fourier_filter(yr + dy, kmax)])


def flow_row(x, y, net, kmax):
    """The flow network's output row for the vesicle (x, y): its input is the relaxation network's, the
    Fourier features (modes <= min(kmax, N/2 - 1)) of the standardised shape (bfloat16 operands as on the
    tensor cores, input first rounded to float32)."""
    from .mlp import forward
    from .standardize import feature_count, fourier_features, standardize
    if callable(net):  # any function of the vesicle giving its row (the pins pass the exact columns)
        return net(x, y)
    dims, params, affine = net
    K = min(kmax, len(x) // 2 - 1)
    xo, yo, _ = standardize(x, y)
    inp = np.zeros((1, dims[0]))
    inp[0, :feature_count(K)] = fourier_features(xo, yo, K)
    out, _ = forward(params, dims, inp, bf16=True, affine=affine)
    return out[0]


def relax_exact(x, y, p):
    """Relaxation (Eq. relaxation_disc): solve (I - dt (I - M*) B*) X^{n+1} = X*."""
    N = len(x)
    ops_s = Operators(x, y, p.kappa, p.mu)
    A = np.eye(2 * N) - p.dt * (ops_s.B - ops_s.T @ np.linalg.solve(ops_s.L, ops_s.P @ ops_s.B))
    return np.linalg.solve(A, np.concatenate([x, y]))


def _tension(ops, x, y, ux, uy, kappa):
    N = len(x)
    rhs = ops.P @ (ops.B @ np.concatenate([x, y]) + np.concatenate([ux, uy]))
    return -np.linalg.solve(ops.L, rhs)


class Suspension:
    """State (X, sigma, A_0, L_0) of M vesicles and the plain step (module header)."""

    def __init__(self, xs, ys, params):
        self.p = params
        self.xs, self.ys, self.sig, self.A0, self.L0 = [], [], [], [], []
        for x, y in zip(xs, ys):
            xr, yr, _ = redistribute(np.asarray(x, float), np.asarray(y, float))
            g = Geometry(xr, yr)
            ops = Operators(xr, yr, params.kappa, params.mu)
            ub = background(params.flow_kind, params.flow_p, xr, yr)
            self.xs.append(xr)
            self.ys.append(yr)
            self.sig.append(_tension(ops, xr, yr, ub[0], ub[1], params.kappa))
            self.A0.append(g.area)
            self.L0.append(g.length)
        self.velocity = [np.zeros(2 * len(x)) for x in self.xs]
        self.corrections = 0
        self.near_pairs = []

    def interaction_velocity(self):
        """u^n = U_far + U_near + u_inf at the current points (Algorithm 1, first line)."""
        p = self.p
        fx, fy = [], []
        for x, y, s in zip(self.xs, self.ys, self.sig):
            a, b = force(x, y, s, p.kappa)
            fx.append(a)
            fy.append(b)
        ux, uy, near = far_field(self.xs, self.ys, fx, fy, p.mu, near_mask=p.near_field)
        if p.near_field and near:
            from .nearfield import near_correction
            layers = None
            if p.relax_net is not None and p.near_net is not None:
                from .learned import near_layers_learned
                nets, Kf, Kout = p.near_net
                kmax = p.relax_net[3]

                def layers(v):
                    rows = [flow_row(self.xs[v], self.ys[v], net, kmax) for net in nets]
                    return near_layers_learned(self.xs[v], self.ys[v], fx[v], fy[v], rows, Kf, Kout, p.mu)
            if p.near_yz and layers is None:
                from .yingzorin import near_correction_yz
                cx, cy = near_correction_yz(self.xs, self.ys, fx, fy, p.mu, near)
            else:
                cx, cy = near_correction(self.xs, self.ys, fx, fy, p.mu, near, layers=layers)
            ux = ux + cx
            uy = uy + cy
        self.near_pairs = near
        out = []
        o = 0
        for x, y in zip(self.xs, self.ys):
            n = len(x)
            bx, by = background(p.flow_kind, p.flow_p, x, y)
            out.append((ux[o:o + n] + bx, uy[o:o + n] + by))
            o += n
        return out

    def step(self):
        p = self.p
        self.nstep = getattr(self, "nstep", 0) + 1
        # learned advection and tension in every step of a hybrid suspension with flow networks
        flow = (p.flow_net, p.relax_net[3]) if p.relax_net is not None and p.flow_net is not None else None
        if p.relax_net is not None and p.exact_every > 0 and self.nstep % p.exact_every == 0:
            import copy
            p = copy.copy(p)
            p.relax_net = None
        u = self.interaction_velocity()
        # in a learned step, vesicles in a near pair (as the target's owner or as the source) relax exactly; with
        # the flow networks they also take the exact advection and tension, in every step
        exact = set()
        if p.relax_net is not None or flow is not None:
            owner = np.repeat(np.arange(len(self.xs)), [len(x) for x in self.xs])
            for t, v in self.near_pairs:
                exact.update((int(owner[t]), int(v)))
            exact.update(close_vesicles(self.xs, self.ys, p.exact_gap))
        nxs, nys, nsig, vel = [], [], [], []
        for v, (x, y) in enumerate(zip(self.xs, self.ys)):
            ux, uy = u[v]
            pv, fv = p, flow
            if v in exact:
                import copy
                pv = copy.copy(p)
                pv.relax_net = None
                fv = None
            xc, yc, sig, fired = advance_vesicle(x, y, ux, uy, self.A0[v], self.L0[v], pv, fv)
            self.corrections += int(fired)
            nxs.append(xc)
            nys.append(yc)
            nsig.append(sig)
            vel.append(np.concatenate([ux, uy]))
        self.xs, self.ys, self.sig, self.velocity = nxs, nys, nsig, vel


def close_vesicles(xs, ys, gap_h):
    """Vesicles with a point within gap_h * max(h_a, h_b) of a point of another vesicle b, h = L/N
    (brute force over all pairs of points)."""
    hs = [Geometry(x, y).length / len(x) for x, y in zip(xs, ys)]
    out = set()
    for a in range(len(xs)):
        for b in range(a + 1, len(xs)):
            d2 = (xs[a][:, None] - xs[b][None, :]) ** 2 + (ys[a][:, None] - ys[b][None, :]) ** 2
            if d2.min() <= (gap_h * max(hs[a], hs[b])) ** 2:
                out.update((a, b))
    return out


def advance_vesicle(x, y, ux, uy, A0, L0, p, flow=None):
    """Steps 3-7 of the module header for one vesicle at X^n = (x, y) given its velocity u^n = (ux, uy):
    returns (x^{n+1}, y^{n+1}, sigma^{n+1}, correction fired). flow = ((adv, ten, Kf, Kout), kmax): the
    advection and the tension from the networks (oracle.learned)."""
    N = len(x)
    ubar = np.concatenate([ux, uy])
    if flow is not None:
        from .learned import advect_learned
        (adv, ten, Kf, Kout), kmax = flow
        zx, zy = advect_learned(x, y, ux, uy, p.dt, flow_row(x, y, adv, kmax), Kf, Kout)
        zs = np.concatenate([zx, zy])
    else:
        ops_n = Operators(x, y, p.kappa, p.mu)
        zs = np.concatenate([x, y]) + p.dt * ops_n.project(ubar)
    if p.relax_net is not None:
        z1 = relax_learned(zs[:N], zs[N:], p.relax_net)
    else:
        z1 = relax_exact(zs[:N], zs[N:], p)
    xr, yr, alpha = redistribute(z1[:N], z1[N:])
    uxr, uyr = eval_interpolant(ux, alpha), eval_interpolant(uy, alpha)
    if flow is not None:
        from .learned import tension_learned
        sig = tension_learned(xr, yr, uxr, uyr, flow_row(xr, yr, ten, kmax), Kf, Kout)
    else:
        ops_r = Operators(xr, yr, p.kappa, p.mu)
        sig = _tension(ops_r, xr, yr, uxr, uyr, p.kappa)
    xc, yc, fired, _ = _corr.correct(xr, yr, A0, L0, tol=p.corr_tol)
    return xc, yc, sig, fired
