"""Near-field correction with five layers and Gaussian RBF interpolation (Sec. 3.3, Algorithm 4,
App. A). Test infrastructure only.

For a source vesicle v with near targets (oracle.farfield's rule):
1. layers: the N points moved along the outward normal by d h_v, d in {-1, -1/2, 0, 1/2, 1}
   (Sec. 3.3; h_v = L_v / N_v);
2. layer velocities S[X_v, f_v] at the 5N layer points. The plain step computes them exactly
   (Table tab:timings: "the input layers of velocities for RBF are computed exactly"):
   on the curve with the self rule (oracle.stokes), off the curve with the trapezoid rule on
   the curve upsampled by rho = ceil(sqrt(N)) (N rho >= N^{3/2} source points, the upsampling the
   paper quotes for near-singular evaluation, Sec. 2.2.2);
3. Gaussian RBF phi(r) = exp(-(r / (c h_v))^2) on the 5N layer points; the SPD system
   (Phi + lam I) w = u_layers is solved by Cholesky (Sec. 3.3);
4. the velocity at a near target x is sum_b phi(|x - x_b|) w_b; it replaces v's trapezoid
   contribution, which the far field masked (Algorithm 4).
Readings: the paper gives neither the RBF width nor a regularisation. We use c = 2 and
lam = 1e-3 (relative to the unit diagonal): on the App. A geometry this reproduces the exact
near-singular integral to about 1% (N = 32) and 0.6% (N = 64, 128) while keeping cond(Phi + lam I)
near 3e4, so an FP32 Cholesky (the paper's precision) agrees with FP64 to about 1e-6.

Pins (tests/test_oracle_nearfield.py): circle layer velocities against the interior/exterior
closed forms; zero response to the normal density; accuracy against the exact integral on the
App. A geometry (density (sin t, cos t)) far better than the plain trapezoid; linearity in f.
"""
import math

import numpy as np

from .spectral import Geometry, upsample
from .stokes import self_single_layer_matrix, single_layer_trapezoid

LAYERS = (-1.0, -0.5, 0.0, 0.5, 1.0)
RBF_C = 2.0
RBF_NUGGET = 1e-3


def upsample_factor(N):
    return int(math.ceil(math.sqrt(N)))


def layer_points(x, y):
    g = Geometry(x, y)
    LX = np.concatenate([x + d * g.h * g.nx for d in LAYERS])
    LY = np.concatenate([y + d * g.h * g.ny for d in LAYERS])
    return LX, LY, g.h


def layer_velocities(x, y, fx, fy, mu):
    """S[X, f] at the 5N layer points (layer-major order), step 2 of the module header."""
    N = len(x)
    g = Geometry(x, y)
    S = self_single_layer_matrix(x, y, mu)
    u0 = S @ np.concatenate([fx, fy])
    rho = upsample_factor(N)
    xu, yu = upsample(x, rho), upsample(y, rho)
    fxu, fyu = upsample(fx, rho), upsample(fy, rho)
    UX, UY = [], []
    for d in LAYERS:
        if d == 0.0:
            UX.append(u0[:N])
            UY.append(u0[N:])
        else:
            a, b = single_layer_trapezoid(xu, yu, fxu, fyu, x + d * g.h * g.nx, y + d * g.h * g.ny, mu)
            UX.append(a)
            UY.append(b)
    return np.concatenate(UX), np.concatenate(UY)


def rbf_weights(LX, LY, UX, UY, h):
    """Solve (Phi + lam I) w = u for both components by Cholesky (step 3)."""
    eps = RBF_C * h
    R2 = (LX[:, None] - LX[None, :]) ** 2 + (LY[:, None] - LY[None, :]) ** 2
    A = np.exp(-R2 / eps ** 2) + RBF_NUGGET * np.eye(len(LX))
    L = np.linalg.cholesky(A)
    W = np.linalg.solve(L.T, np.linalg.solve(L, np.stack([UX, UY], axis=1)))
    return W[:, 0], W[:, 1]


def rbf_eval(LX, LY, WX, WY, h, tx, ty):
    eps = RBF_C * h
    Q = np.exp(-((np.asarray(tx)[:, None] - LX[None, :]) ** 2 + (np.asarray(ty)[:, None] - LY[None, :]) ** 2) / eps ** 2)
    return Q @ WX, Q @ WY


def near_correction(xs, ys, fxs, fys, mu, near_pairs, layers=None):
    """Velocity added at every point (flat over all points) by the near-field rule of the
    sorted (target, source vesicle) pairs. layers(v) -> (UX, UY), when given, supplies source vesicle v's
    layer velocities instead of step 2 (the learned near field, oracle.learned.near_layers_learned)."""
    P = sum(len(x) for x in xs)
    X = np.concatenate(xs)
    Y = np.concatenate(ys)
    cx = np.zeros(P)
    cy = np.zeros(P)
    by_src = {}
    for t, v in near_pairs:
        by_src.setdefault(v, []).append(t)
    for v, targets in sorted(by_src.items()):
        LX, LY, h = layer_points(xs[v], ys[v])
        UX, UY = layer_velocities(xs[v], ys[v], fxs[v], fys[v], mu) if layers is None else layers(v)
        WX, WY = rbf_weights(LX, LY, UX, UY, h)
        t = np.array(targets)
        ax, ay = rbf_eval(LX, LY, WX, WY, h, X[t], Y[t])
        np.add.at(cx, t, ax)
        np.add.at(cy, t, ay)
    return cx, cy
