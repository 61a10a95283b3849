"""Far-field single-layer sum over all other vesicles (Sec. 2.2.2, Sec. 4.1, Algorithm 4).

Test infrastructure only.

u_far(x_i) = sum over vesicles v != vesicle(i) that are NOT near x_i of
             sum_j G(x_i - X_vj) f_vj |X_alpha|_vj (2 pi / N_v)        (trapezoid rule)
with the Stokeslet of oracle.stokes. Near-field rule (Eq. membrane_tension text, Sec. 3.3):
x_i is near vesicle v when its distance to v is at most v's arclength spacing h_v = L_v/N_v;
reading: the distance to the curve is taken as the minimum over v's discrete points.
Near pairs are excluded from this sum (Sec. 4.1: the mask zeroes them) and reported.

Brute force in FP64: every (target, source) pair is evaluated, then summed per source vesicle.
Pins (tests/test_oracle_farfield.py): exterior closed form of a circle with constant density,
S[n] = 0 at exterior targets, pure-Python loop on tiny inputs, mask semantics.
"""
import numpy as np

from .spectral import Geometry


def source_weights(xs, ys):
    """Per-point quadrature weight |X_alpha| 2 pi / N and arclength spacing h of each vesicle."""
    w, h = [], []
    for x, y in zip(xs, ys):
        g = Geometry(x, y)
        w.append(g.sa * 2.0 * np.pi / g.N)
        h.append(g.h)
    return w, np.array(h)


def far_field(xs, ys, fxs, fys, mu, near_mask=True, targets=None, chunk=32):
    """Far-field velocity at every point of every vesicle (or at a subset of global indices).

    xs, ys, fxs, fys: lists of per-vesicle arrays (uneven N allowed).
    Returns (ux, uy) as flat arrays over the selected targets, and the sorted list of near
    pairs (global target index, source vesicle) found.
    """
    M = len(xs)
    w, h = source_weights(xs, ys)
    counts = np.array([len(x) for x in xs])
    offsets = np.concatenate([[0], np.cumsum(counts)])
    X = np.concatenate(xs)
    Y = np.concatenate(ys)
    GX = np.concatenate([f * ww for f, ww in zip(fxs, w)])
    GY = np.concatenate([f * ww for f, ww in zip(fys, w)])
    owner = np.repeat(np.arange(M), counts)
    if targets is None:
        targets = np.arange(offsets[-1])
    targets = np.asarray(targets)
    c = 1.0 / (4.0 * np.pi * mu)
    ux = np.zeros(len(targets))
    uy = np.zeros(len(targets))
    near = []
    starts = offsets[:-1]
    for a in range(0, len(targets), chunk):
        t = targets[a:a + chunk]
        rx = X[t][:, None] - X[None, :]
        ry = Y[t][:, None] - Y[None, :]
        r2 = rx * rx + ry * ry
        own = owner[t][:, None] == owner[None, :]
        r2s = np.where(own, 1.0, r2)
        lg = -0.5 * np.log(r2s)
        rg = (rx * GX[None, :] + ry * GY[None, :]) / r2s
        cx = np.where(own, 0.0, lg * GX[None, :] + rg * rx)
        cy = np.where(own, 0.0, lg * GY[None, :] + rg * ry)
        sx = np.add.reduceat(cx, starts, axis=1)
        sy = np.add.reduceat(cy, starts, axis=1)
        keep = np.ones((len(t), M), dtype=bool)
        keep[np.arange(len(t)), owner[t]] = False
        if near_mask:
            minr2 = np.minimum.reduceat(np.where(own, np.inf, r2), starts, axis=1)
            is_near = minr2 <= (h ** 2)[None, :]
            is_near[np.arange(len(t)), owner[t]] = False
            for ti, v in zip(*np.nonzero(is_near)):
                near.append((int(t[ti]), int(v)))
            keep &= ~is_near
        ux[a:a + chunk] = c * np.where(keep, sx, 0.0).sum(axis=1)
        uy[a:a + chunk] = c * np.where(keep, sy, 0.0).sum(axis=1)
    near.sort()
    return ux, uy, near
