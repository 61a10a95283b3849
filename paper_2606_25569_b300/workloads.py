"""Seeded synthetic suspensions shaped like the paper's workloads (Sec. 5, Table tab:timings).

This module only draws inputs: vesicle outlines, centres, orientations and (for the far-field
workload) densities. It contains none of the time-step arithmetic, so both the CUDA library
and the FP64 oracle consume its output unchanged.

Outline recipe: an ellipse of equivalent radius R (area pi R^2) whose aspect ratio is found by
bisection so that its reduced area 4 pi A / L^2 equals nu (Sec. 3.4.1), sampled at the
parameters alpha_j = 2 pi j / N, plus seeded Fourier noise
    x_j += eps R sum_{k=1}^{8} (a_k cos k alpha_j + b_k sin k alpha_j) / k   (same for y),
a_k, b_k ~ N(0, 1), then a rotation. The points are not equally spaced in arclength: the
library (and the oracle) redistribute them when a suspension is created.
"""
from dataclasses import dataclass, field
from functools import lru_cache

import numpy as np


def _ellipse_perimeter(a, b):
    """Perimeter 4 a E(1 - b^2/a^2) of the ellipse with semi-axes a >= b (complete elliptic integral)."""
    from scipy.special import ellipe
    return float(4.0 * a * ellipe(1.0 - (b / a) ** 2))


@lru_cache(maxsize=65536)
def _aspect(nu):
    """q = a/b of the ellipse with reduced area nu (nu does not depend on the size), by bisection."""
    lo, hi = 1.0, 400.0
    for _ in range(80):
        q = 0.5 * (lo + hi)
        L = _ellipse_perimeter(np.sqrt(q), 1.0 / np.sqrt(q))
        if 4.0 * np.pi * np.pi / (L * L) > nu:
            lo = q
        else:
            hi = q
    return 0.5 * (lo + hi)


def ellipse_axes(nu, R):
    """Semi-axes (a, b), a >= b, of the ellipse with area pi R^2 and reduced area nu."""
    if not (0.0 < nu <= 1.0):
        raise ValueError("reduced area must be in (0, 1]")
    if nu == 1.0:
        return R, R
    q = _aspect(float(nu))
    return R * np.sqrt(q), R / np.sqrt(q)


def vesicle_outline(N, nu, R, eps, rng, theta):
    """One noisy, rotated ellipse outline centred at the origin (module header)."""
    a, b = ellipse_axes(nu, R)
    al = 2.0 * np.pi * np.arange(N) / N
    x = a * np.cos(al)
    y = b * np.sin(al)
    if eps > 0.0:
        k = np.arange(1, 9)[:, None]
        for comp in (0, 1):
            ca, cb = rng.standard_normal(8), rng.standard_normal(8)
            noise = eps * R * np.sum((ca[:, None] * np.cos(k * al) + cb[:, None] * np.sin(k * al)) / k, axis=0)
            if comp == 0:
                x = x + noise
            else:
                y = y + noise
    c, s = np.cos(theta), np.sin(theta)
    return c * x - s * y, s * x + c * y


@dataclass
class Workload:
    """A suspension: CSR points (x then y per vesicle, in one flat array) plus run parameters."""
    name: str
    xs: list
    ys: list
    kappa: float = 1.0
    mu: float = 1.0
    dt: float = 1e-4
    flow_kind: int = 0
    flow_p: tuple = (0.0, 0.0, 0.0, 0.0)
    steps: int = 1
    near_field: bool = False
    extra: dict = field(default_factory=dict)

    @property
    def M(self):
        return len(self.xs)

    @property
    def counts(self):
        return np.array([len(x) for x in self.xs], dtype=np.int64)

    @property
    def offsets(self):
        return np.concatenate([[0], np.cumsum(self.counts)]).astype(np.int64)

    def flat_xy(self):
        """CSR layout used by the library: per vesicle its N x values then its N y values."""
        return np.concatenate([np.concatenate([x, y]) for x, y in zip(self.xs, self.ys)])


def _place_random(M, radius, box, gap, rng, max_tries=200000):
    centres = np.zeros((M, 2))
    placed = 0
    tries = 0
    while placed < M:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place %d vesicles" % M)
        c = rng.uniform(-0.5 * box + radius, 0.5 * box - radius, size=2)
        if placed and np.min(np.hypot(*(centres[:placed] - c).T)) < 2.0 * radius + gap:
            continue
        centres[placed] = c
        placed += 1
    return centres


def single_shear(N=32, seed=1):
    """One vesicle, reduced area 0.65, R = 1, kappa = 1, shear u = (y, 0), dt = 1e-4, 200 steps."""
    rng = np.random.default_rng(seed)
    x, y = vesicle_outline(N, 0.65, 1.0, 1e-2, rng, rng.uniform(0, 2 * np.pi))
    return Workload("single vesicle 32 pts shear", [x], [y], kappa=1.0, mu=1.0, dt=1e-4,
                    flow_kind=1, flow_p=(1.0, 0.0, 0.0, 0.0), steps=200)


def taylor_green(M=64, N=128, seed=2, area_fraction=0.10):
    """M vesicles, R = 1, reduced areas U[0.6, 0.9], Taylor-Green flow (Eq. tayGreenFlow).

    Cell length W from the paper's ratio vesicle length / W = 0.4 (Sec. 5.5), U = W so the
    flow time scale W/U is 1; centres drawn without overlap in a square holding the requested
    area fraction; dt = 1e-3, 500 steps.
    """
    rng = np.random.default_rng(seed)
    nus = rng.uniform(0.6, 0.9, size=M)
    box = np.sqrt(M * np.pi / area_fraction)
    amax = max(ellipse_axes(float(nu), 1.0)[0] for nu in nus) * 1.1
    centres = _place_random(M, amax, box, 4.0 * 2 * np.pi * 1.0 / (0.6 ** 0.5) / N, rng)
    xs, ys = [], []
    for v in range(M):
        x, y = vesicle_outline(N, float(nus[v]), 1.0, 1e-2, rng, rng.uniform(0, 2 * np.pi))
        xs.append(x + centres[v, 0])
        ys.append(y + centres[v, 1])
    Lves = 2 * np.pi / np.sqrt(0.75)
    W = Lves / 0.4
    return Workload("taylor-green %dx%d" % (M, N), xs, ys, kappa=1.0, mu=1.0, dt=1e-3,
                    flow_kind=2, flow_p=(W, W, 0.0, 0.0), steps=500)


def farfield_box(M=2000, N=128, seed=3, R=0.08, box=20.0):
    """Far-field workload: M vesicles in a box, random orientations, densities f ~ N(0, 1).

    Returns (workload, fx list, fy list).
    """
    rng = np.random.default_rng(seed)
    nus = rng.uniform(0.6, 0.9, size=M)
    amax = ellipse_axes(0.6, R)[0] * 1.05
    centres = _place_random(M, amax, box, 0.0, rng)
    xs, ys, fxs, fys = [], [], [], []
    for v in range(M):
        x, y = vesicle_outline(N, float(nus[v]), R, 1e-2, rng, rng.uniform(0, 2 * np.pi))
        xs.append(x + centres[v, 0])
        ys.append(y + centres[v, 1])
        fxs.append(rng.standard_normal(N))
        fys.append(rng.standard_normal(N))
    return Workload("far field %dx%d box %g" % (M, N, box), xs, ys), fxs, fys


def poiseuille_dense(M=2000, N=64, seed=5, area_fraction=0.30, Cn=0.025, Ca=2.0, close_fraction=0.0, close_gap=0.5):
    """Dense Poiseuille suspension (Sec. 5.5): channel of width 1 (walls y = +-1/2),
    R = Cn W with W = 1/2, reduced area 0.65, u_max from Ca = 2 eta u_max R^3/(kappa W)
    (Sec. 5.3), dt = 0.01 W/u_max, jittered lattice with principal axes along x (Sec. 5.3).

    N: points per vesicle, or a sequence of point counts taken in turn (a suspension of uneven N).
    close_fraction: that fraction of the vesicles (every k-th) is moved along x towards its neighbour in the
    same lattice row until the smallest gap between them is close_gap times the larger arclength spacing
    h = L/N, so that the near-field rule (gap <= h) has pairs from the first step.
    """
    rng = np.random.default_rng(seed)
    W = 0.5
    R = Cn * W
    kappa, mu = 1.0, 1.0
    umax = Ca * kappa * W / (2.0 * mu * R ** 3)
    cell = np.pi * R * R / area_fraction
    a, b = ellipse_axes(0.65, R)
    rows = int(np.floor((2 * W) / np.sqrt(cell * (b / a) * 1.0)))
    rows = max(1, min(rows, int((2 * W - 2 * b) / (2.5 * b))))
    dy = (2 * W - 4 * b) / rows
    dx = cell / dy
    cols = int(np.ceil(M / rows))
    Ns = [int(N)] * M if np.isscalar(N) else [int(N[v % len(N)]) for v in range(M)]
    xs, ys = [], []
    for v in range(M):
        r, c = v % rows, v // rows
        cx = c * dx + rng.uniform(-0.1, 0.1) * (dx - 2 * a)
        cy = -W + 2 * b + (r + 0.5) * dy + rng.uniform(-0.1, 0.1) * (dy - 2 * b)
        x, y = vesicle_outline(Ns[v], 0.65, R, 1e-2, rng, rng.uniform(-0.05, 0.05))
        xs.append(x + cx)
        ys.append(y + cy)
    if close_fraction > 0.0:
        step = max(1, int(round(1.0 / close_fraction)))
        for v in range(0, M - rows, step):
            w = v + rows  # right-hand neighbour in the same row
            hv = np.sum(np.hypot(np.diff(xs[v], append=xs[v][0]), np.diff(ys[v], append=ys[v][0]))) / Ns[v]
            hw = np.sum(np.hypot(np.diff(xs[w], append=xs[w][0]), np.diff(ys[w], append=ys[w][0]))) / Ns[w]
            target = close_gap * max(hv, hw)

            def gap(shift):
                return np.sqrt(((xs[v] + shift)[:, None] - xs[w][None, :]) ** 2
                               + (ys[v][:, None] - ys[w][None, :]) ** 2).min()

            lo, hi = 0.0, float(xs[w].min() - xs[v].max()) + 2.0 * target
            if gap(0.0) <= target:
                continue
            for _ in range(60):  # bisection on the shift along x: the smallest point distance falls with it
                mid = 0.5 * (lo + hi)
                if gap(mid) > target:
                    lo = mid
                else:
                    hi = mid
            xs[v] = xs[v] + lo
    name = "poiseuille %dx%s af %.2f" % (M, N if np.isscalar(N) else "/".join(str(n) for n in N), area_fraction)
    if close_fraction > 0.0:
        name += " close %.2f at %.2f h" % (close_fraction, close_gap)
    return Workload(name, xs, ys, kappa=kappa, mu=mu,
                    dt=0.01 * W / umax, flow_kind=3, flow_p=(umax, W, 0.0, 0.0), steps=1000,
                    near_field=True, extra={"cols": cols, "dx": dx, "dy": dy})


def min_gap(xs, ys):
    """Smallest distance between points of different vesicles (brute force, for checks)."""
    P = np.stack([np.concatenate(xs), np.concatenate(ys)], axis=1)
    owner = np.repeat(np.arange(len(xs)), [len(x) for x in xs])
    best = np.inf
    for i in range(0, len(P), 256):
        d = np.hypot(P[i:i + 256, None, 0] - P[None, :, 0], P[i:i + 256, None, 1] - P[None, :, 1])
        d[owner[i:i + 256, None] == owner[None, :]] = np.inf
        best = min(best, float(d.min()))
    return best
