"""Helpers shared by the GPU parity tests (no arithmetic of the method here)."""
import functools

import numpy as np


def csr(xs, ys):
    return np.concatenate([np.concatenate([x, y]) for x, y in zip(xs, ys)])


def offsets(xs):
    return np.concatenate([[0], np.cumsum([len(x) for x in xs])]).astype(np.int64)


def split(flat, counts):
    """CSR blocks -> (list of x, list of y)."""
    xs, ys = [], []
    o = 0
    for n in counts:
        xs.append(flat[2 * o:2 * o + n])
        ys.append(flat[2 * o + n:2 * o + 2 * n])
        o += n
    return xs, ys


def rel_err_per_vesicle(xs_a, ys_a, xs_b, ys_b):
    """max over vesicles of ||X_a - X_b|| / ||X_b||."""
    e = 0.0
    for xa, ya, xb, yb in zip(xs_a, ys_a, xs_b, ys_b):
        d = np.sqrt(np.sum((xa - xb) ** 2 + (ya - yb) ** 2))
        n = np.sqrt(np.sum(xb ** 2 + yb ** 2))
        e = max(e, d / n)
    return e


# Tension tolerances. sigma = -L^-1 P (B X + u) is sensitive to rounding-level differences in X (B is a
# fourth derivative smoothed once by S): in the FP64 oracle itself, seeded white noise of 2e-13 of the
# vesicle's size in X moves sigma by 1.1e-10..6.0e-10 of its largest value on the 128-point Taylor-Green
# vesicles (and 5e-11..8e-11 at 64 points), spread over all of its modes. The two sides agree in X to
# about 2e-13 after a step, so sigma is held to 1e-10 where N <= 32 and to 1e-9 where N >= 64.
SIGMA_TOL, SIGMA_TOL_N64 = 1e-10, 1e-9
# the same sensitivity per unit of relative position difference: 1.1e-10..6.0e-10 for 1e-13..2e-13, i.e. up
# to about 3e3 on those vesicles
SIGMA_PER_X = 5e3


def sigma_error(sg, so_list):
    """Largest difference of the library's flat tension sg from the oracle's per-vesicle arrays, relative to
    the largest |sigma| of the oracle."""
    so = np.concatenate(so_list)
    return float(np.max(np.abs(sg - so)) / np.max(np.abs(so)))


def sigma_tolerance(so_list, tol_s=None, ex=0.0):
    """tol_s, or the FP64 tolerance of SIGMA_TOL for the largest vesicle; along a trajectory whose positions
    differ by ex (relative), at least SIGMA_PER_X * ex (the sensitivity measured on the oracle, rounded up)."""
    if tol_s is not None:
        return tol_s
    base = SIGMA_TOL if max(len(s) for s in so_list) <= 32 else SIGMA_TOL_N64
    return max(base, SIGMA_PER_X * ex)


def _elementwise(got, ref):
    """Per-element error relative to the element's size plus the root mean square of the reference (the
    floor keeps elements that happen to be near zero from reading as large relative errors)."""
    return np.abs(got - ref) / (np.abs(ref) + np.sqrt(np.mean(ref ** 2)))


def check_network_output(got, ref, tol_l2, tol_elem, what):
    """Relative L2 error within tol_l2 and every element (_elementwise) within tol_elem."""
    l2 = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    e = _elementwise(got, ref)
    print("%s: relative L2 %.3e, element-wise max %.3e (99.9%% %.3e)" % (what, l2, e.max(), np.quantile(e, 0.999)))
    assert l2 <= tol_l2, l2
    assert e.max() <= tol_elem, e.max()


@functools.lru_cache(maxsize=1)
def poiseuille_oracle_state():
    """The oracle's own initial state of the dense Poiseuille suspension (2000 x 64, seed 5; its
    redistribution and initial tension) and the membrane forces at it: (workload, oracle suspension, fx, fy).
    Expected values built on it never pass through the library."""
    from oracle.spectral import force
    from oracle.step import Params, Suspension
    from paper_2606_25569_b300.workloads import poiseuille_dense
    wl = poiseuille_dense(2000, 64, seed=5)
    p = Params(kappa=wl.kappa, mu=wl.mu, dt=wl.dt, flow_kind=wl.flow_kind, flow_p=wl.flow_p, corr_tol=0.01,
               near_field=True)
    o = Suspension(wl.xs, wl.ys, p)
    fx, fy = [], []
    for v in range(wl.M):
        a, b = force(o.xs[v], o.ys[v], o.sig[v], wl.kappa)
        fx.append(a)
        fy.append(b)
    return wl, o, fx, fy
