"""Helpers shared by the GPU parity tests (no arithmetic of the method here)."""
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
