"""Pins for oracle.ivnet (Sec. 3.4.2, Fig. fig:net)."""
import numpy as np

from oracle.ivnet import (convs, forward, gather, init_params, loss_and_gradient, param_count, scatter, unpack,
                          up, up_T)


def test_convolution_against_explicit_loops():
    rng = np.random.default_rng(1)
    B, n, ci, co, k, s, d = 2, 8, 3, 4, 3, 2, 2
    x = rng.standard_normal((B, n, ci))
    W = rng.standard_normal((co, ci, k))
    b = rng.standard_normal(co)
    col = gather(x, k, s, d)
    got = col @ W.reshape(co, -1).T + b
    ref = np.zeros((B, n // s, co))
    for bb in range(B):
        for p in range(n // s):
            for o in range(co):
                acc = b[o]
                for c in range(ci):
                    for t in range(k):
                        acc += W[o, c, t] * x[bb, (s * p + d * (t - 1)) % n, c]
                ref[bb, p, o] = acc
    assert np.max(np.abs(got - ref)) < 1e-12


def test_gather_and_interpolation_adjoints():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 16, 3))
    g = rng.standard_normal((2, 8, 9))
    assert abs(np.sum(gather(x, 3, 2, 2) * g) - np.sum(x * scatter(g, 16, 3, 3, 2, 2))) < 1e-11
    y = rng.standard_normal((2, 32, 3))
    assert abs(np.sum(up(x) * y) - np.sum(x * up_T(y))) < 1e-11
    # interpolation keeps the samples and averages neighbours
    u = up(x)
    assert np.array_equal(u[:, 0::2], x)
    assert np.allclose(u[:, 1::2], 0.5 * (x + np.roll(x, -1, axis=1)))


def test_gradient_against_finite_differences():
    C, nb, N, B = 8, 2, 16, 3
    rng = np.random.default_rng(3)
    p = init_params(C, nb, rng)
    p[-2:] = 0.1  # non-zero output bias
    X = rng.standard_normal((B, 2 * N))
    Y = rng.standard_normal((B, 2 * N))
    _, g = loss_and_gradient(p, C, nb, X, Y, beta=0.5)
    idx = rng.choice(len(p), 40, replace=False)
    for i in idx:
        e = np.zeros(len(p))
        e[i] = 1e-6
        lp, _ = loss_and_gradient(p + e, C, nb, X, Y, beta=0.5)
        lm, _ = loss_and_gradient(p - e, C, nb, X, Y, beta=0.5)
        fd = (lp - lm) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_equivariant_under_shifts_by_multiples_of_four():
    # circular convolutions with two stride-2 levels: shifting the points by 4 shifts the output by 4
    C, nb, N = 8, 2, 32
    rng = np.random.default_rng(4)
    p = init_params(C, nb, rng)
    X = rng.standard_normal((2, 2 * N))
    sh = lambda R, m: np.concatenate([np.roll(R[:, :N], m, axis=1), np.roll(R[:, N:], m, axis=1)], axis=1)
    Y, _ = forward(p, C, nb, X)
    Ys, _ = forward(p, C, nb, sh(X, 4))
    assert np.max(np.abs(Ys - sh(Y, 4))) < 1e-12
    Y2, _ = forward(p, C, nb, sh(X, 2))  # not a multiple of 4: the strided levels see other points
    assert np.max(np.abs(Y2 - sh(Y, 2))) > 1e-6


def test_parameter_layout():
    C, nb = 64, 8
    assert param_count(C, nb) == 429122
    p = np.arange(param_count(C, nb), dtype=np.float64)
    ws, bs = unpack(p, C, nb)
    assert len(ws) == len(convs(C, nb)) == 2 + 7 * nb
    assert ws[0].shape == (C, 2, 3) and bs[-1].shape == (2,)
    assert ws[1].shape == (C // 2, C, 3) and ws[7].shape == (C, C, 1)
