"""Pins for oracle.mlp (Sec. 3.4.2): finite-difference gradients, AdamW closed form, bf16 rounding."""
import numpy as np

from oracle.mlp import AdamW, bf16_round, init_params, loss_and_gradient, forward


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    dims = [8, 12, 10, 8]
    p = init_params(dims, rng) + 0.01 * rng.standard_normal(sum(a * b + b for a, b in zip(dims[:-1], dims[1:])))
    X = rng.standard_normal((5, 8))
    Y = rng.standard_normal((5, 8))
    loss, g = loss_and_gradient(p, dims, X, Y, beta=0.7, ncomp=2)
    h = 1e-6
    idx = rng.choice(len(p), 40, replace=False)
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (loss_and_gradient(p + e, dims, X, Y, 0.7, 2)[0] - loss_and_gradient(p - e, dims, X, Y, 0.7, 2)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_perfect_prediction_has_zero_loss():
    rng = np.random.default_rng(1)
    dims = [6, 9, 4]
    p = init_params(dims, rng)
    X = rng.standard_normal((3, 6))
    Y, _ = forward(p, dims, X)
    loss, g = loss_and_gradient(p, dims, X, Y, beta=1.0, ncomp=2)
    assert loss == 0.0 and np.all(g == 0.0)


def test_adamw_first_step_closed_form():
    # first step: mhat = g, vhat = g^2, so w1 = w0 (1 - lr wd) - lr g / (|g| + eps)
    rng = np.random.default_rng(2)
    w = rng.standard_normal(50)
    g = rng.standard_normal(50)
    opt = AdamW(50, lr=1e-3, weight_decay=0.01)
    w1 = opt.step(w, g)
    assert np.allclose(w1, w * (1 - 1e-5) - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_bf16_rounding_ties_to_even():
    # 1 + 2^-8 lies halfway between bf16 neighbours 1 and 1 + 2^-7: rounds to 1 (even)
    assert bf16_round(np.array([1.0 + 2 ** -8]))[0] == 1.0
    assert bf16_round(np.array([1.0 + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6
    assert bf16_round(np.array([-2.5]))[0] == -2.5
    x = np.array([3.14159265])
    assert abs(bf16_round(x)[0] - x[0]) <= 2 ** -8 * 4


def _folded(p, dims, aff):
    """The same network with the affine maps folded into the first and last layers."""
    from oracle.mlp import unpack
    ws, bs = unpack(p, dims)
    ws, bs = [w.copy() for w in ws], [b.copy() for b in bs]
    sh, sc, osh, osc = aff
    bs[0] = bs[0] - ws[0] @ (sh * sc)
    ws[0] = ws[0] * sc[None, :]
    ws[-1] = ws[-1] * osc[:, None]
    bs[-1] = bs[-1] * osc + osh
    return np.concatenate([w.ravel() for w in ws] + bs)


def _affine(rng, d0, dL):
    return (rng.standard_normal(d0), rng.uniform(0.5, 3.0, d0), rng.standard_normal(dL), rng.uniform(0.1, 2.0, dL))


def test_affine_maps_fold_into_first_and_last_layers():
    rng = np.random.default_rng(5)
    dims = [6, 10, 8, 4]
    p = init_params(dims, rng) + 0.05 * rng.standard_normal(sum(a * b + b for a, b in zip(dims[:-1], dims[1:])))
    aff = _affine(rng, 6, 4)
    X = rng.standard_normal((7, 6))
    Ya, _ = forward(p, dims, X, affine=aff)
    Yf, _ = forward(_folded(p, dims, aff), dims, X)
    assert np.max(np.abs(Ya - Yf)) <= 1e-12 * np.max(np.abs(Yf))


def test_affine_loss_zero_at_mapped_prediction_and_gradient_by_differences():
    rng = np.random.default_rng(6)
    dims = [8, 12, 8]
    p = init_params(dims, rng) + 0.01 * rng.standard_normal(sum(a * b + b for a, b in zip(dims[:-1], dims[1:])))
    aff = _affine(rng, 8, 8)
    X = rng.standard_normal((4, 8))
    Yp, _ = forward(p, dims, X, affine=aff)
    loss0, _ = loss_and_gradient(p, dims, X, Yp, beta=0.5, ncomp=2, affine=aff)
    assert loss0 <= 1e-12
    Y = rng.standard_normal((4, 8))
    loss, g = loss_and_gradient(p, dims, X, Y, beta=0.5, ncomp=2, affine=aff)
    h = 1e-6
    for i in rng.choice(len(p), 30, replace=False):
        e = np.zeros_like(p)
        e[i] = h
        fd = (loss_and_gradient(p + e, dims, X, Y, 0.5, 2, affine=aff)[0]
              - loss_and_gradient(p - e, dims, X, Y, 0.5, 2, affine=aff)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])
