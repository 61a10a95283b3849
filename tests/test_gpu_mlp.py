"""GPU parity of the tensor-core MLP (forward, gradients, AdamW) against the FP64 oracle with the
same bfloat16 rounding points (oracle.mlp, bf16=True)."""
import numpy as np
import pytest

from oracle.mlp import AdamW, forward, init_params, loss_and_gradient
from paper_2606_25569_b300 import binding

from .gpu_util import check_network_output

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DIMS = [128, 512, 512, 512, 128]


def _data(batch, seed):
    rng = np.random.default_rng(seed)
    p = init_params(DIMS, rng)
    p[-sum(DIMS[1:]):] = 0.05 * rng.standard_normal(sum(DIMS[1:]))
    X = rng.standard_normal((batch, DIMS[0]))
    Y = rng.standard_normal((batch, DIMS[-1]))
    return p, X, Y


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


# Tolerances. Both sides round the GEMM operands to bfloat16 at the same points and differ only in the
# accumulation (FP32 in the tensor cores, FP64 in the oracle). A single layer (no rounded hidden
# activation between two GEMMs) therefore agrees per element to FP32 accumulation accuracy: 1e-5 forward,
# 1e-3 for gradients (the output gradient is itself rounded to bfloat16 before the weight GEMM, and an FP32
# difference can move one of its elements across a rounding boundary). With hidden layers the FP32/FP64
# difference can move a hidden activation across a bfloat16 rounding boundary (in these networks most rows
# have an activation within 1e-6 of one), changing it by 2^-8 of itself on one side only: deep networks
# are held to 1e-3 in relative L2 and 1e-2 per element.
ONE_FWD, ONE_GRAD = 1e-5, 1e-3
DEEP_L2, DEEP_ELEM = 1e-3, 1e-2


def _check_layers(g, go, dims, tol_l2, tol_elem, what):
    """check_network_output on each weight matrix and bias vector of the flat gradient separately."""
    from oracle.mlp import unpack
    gw, gb = unpack(np.asarray(g, dtype=np.float64), dims)
    ow, ob = unpack(go, dims)
    for i, (a, b) in enumerate(zip(gw + gb, ow + ob)):
        check_network_output(a, b, tol_l2, tol_elem, "%s, %s %d" % (what, "W" if i < len(gw) else "b", i % len(gw)))


@pytest.mark.parametrize("dims", [[512, 256], [256, 1024], [128, 8192]])
def test_single_layer_matches_oracle_per_element(dims):
    # one tensor-core GEMM with its bias: forward and gradient element by element
    batch = 384
    rng = np.random.default_rng(5)
    p = init_params(dims, rng)
    p[-dims[1]:] = 0.05 * rng.standard_normal(dims[1])
    p32 = p.astype(np.float32).astype(np.float64)
    X = rng.standard_normal((batch, dims[0])).astype(np.float32).astype(np.float64)
    Y = rng.standard_normal((batch, dims[1])).astype(np.float32).astype(np.float64)
    net = binding.Mlp(dims, max_batch=batch, ncomp=2, beta=0.5)
    net.set_params(p32)
    y = torch.empty(batch, dims[1], dtype=torch.float32, device="cuda")
    net.forward(_dev(X), y, batch)
    net.sync()
    ref, _ = forward(p32, dims, X, bf16=True)
    check_network_output(y.cpu().numpy().astype(np.float64), ref, ONE_FWD, ONE_FWD, "single layer %s forward" % dims)
    loss, g = net.loss_grad(_dev(X), _dev(Y), batch)
    lo, go = loss_and_gradient(p32, dims, X, Y, beta=0.5, ncomp=2, bf16=True)
    assert abs(loss - lo) <= 1e-5 * abs(lo)
    _check_layers(g, go, dims, ONE_GRAD, ONE_GRAD, "single layer %s gradient" % dims)


@pytest.mark.parametrize("batch", [300, 512])
def test_forward_matches_oracle(batch):
    p, X, _ = _data(batch, 1)
    p32 = p.astype(np.float32).astype(np.float64)
    net = binding.Mlp(DIMS, max_batch=batch)
    net.set_params(p32)
    y = torch.empty(batch, DIMS[-1], dtype=torch.float32, device="cuda")
    net.forward(_dev(X), y, batch)
    net.sync()
    got = y.cpu().numpy().astype(np.float64)
    X32 = X.astype(np.float32).astype(np.float64)
    ref, _ = forward(p32, DIMS, X32, bf16=True)
    check_network_output(got, ref, DEEP_L2, DEEP_ELEM, "forward batch %d" % batch)


def test_gradient_matches_oracle():
    batch = 256
    p, X, Y = _data(batch, 2)
    p32 = p.astype(np.float32).astype(np.float64)
    X32, Y32 = X.astype(np.float32).astype(np.float64), Y.astype(np.float32).astype(np.float64)
    net = binding.Mlp(DIMS, max_batch=batch, ncomp=2, beta=0.5)
    net.set_params(p32)
    loss, g = net.loss_grad(_dev(X), _dev(Y), batch)
    lo, go = loss_and_gradient(p32, DIMS, X32, Y32, beta=0.5, ncomp=2, bf16=True)
    assert abs(loss - lo) <= 1e-4 * abs(lo)
    _check_layers(g, go, DIMS, DEEP_L2, DEEP_ELEM, "gradient")


def test_adamw_step_and_training_reduces_loss():
    batch = 512
    rng = np.random.default_rng(3)
    p = init_params(DIMS, rng)
    X = rng.standard_normal((batch, DIMS[0]))
    W = rng.standard_normal((DIMS[-1], DIMS[0])) / np.sqrt(DIMS[0])
    Y = np.tanh(X @ W.T)
    net = binding.Mlp(DIMS, max_batch=batch, ncomp=2, beta=0.1)
    p32 = p.astype(np.float32)
    net.set_params(p32)
    xd, yd = _dev(X), _dev(Y)
    # one step against the oracle's AdamW applied to the GPU gradient
    _, g = net.loss_grad(xd, yd, batch)
    opt = AdamW(net.nparam, lr=1e-3, weight_decay=0.01)
    expect = opt.step(p32.astype(np.float64), g.astype(np.float64))
    net.train_step(xd, yd, batch, lr=1e-3, weight_decay=0.01)
    got = net.get_params().astype(np.float64)
    assert np.max(np.abs(got - expect)) <= 2e-6
    losses = [net.train_step(xd, yd, batch, want_loss=True) for _ in range(60)]
    assert losses[-1] < 0.5 * losses[0], (losses[0], losses[-1])


def _affine(rng):
    return (0.3 * rng.standard_normal(DIMS[0]), rng.uniform(0.5, 4.0, DIMS[0]), 0.2 * rng.standard_normal(DIMS[-1]),
            rng.uniform(0.05, 2.0, DIMS[-1]))


def test_forward_and_gradient_with_affine_maps_match_oracle():
    batch = 256
    p, X, Y = _data(batch, 7)
    rng = np.random.default_rng(8)
    aff = tuple(a.astype(np.float32).astype(np.float64) for a in _affine(rng))
    p32 = p.astype(np.float32).astype(np.float64)
    X32, Y32 = X.astype(np.float32).astype(np.float64), Y.astype(np.float32).astype(np.float64)
    net = binding.Mlp(DIMS, max_batch=batch, ncomp=2, beta=0.5)
    net.set_params(p32)
    net.set_affine(*aff)
    back = net.get_affine()
    for a, b in zip(aff, back):
        assert np.array_equal(a.astype(np.float32), b)
    y = torch.empty(batch, DIMS[-1], dtype=torch.float32, device="cuda")
    net.forward(_dev(X), y, batch)
    net.sync()
    ref, _ = forward(p32, DIMS, X32, bf16=True, affine=aff)
    check_network_output(y.cpu().numpy().astype(np.float64), ref, DEEP_L2, DEEP_ELEM, "forward with maps")
    loss, g = net.loss_grad(_dev(X), _dev(Y), batch)
    lo, go = loss_and_gradient(p32, DIMS, X32, Y32, beta=0.5, ncomp=2, bf16=True, affine=aff)
    assert abs(loss - lo) <= 1e-4 * abs(lo)
    _check_layers(g, go, DIMS, DEEP_L2, DEEP_ELEM, "gradient with maps")
    # removing the maps restores the plain network
    net.set_affine()
    net.forward(_dev(X), y, batch)
    net.sync()
    ref, _ = forward(p32, DIMS, X32, bf16=True)
    check_network_output(y.cpu().numpy().astype(np.float64), ref, DEEP_L2, DEEP_ELEM, "forward without maps")


def test_fit_affine_column_statistics():
    rows = 1000
    rng = np.random.default_rng(9)
    X = (rng.standard_normal((rows, DIMS[0])) * rng.uniform(1e-3, 10.0, DIMS[0]) + rng.standard_normal(DIMS[0]))
    Y = rng.standard_normal((rows, DIMS[-1])) * rng.uniform(1e-4, 1.0, DIMS[-1])
    X[:, 3] = 2.5  # a constant column keeps scale 1
    X, Y = X.astype(np.float32), Y.astype(np.float32)
    net = binding.Mlp(DIMS, max_batch=128)
    net.fit_affine(_dev(X), _dev(Y), rows)
    ish, isc, osh, osc = net.get_affine()
    Xd, Yd = X.astype(np.float64), Y.astype(np.float64)
    sdx = Xd.std(axis=0)
    assert np.allclose(ish, Xd.mean(axis=0), rtol=1e-6, atol=1e-6)
    expect = np.where(sdx > 0, 1.0 / np.where(sdx > 0, sdx, 1.0), 1.0)
    assert np.allclose(isc, expect, rtol=1e-5)
    assert isc[3] == 1.0
    assert np.allclose(osh, Yd.mean(axis=0), rtol=1e-6, atol=1e-7)
    assert np.allclose(osc, Yd.std(axis=0), rtol=1e-5)


def test_fit_affine_relative_floor():
    rows = 500
    rng = np.random.default_rng(10)
    X = (rng.standard_normal((rows, DIMS[0])) * np.logspace(-6, 0, DIMS[0])).astype(np.float32)
    Y = (rng.standard_normal((rows, DIMS[-1])) * np.logspace(-8, 0, DIMS[-1])).astype(np.float32)
    net = binding.Mlp(DIMS, max_batch=128)
    net.fit_affine(_dev(X), _dev(Y), rows, rel_floor=1e-2)
    _, isc, _, osc = net.get_affine()
    sdx, sdy = X.astype(np.float64).std(axis=0), Y.astype(np.float64).std(axis=0)
    assert np.allclose(isc, 1.0 / np.maximum(sdx, 1e-2 * sdx.max()), rtol=1e-5)
    assert np.allclose(osc, np.maximum(sdy, 1e-2 * sdy.max()), rtol=1e-5)
