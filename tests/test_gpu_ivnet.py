"""GPU parity of IVNet (Sec. 3.4.2, Fig. fig:net; vs_ivnet) against the FP64 oracle with the same bfloat16
rounding points (oracle.ivnet, bf16=True), its training, and the feature-to-point conversion.

Tolerances as for the deep MLP (tests/test_gpu_mlp.py): the FP32/FP64 accumulation difference moves some
activations across a bfloat16 rounding boundary on one side only, so outputs and gradients are held to 1e-3
in relative L2 and 1e-2 per element (relative to the element plus the RMS)."""
import numpy as np
import pytest

from oracle import ivnet as ov
from oracle.mlp import AdamW
from oracle.standardize import features_to_samples
from paper_2606_25569_b300 import binding

from .gpu_util import check_network_output

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DEEP_L2, DEEP_ELEM = 1e-3, 1e-2


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def _data(N, C, nb, batch, seed):
    rng = np.random.default_rng(seed)
    p = ov.init_params(C, nb, rng)
    # non-zero biases
    ws, bs = ov.unpack(p, C, nb)
    for b in bs:
        b[:] = 0.05 * rng.standard_normal(len(b))
    p = np.concatenate([np.concatenate([w.ravel(), b]) for w, b in zip(ws, bs)])
    X = rng.standard_normal((batch, 2 * N))
    Y = rng.standard_normal((batch, 2 * N))
    return (p.astype(np.float32).astype(np.float64), X.astype(np.float32).astype(np.float64),
            Y.astype(np.float32).astype(np.float64))


def _blocks(g, C, nb):
    ws, bs = ov.unpack(np.asarray(g, dtype=np.float64), C, nb)
    return ws + bs


# The oracle itself, with a relative 3e-8 perturbation after each convolution (FP32 accumulation), moves by
# 2.3e-4 in L2 and 5.4e-3 per element at (32, 32, 2) and by 1.9e-3 and 2.3e-2 at (64, 64, 3): the larger
# network is held to 5e-3 and 5e-2.
@pytest.mark.parametrize("N,C,nb,batch,tol", [(32, 32, 2, 200, (DEEP_L2, DEEP_ELEM)), (64, 64, 3, 130, (5e-3, 5e-2))])
def test_forward_and_gradient_match_oracle(N, C, nb, batch, tol):
    p, X, Y = _data(N, C, nb, batch, 1)
    net = binding.Ivnet(N, C, nb, max_batch=batch, beta=0.5)
    assert net.nparam == ov.param_count(C, nb)
    net.set_params(p)
    assert np.array_equal(net.get_params(), p.astype(np.float32))
    y = torch.empty(batch, 2 * N, dtype=torch.float32, device="cuda")
    net.forward(_dev(X), y, batch)
    net.sync()
    ref, _ = ov.forward(p, C, nb, X, bf16=True)
    check_network_output(y.cpu().numpy().astype(np.float64), ref, tol[0], tol[1], "IVNet forward N=%d" % N)
    loss, g = net.loss_grad(_dev(X), _dev(Y), batch)
    lo, go = ov.loss_and_gradient(p, C, nb, X, Y, beta=0.5, bf16=True)
    assert abs(loss - lo) <= 10 * tol[0] * abs(lo)
    for i, (a, b) in enumerate(zip(_blocks(g, C, nb), _blocks(go, C, nb))):
        check_network_output(a.ravel(), b.ravel(), tol[0], tol[1], "IVNet gradient block %d" % i)
    net.close()


@pytest.mark.parametrize("cin", [2, 4])
def test_affine_maps_match_oracle(cin):
    N, C, nb, batch = 32, 32, 2, 160
    rng = np.random.default_rng(2)
    p = ov.init_params(C, nb, rng, cin).astype(np.float32).astype(np.float64)
    X = rng.standard_normal((batch, cin * N)).astype(np.float32).astype(np.float64)
    Y = rng.standard_normal((batch, 2 * N)).astype(np.float32).astype(np.float64)
    aff = tuple(a.astype(np.float32).astype(np.float64) for a in (
        0.3 * rng.standard_normal(cin * N), rng.uniform(0.5, 3.0, cin * N), 0.2 * rng.standard_normal(2 * N),
        rng.uniform(0.05, 2.0, 2 * N)))
    net = binding.Ivnet(N, C, nb, max_batch=batch, beta=0.5, in_channels=cin)
    net.set_params(p)
    net.set_affine(*aff)
    y = torch.empty(batch, 2 * N, dtype=torch.float32, device="cuda")
    net.forward(_dev(X), y, batch)
    net.sync()
    ref, _ = ov.forward(p, C, nb, X, bf16=True, affine=aff, cin=cin)
    check_network_output(y.cpu().numpy().astype(np.float64), ref, DEEP_L2, DEEP_ELEM, "IVNet forward with maps")
    loss, g = net.loss_grad(_dev(X), _dev(Y), batch)
    lo, go = ov.loss_and_gradient(p, C, nb, X, Y, beta=0.5, bf16=True, affine=aff, cin=cin)
    assert abs(loss - lo) <= 1e-4 * abs(lo)
    check_network_output(np.asarray(g, np.float64), go, DEEP_L2, DEEP_ELEM, "IVNet gradient with maps")
    net.close()


def test_adamw_step_and_training_reduces_loss():
    N, C, nb, batch = 32, 32, 2, 256
    rng = np.random.default_rng(4)
    p = ov.init_params(C, nb, rng).astype(np.float32)
    X = rng.standard_normal((batch, 2 * N))
    W = rng.standard_normal((2 * N, 2 * N)) / np.sqrt(2 * N)
    Y = np.tanh(X @ W.T)
    net = binding.Ivnet(N, C, nb, max_batch=batch, beta=0.1)
    net.set_params(p)
    xd, yd = _dev(X), _dev(Y)
    _, g = net.loss_grad(xd, yd, batch)
    opt = AdamW(net.nparam, lr=1e-3, weight_decay=0.01)
    expect = opt.step(p.astype(np.float64), g.astype(np.float64))
    net.train_step(xd, yd, batch, lr=1e-3, weight_decay=0.01)
    got = net.get_params().astype(np.float64)
    assert np.max(np.abs(got - expect)) <= 2e-6
    losses = [net.train_step(xd, yd, batch, want_loss=True) for _ in range(150)]
    print("IVNet training loss %.3f -> %.3f" % (losses[0], losses[-1]))
    assert losses[-1] < 0.7 * losses[0], (losses[0], losses[-1])
    net.close()


def test_feature_points_match_oracle():
    N, K, rows = 64, 16, 37
    rng = np.random.default_rng(5)
    F = rng.standard_normal((rows, 80)).astype(np.float32)  # 4K + 2 = 66 features, padded rows of 80
    out = torch.empty(rows, 2 * N, dtype=torch.float32, device="cuda")
    binding.feature_points(_dev(F), rows, 80, N, K, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for r in range(rows):
        x, y = features_to_samples(F[r, :4 * K + 2].astype(np.float64), K, N)
        assert np.max(np.abs(got[r] - np.concatenate([x, y]))) <= 1e-5 * np.max(np.abs(np.concatenate([x, y])))
