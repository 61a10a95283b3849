"""GPU parity of the learned near field (Sec. 3.3, Eq. NearFieldMap) against the FP64 oracle
(oracle.learned): the exact columns the layer networks are trained to (vs_near_maps), and the hybrid step
with the near-field networks set (vs_set_near_networks) given the same networks."""
import numpy as np
import pytest

from oracle.learned import near_columns
from oracle.mlp import init_params
from oracle.standardize import feature_count, fourier_features, standardize
from oracle.step import Params, Suspension as OracleSuspension
from paper_2606_25569_b300 import binding
from paper_2606_25569_b300.workloads import vesicle_outline

from .gpu_util import csr, offsets, rel_err_per_vesicle, sigma_error, split

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _shapes(M, N, seed, spacing=3.0, eps=3e-2):
    rng = np.random.default_rng(seed)
    xs, ys = [], []
    for v in range(M):
        x, y = vesicle_outline(N, 0.65, 1.0, eps, rng, rng.uniform(0, 2 * np.pi))
        xs.append(x + spacing * (v % 4))
        ys.append(y + spacing * (v // 4))
    return xs, ys


@pytest.mark.parametrize("N,Kf,Kout", [(32, 6, 12), (64, 8, 20)])
def test_near_maps_are_the_oracle_near_columns(N, Kf, Kout):
    # the layers off the curve are FP32 sums on the upsampled curve (as in the plain near field), the one on
    # the curve the self rule: each row is held to 1e-5 of its largest entry
    M, kmax = 4, 12
    xs, ys = _shapes(M, N, 3)
    kw = dict(kappa=1.0, mu=0.7, dt=1e-3)
    g = binding.Suspension(csr(xs, ys), offsets(xs), near_field=True, farfield_fp64=True, **kw)
    o = OracleSuspension(xs, ys, Params(**kw))  # the same redistributed shapes as the library's
    W = binding.feature_width(N, kmax)
    width = binding.flow_widths(Kf, Kout)[0]
    X = torch.zeros(M, W, dtype=torch.float32, device="cuda")
    R = torch.zeros(5, M, width, dtype=torch.float32, device="cuda")
    g.near_maps(Kf, Kout, kmax, X, R)
    gX, gR = X.cpu().numpy(), R.cpu().numpy()
    F = feature_count(min(kmax, N // 2 - 1))
    worst = np.zeros(5)
    for v in range(M):
        xo, yo, _ = standardize(o.xs[v], o.ys[v])
        fx = fourier_features(xo, yo, min(kmax, N // 2 - 1))
        assert np.max(np.abs(gX[v, :F] - fx)) <= 1e-6 * np.max(np.abs(fx))
        rows = near_columns(o.xs[v], o.ys[v], Kf, Kout)
        for d in range(5):
            e = np.max(np.abs(gR[d, v, :len(rows[d])] - rows[d])) / np.max(np.abs(rows[d]))
            worst[d] = max(worst[d], e)
            assert np.all(gR[d, v, len(rows[d]):] == 0)
    print("near maps N=%d: per-layer worst relative error %s" % (N, np.array2string(worst, precision=2)))
    assert np.all(worst <= 1e-5), worst
    # the suspension still steps as before
    o.step()
    g.step()
    gx, gy = split(g.positions(), [N] * M)
    assert rel_err_per_vesicle(gx, gy, o.xs, o.ys) <= 1e-10


def _net(dims, rng, scale):
    p = init_params(dims, rng)
    p[:-sum(dims[1:])] *= scale
    p[-sum(dims[1:]):] = scale * 0.1 * rng.standard_normal(sum(dims[1:]))
    return p.astype(np.float32).astype(np.float64)


def _near_net(W, width, row, rng, scale):
    """One-layer network whose output is the given row (bias) plus a small input-dependent part: layer
    velocities as smooth as real ones, so that the FP32 RBF solve after them stays well conditioned."""
    w = scale * rng.standard_normal((width, W)) / np.sqrt(W)
    b = np.zeros(width)
    b[:len(row)] = row
    return np.concatenate([w.ravel(), b]).astype(np.float32).astype(np.float64)


def test_hybrid_step_with_learned_near_field_matches_oracle():
    # one-layer networks (both sides agree to FP32 accumulation accuracy): the plumbing of the learned near
    # field (frames, basis, contraction, scaling, the log L term) is compared, with the FP32 RBF after it. The
    # networks give the columns of one of the vesicles' shapes plus a small input-dependent part
    from .test_gpu_parity import _close_pair
    xs, ys = _close_pair()
    N, M, kmax, Kf, Kout = 32, 3, 12, 6, 12
    W = binding.feature_width(N, kmax)
    width = binding.flow_widths(Kf, Kout)[0]
    rng = np.random.default_rng(7)
    p_rel = _net([W, W], rng, 1.0)
    cols = near_columns(xs[0], ys[0], Kf, Kout)
    p_near = [_near_net(W, width, cols[d], rng, 1e-3) for d in range(5)]
    kw = dict(kappa=1.0, mu=0.9, dt=1e-3, flow_kind=1, flow_p=(0.5, 0.0, 0.0, 0.0), near_field=True)
    stream = torch.cuda.current_stream()
    rel = binding.Mlp([W, W], max_batch=M, stream=stream)
    rel.set_params(p_rel)
    nets = []
    for p in p_near:
        n = binding.Mlp([W, width], max_batch=M, stream=stream)
        n.set_params(p)
        nets.append(n)
    scale = 2e-4
    relax_net = ([W, W], p_rel, scale, kmax)
    near_net = ([([W, width], p, None) for p in p_near], Kf, Kout)
    o = OracleSuspension(xs, ys, Params(relax_net=relax_net, near_net=near_net, **kw))
    g = binding.Suspension(csr(xs, ys), offsets(xs), farfield_fp64=True, stream=stream, mode=1, use_graph=True, **kw)
    g.set_network(rel, scale, kmax)
    g.set_near_networks(nets, Kf, Kout)
    # the same suspension without the near-field networks, to see that they act
    e = binding.Suspension(csr(xs, ys), offsets(xs), farfield_fp64=True, stream=stream, mode=1, **kw)
    e.set_network(rel, scale, kmax)
    for k in range(3):
        o.step()
        g.step()
        e.step()
        assert len(o.near_pairs) > 0
        gx, gy = split(g.positions(), [N] * M)
        ex = rel_err_per_vesicle(gx, gy, o.xs, o.ys)
        es = sigma_error(g.tension(), o.sig)
        hx, hy = split(e.positions(), [N] * M)
        dn = rel_err_per_vesicle(hx, hy, o.xs, o.ys)
        print("hybrid step %d with learned near field: positions %.3e, tension %.3e (without the networks %.3e)"
              % (k + 1, ex, es, dn))
        assert ex <= 1e-8 and es <= 1e-5, (ex, es)
        assert dn >= 100 * max(ex, 1e-12)
    g.set_near_networks(None, Kf, Kout)
    g.close()
    e.close()
