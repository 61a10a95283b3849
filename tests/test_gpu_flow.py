"""GPU parity of the learned advection and tension (Sec. 3.2: Eqs. advectionMap, advTenMap and S_sigma)
against the FP64 oracle (oracle.learned): the exact columns the networks are trained to (vs_flow_maps),
and the hybrid step with the flow networks set (vs_set_flow_networks) given the same networks."""
import numpy as np
import pytest

from oracle.learned import exact_columns
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


@pytest.mark.parametrize("N,Kf,Kout", [(64, 6, 20), (32, 8, 15)])
def test_flow_maps_are_the_oracle_exact_columns(N, Kf, Kout):
    M, kmax = 5, 12
    xs, ys = _shapes(M, N, 3)
    kw = dict(kappa=1.3, mu=0.9, dt=1e-3)
    g = binding.Suspension(csr(xs, ys), offsets(xs), farfield_fp64=True, **kw)
    o = OracleSuspension(xs, ys, Params(**kw))  # the same redistributed shapes as the library's
    W = binding.feature_width(N, kmax)
    la, lt = binding.flow_widths(Kf, Kout)
    X = torch.zeros(M, W, dtype=torch.float32, device="cuda")
    A = torch.zeros(M, la, dtype=torch.float32, device="cuda")
    T = torch.zeros(M, lt, dtype=torch.float32, device="cuda")
    g.flow_maps(Kf, Kout, kmax, X, A, T)
    gX, gA, gT = X.cpu().numpy(), A.cpu().numpy(), T.cpu().numpy()
    F = feature_count(min(kmax, N // 2 - 1))
    worst = [0.0, 0.0]
    for v in range(M):
        xo, yo, _ = standardize(o.xs[v], o.ys[v])
        fx = fourier_features(xo, yo, min(kmax, N // 2 - 1))
        assert np.max(np.abs(gX[v, :F] - fx)) <= 1e-6 * np.max(np.abs(fx))
        adv, ten = exact_columns(o.xs[v], o.ys[v], Kf, Kout, kappa=1.3, mu=0.9)
        ea = np.max(np.abs(gA[v, :len(adv)] - adv)) / np.max(np.abs(adv))
        et = np.max(np.abs(gT[v, :len(ten)] - ten)) / np.max(np.abs(ten))
        worst = [max(worst[0], ea), max(worst[1], et)]
        assert np.all(gA[v, len(adv):] == 0) and np.all(gT[v, len(ten):] == 0)
    print("flow maps N=%d: advection columns %.3e, tension columns %.3e" % (N, worst[0], worst[1]))
    # FP32 rows of FP64-accurate maps
    assert worst[0] <= 2e-6 and worst[1] <= 2e-6, worst
    # the suspension still steps as before: the maps leave its state and operator cache alone
    o.step()
    g.step()
    counts = [len(x) for x in xs]
    gx, gy = split(g.positions(), counts)
    assert rel_err_per_vesicle(gx, gy, o.xs, o.ys) <= 1e-10


def _net(dims, rng, scale):
    p = init_params(dims, rng)
    p[:-sum(dims[1:])] *= scale
    p[-sum(dims[1:]):] = scale * 0.1 * rng.standard_normal(sum(dims[1:]))
    return p.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("exact_every", [1, 0])
def test_hybrid_flow_step_matches_oracle(exact_every):
    # one-layer networks (no rounded hidden activation, so both sides agree to FP32 accumulation accuracy):
    # the plumbing of the learned advection and tension (frames, basis, contraction, scaling) is compared
    N, M, kmax, Kf, Kout = 64, 4, 12, 6, 16
    xs, ys = _shapes(M, N, 5, eps=1e-2)
    W = binding.feature_width(N, kmax)
    la, lt = binding.flow_widths(Kf, Kout)
    rng = np.random.default_rng(6)
    p_rel = _net([W, W], rng, 1.0)
    p_adv = _net([W, la], rng, 0.5)
    p_ten = _net([W, lt], rng, 0.5)
    kw = dict(kappa=1.0, mu=1.0, dt=1e-3, flow_kind=1, flow_p=(1.0, 0.0, 0.0, 0.0))
    stream = torch.cuda.current_stream()
    nets = []
    for dims, p in (([W, W], p_rel), ([W, la], p_adv), ([W, lt], p_ten)):
        n = binding.Mlp(dims, max_batch=M, stream=stream)
        n.set_params(p)
        nets.append(n)
    scale = 2e-4
    relax_net = ([W, W], p_rel, scale, kmax)
    flow_net = (([W, la], p_adv, None), ([W, lt], p_ten, None), Kf, Kout)
    o = OracleSuspension(xs, ys, Params(relax_net=relax_net, exact_every=exact_every, flow_net=flow_net, **kw))
    g = binding.Suspension(csr(xs, ys), offsets(xs), farfield_fp64=True, stream=stream, mode=1,
                           exact_every=exact_every, use_graph=True, **kw)
    g.set_network(nets[0], scale, kmax)
    g.set_flow_networks(nets[1], nets[2], Kf, Kout)
    counts = [N] * M
    for k in range(3):
        o.step()
        g.step()
        gx, gy = split(g.positions(), counts)
        ex = rel_err_per_vesicle(gx, gy, o.xs, o.ys)
        es = sigma_error(g.tension(), o.sig)
        print("hybrid flow step %d (exact relaxation every %d): positions %.3e, tension %.3e"
              % (k + 1, exact_every, ex, es))
        assert ex <= 1e-8 and es <= 1e-5, (ex, es)
    g.close()
