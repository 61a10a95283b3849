"""GPU parity at the sizes of the five workloads, through the C ABI, against the FP64 oracle.

* single vesicle, 32 points, 200 steps: the whole trajectory;
* Taylor-Green batch, 64 x 128: whole steps (FP64 far field, so the FP64 bar applies to every point);
* far field alone, 2000 x 128 in the 20 x 20 box: sampled targets, FP32 (1e-5) and FP64 (1e-10);
* MLP on 128-point shapes (256 -> 512 x 3 -> 256), batch 4096: the forward pass;
* dense Poiseuille, 2000 x 64, in the launch configuration the benchmark times (mixed precision, FP32
  far field, near-field correction on, CUDA-graph replay): the velocity u^n at sampled targets against
  the oracle's brute-force far field (2e-5, see the test), and X^{n+1}, sigma^{n+1} of sampled vesicles
  against the oracle's per-vesicle step given the same u^n (1e-10, 1e-8).
"""
import numpy as np
import pytest

from oracle.farfield import far_field
from oracle.flows import background
from oracle.mlp import forward, init_params
from oracle.spectral import force
from oracle.step import Params, Suspension as OracleSuspension, advance_vesicle
from paper_2606_25569_b300 import binding
from paper_2606_25569_b300.workloads import farfield_box, poiseuille_dense, single_shear, taylor_green

from .gpu_util import csr, offsets, rel_err_per_vesicle, split

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _dev(a, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64, device="cuda")


def _compare(o, g, tol_x=1e-10, tol_s=1e-8):
    counts = [len(x) for x in o.xs]
    gx, gy = split(g.positions(), counts)
    ex = rel_err_per_vesicle(gx, gy, o.xs, o.ys)
    sg = g.tension()
    so = np.concatenate(o.sig)
    es = np.max(np.abs(sg - so)) / np.max(np.abs(so))
    assert ex <= tol_x, ex
    assert es <= tol_s, es


def _pair(wl, fp64=True):
    p = Params(kappa=wl.kappa, mu=wl.mu, dt=wl.dt, flow_kind=wl.flow_kind, flow_p=wl.flow_p, corr_tol=0.01)
    o = OracleSuspension(wl.xs, wl.ys, p)
    g = binding.Suspension(wl.flat_xy(), wl.offsets, kappa=wl.kappa, mu=wl.mu, dt=wl.dt, corr_tol=0.01,
                           flow_kind=wl.flow_kind, flow_p=wl.flow_p, farfield_fp64=fp64)
    return o, g


def test_single_vesicle_200_steps():
    wl = single_shear()
    assert wl.steps == 200
    o, g = _pair(wl)
    for _ in range(wl.steps):
        o.step()
    g.step(wl.steps)
    g.sync()
    _compare(o, g)
    g.close()


def test_taylor_green_64x128_steps():
    wl = taylor_green()
    assert (wl.M, len(wl.xs[0])) == (64, 128)
    o, g = _pair(wl, fp64=True)
    for _ in range(2):
        o.step()
        g.step()
        _compare(o, g)
    g.close()


# FP64: 1e-10, the stated FP64 bar (a sum of 256k random-sign terms loses a few digits to cancellation in
# any summation order; the same kernel meets 1e-12 on 19k sources)
# precision 0 takes the symmetric pair kernel here (N = 128), 3 the per-target kernel
@pytest.mark.parametrize("precision,tol", [(0, 1e-5), (3, 1e-5), (1, 1e-10)])
def test_farfield_2000x128_sampled_targets(precision, tol):
    wl, fx, fy = farfield_box()
    assert (wl.M, len(wl.xs[0])) == (2000, 128)
    off = wl.offsets
    plan = binding.FarFieldPlan(off, mu=1.0, near_mask=False, precision=precision)
    u = torch.empty(2 * off[-1], dtype=torch.float64, device="cuda")
    plan.eval(_dev(wl.flat_xy()), _dev(csr(fx, fy)), u)
    got = u.cpu().numpy()
    plan.close()
    rng = np.random.default_rng(11)
    tgt = np.sort(rng.choice(off[-1], 256, replace=False))
    ux, uy, _ = far_field(wl.xs, wl.ys, fx, fy, 1.0, near_mask=False, targets=tgt)
    owner = np.repeat(np.arange(wl.M), wl.counts)
    loc = tgt - off[owner[tgt]]
    gx = got[2 * off[owner[tgt]] + loc]
    gy = got[2 * off[owner[tgt]] + wl.counts[owner[tgt]] + loc]
    err = np.sqrt(np.sum((gx - ux) ** 2 + (gy - uy) ** 2) / np.sum(ux ** 2 + uy ** 2))
    print("far field 2000x128 precision %d: relative L2 error %.3e" % (precision, err))
    assert err <= tol, err


def test_mlp_forward_256x512x3_batch4096():
    dims = [256, 512, 512, 512, 256]
    batch = 4096
    rng = np.random.default_rng(4)
    p = init_params(dims, rng)
    p[-sum(dims[1:]):] = 0.05 * rng.standard_normal(sum(dims[1:]))
    p32 = p.astype(np.float32).astype(np.float64)
    X = rng.standard_normal((batch, dims[0])).astype(np.float32)
    net = binding.Mlp(dims, max_batch=batch)
    net.set_params(p32)
    y = torch.empty(batch, dims[-1], dtype=torch.float32, device="cuda")
    net.forward(_dev(X, torch.float32), y, batch)
    net.sync()
    got = y.cpu().numpy().astype(np.float64)
    ref, _ = forward(p32, dims, X.astype(np.float64), bf16=True)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= 1e-3, err


def test_poiseuille_2000x64_bench_configuration_sampled():
    wl = poiseuille_dense(2000, 64, seed=5)
    stream = torch.cuda.current_stream()
    g = binding.Suspension(wl.flat_xy(), wl.offsets, kappa=wl.kappa, mu=wl.mu, dt=wl.dt, corr_tol=0.01,
                           flow_kind=wl.flow_kind, flow_p=wl.flow_p, near_field=True, stream=stream,
                           use_graph=True)
    counts = list(wl.counts)
    off = wl.offsets
    x0s, y0s = split(g.positions(), counts)
    s0 = g.tension()
    a0l0 = g.reference()
    A0, L0 = a0l0[0], a0l0[1]
    g.step(1)
    g.sync()
    u0 = g.velocity()
    x1s, y1s = split(g.positions(), counts)
    s1 = g.tension()
    c = g.counters()
    g.close()
    assert c["err"] == 0

    # u^n at sampled targets: background flow + brute-force far field of the oracle's forces
    fx, fy = [], []
    for v in range(wl.M):
        a, b = force(x0s[v], y0s[v], s0[off[v]:off[v + 1]], wl.kappa)
        fx.append(a)
        fy.append(b)
    rng = np.random.default_rng(12)
    tgt = np.sort(rng.choice(off[-1], 256, replace=False))
    ux, uy, near = far_field(x0s, y0s, fx, fy, wl.mu, near_mask=True, targets=tgt)
    assert not near  # the lattice starts with every gap wider than the near-field threshold
    owner = np.repeat(np.arange(wl.M), wl.counts)
    loc = tgt - off[owner[tgt]]
    X, Y = np.concatenate(x0s), np.concatenate(y0s)
    bx, by = background(wl.flow_kind, wl.flow_p, X[tgt], Y[tgt])
    gx = u0[2 * off[owner[tgt]] + loc] - bx
    gy = u0[2 * off[owner[tgt]] + wl.counts[owner[tgt]] + loc] - by
    err = np.sqrt(np.sum((gx - ux) ** 2 + (gy - uy) ** 2) / np.sum(ux ** 2 + uy ** 2))
    print("poiseuille 2000x64 far-field velocity: relative L2 error %.3e" % err)
    # 2e-5 here, 1e-5 on the far-field workload above: in this dense suspension each source vesicle's 64
    # terms nearly cancel (its densities sum to zero), so the FP32 rounding of each term (5.7e-6 by an
    # FP32 emulation with FP64 sums) and of the 64-term sums leaves about 1.2e-5 of the far field
    assert err <= 2e-5, err

    # one step of sampled vesicles given the same u^n
    p = Params(kappa=wl.kappa, mu=wl.mu, dt=wl.dt, flow_kind=wl.flow_kind, flow_p=wl.flow_p, corr_tol=0.01)
    uxs, uys = split(u0, counts)
    for v in rng.choice(wl.M, 16, replace=False):
        xo, yo, so, _ = advance_vesicle(x0s[v], y0s[v], uxs[v], uys[v], A0[v], L0[v], p)
        ex = rel_err_per_vesicle([x1s[v]], [y1s[v]], [xo], [yo])
        assert ex <= 1e-10, (v, ex)
        es = np.max(np.abs(s1[off[v]:off[v + 1]] - so)) / np.max(np.abs(so))
        assert es <= 1e-8, (v, es)
