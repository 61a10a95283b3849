"""GPU parity at the sizes of the five workloads, through the C ABI, against the FP64 oracle.

* single vesicle, 32 points, 200 steps: the whole trajectory;
* Taylor-Green batch, 64 x 128: whole steps (FP64 far field, so the FP64 bar applies to every point), and
  the whole 500-step trajectory against the oracle's, stored under tests/golden/;
* far field alone, 2000 x 128 in the 20 x 20 box: sampled targets, FP32 (1e-5) and FP64 (1e-10);
* MLP on 128-point shapes (256 -> 512 x 3 -> 256), batch 4096: the forward pass;
* dense Poiseuille, 2000 x 64, in the launch configuration the benchmark times (mixed precision, FP32
  far field, near-field correction on, CUDA-graph replay): the velocity u^n at sampled targets against
  the oracle's brute-force far field at its own initial state (1e-5); with the FP64 far field,
  X^{n+1}, sigma^{n+1} of sampled vesicles against the oracle's step of them (1e-10; sigma by
  gpu_util.SIGMA_TOL).
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

from .gpu_util import (check_network_output, csr, offsets, poiseuille_oracle_state, rel_err_per_vesicle, sigma_error,
                       sigma_tolerance, split)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _dev(a, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype or torch.float64, device="cuda")


def _compare(o, g, tol_x=1e-10, tol_s=None):
    """Positions per vesicle at tol_x; tension at tol_s (None: the FP64 tolerance of gpu_util.SIGMA_TOL)."""
    counts = [len(x) for x in o.xs]
    gx, gy = split(g.positions(), counts)
    ex = rel_err_per_vesicle(gx, gy, o.xs, o.ys)
    es = sigma_error(g.tension(), o.sig)
    print("positions %.3e, tension %.3e" % (ex, es))
    assert ex <= tol_x, ex
    assert es <= sigma_tolerance(o.sig, tol_s), es


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


def test_taylor_green_64x128_500_steps_against_oracle_trajectory():
    # the oracle's 500-step trajectory of the whole suspension, stored by tests/golden/
    # make_taylor_green_trajectory.py (every eighth vesicle at nine steps); the library runs the same 500
    # steps (FP64 far field) and is compared at each stored step, recording how the difference grows
    import os
    ref = np.load(os.path.join(os.path.dirname(__file__), "golden", "taylor_green_64x128_trajectory.npz"))
    wl = taylor_green()
    _, g = _pair(wl, fp64=True)
    counts = list(wl.counts)
    sample = [int(v) for v in ref["vesicles"]]
    done = 0
    rows = []
    for k, n in enumerate(ref["steps"]):
        g.step(int(n) - done)
        done = int(n)
        gx, gy = split(g.positions(), counts)
        sg = g.tension()
        off = wl.offsets
        ox, oy, os_ = split(ref["xy"][k], [counts[v] for v in sample]) + ([],)
        for i, v in enumerate(sample):
            os_.append(ref["sigma"][k][sum(counts[u] for u in sample[:i]):][:counts[v]])
        ex = rel_err_per_vesicle([gx[v] for v in sample], [gy[v] for v in sample], ox, oy)
        es = sigma_error(np.concatenate([sg[off[v]:off[v + 1]] for v in sample]), os_)
        rows.append((done, ex, es, g.counters()["corrections"], int(ref["corrections"][k])))
    g.close()
    for r in rows:
        print("step %4d: positions %.3e, tension %.3e, corrections %d (oracle %d)" % r)
    for done, ex, es, cg, co in rows:
        assert cg == co, (done, cg, co)
        assert ex <= 1e-10, (done, ex)
        # sigma follows the positions' difference through its sensitivity to X (gpu_util.SIGMA_PER_X)
        assert es <= sigma_tolerance([np.zeros(128)], ex=ex), (done, es)


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
    # hidden activations rounded to bfloat16 on both sides: relative L2 1e-3, 1e-2 per element (test_gpu_mlp)
    check_network_output(got, ref, 1e-3, 1e-2, "network 256-512x3-256, batch 4096")


def test_poiseuille_2000x64_bench_configuration_sampled():
    # Every expected value comes from the oracle's own state (its redistribution and initial tension of the
    # workload), never from the library's output.
    wl, o, fx, fy = poiseuille_oracle_state()
    p = o.p
    off = wl.offsets
    X, Y = np.concatenate(o.xs), np.concatenate(o.ys)
    owner = np.repeat(np.arange(wl.M), wl.counts)
    rng = np.random.default_rng(12)

    # u^n of the launch configuration the benchmark times (FP32 far field, near-field correction, CUDA
    # graph) at sampled targets: background flow + the oracle's brute-force far field, relative L2 1e-5
    stream = torch.cuda.current_stream()
    g = binding.Suspension(wl.flat_xy(), off, kappa=wl.kappa, mu=wl.mu, dt=wl.dt, corr_tol=0.01,
                           flow_kind=wl.flow_kind, flow_p=wl.flow_p, near_field=True, stream=stream,
                           use_graph=True)
    g.step(1)
    g.sync()
    u0 = g.velocity()
    c = g.counters()
    g.close()
    assert c["err"] == 0
    tgt = np.sort(rng.choice(off[-1], 256, replace=False))
    ux, uy, near = far_field(o.xs, o.ys, fx, fy, wl.mu, near_mask=True, targets=tgt)
    assert not near  # the lattice starts with every gap wider than the near-field threshold
    loc = tgt - off[owner[tgt]]
    bx, by = background(wl.flow_kind, wl.flow_p, X[tgt], Y[tgt])
    gx = u0[2 * off[owner[tgt]] + loc] - bx
    gy = u0[2 * off[owner[tgt]] + wl.counts[owner[tgt]] + loc] - by
    err = np.sqrt(np.sum((gx - ux) ** 2 + (gy - uy) ** 2) / np.sum(ux ** 2 + uy ** 2))
    print("poiseuille 2000x64 far-field velocity: relative L2 error %.3e" % err)
    assert err <= 1e-5, err

    # one whole step of sampled vesicles (the same per-vesicle kernels, far field in FP64 so that the FP64
    # bar applies): the oracle's u^n at their points, then its per-vesicle step
    g = binding.Suspension(wl.flat_xy(), off, kappa=wl.kappa, mu=wl.mu, dt=wl.dt, corr_tol=0.01,
                           flow_kind=wl.flow_kind, flow_p=wl.flow_p, near_field=True, farfield_fp64=True,
                           stream=stream, use_graph=True)
    g.step(1)
    g.sync()
    x1s, y1s = split(g.positions(), list(wl.counts))
    s1 = g.tension()
    g.close()
    sample = np.sort(rng.choice(wl.M, 16, replace=False))
    pts = np.concatenate([np.arange(off[v], off[v + 1]) for v in sample])
    ux, uy, near = far_field(o.xs, o.ys, fx, fy, wl.mu, near_mask=True, targets=pts)
    assert not near
    worst = [0.0, 0.0]
    for i, v in enumerate(sample):
        n = int(wl.counts[v])
        bx, by = background(wl.flow_kind, wl.flow_p, o.xs[v], o.ys[v])
        xo, yo, so, _ = advance_vesicle(o.xs[v], o.ys[v], ux[i * n:(i + 1) * n] + bx, uy[i * n:(i + 1) * n] + by,
                                        o.A0[v], o.L0[v], p)
        ex = rel_err_per_vesicle([x1s[v]], [y1s[v]], [xo], [yo])
        es = sigma_error(s1[off[v]:off[v + 1]], [so])
        worst = [max(worst[0], ex), max(worst[1], es)]
        assert ex <= 1e-10, (v, ex)
        assert es <= sigma_tolerance([so]), (v, es)
    print("poiseuille 2000x64 sampled vesicles after one step: positions %.3e, tension %.3e" % tuple(worst))
