"""GPU checks of the multipole far field (VS_FLAG_FARFIELD_MULTIPOLE / plan precision 2) against the FP64
oracle's all-pairs sum and against the point-sum FP32 far field."""
import numpy as np
import pytest

from oracle.farfield import far_field
from oracle.flows import background
from paper_2606_25569_b300 import binding
from paper_2606_25569_b300.workloads import farfield_box, poiseuille_dense

from .gpu_util import csr, poiseuille_oracle_state, split

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def test_multipole_far_field_2000x128_sampled_targets():
    wl, fx, fy = farfield_box()
    off = wl.offsets
    got = {}
    for prec in (0, 2):
        plan = binding.FarFieldPlan(off, mu=1.0, near_mask=False, precision=prec)
        u = torch.empty(2 * off[-1], dtype=torch.float64, device="cuda")
        plan.eval(_dev(wl.flat_xy()), _dev(csr(fx, fy)), u)
        got[prec] = u.cpu().numpy()
        plan.close()
    rng = np.random.default_rng(21)
    tgt = np.sort(rng.choice(off[-1], 256, replace=False))
    ux, uy, _ = far_field(wl.xs, wl.ys, fx, fy, 1.0, near_mask=False, targets=tgt)
    owner = np.repeat(np.arange(wl.M), wl.counts)
    loc = tgt - off[owner[tgt]]
    for prec in (0, 2):
        gx = got[prec][2 * off[owner[tgt]] + loc]
        gy = got[prec][2 * off[owner[tgt]] + wl.counts[owner[tgt]] + loc]
        err = np.sqrt(np.sum((gx - ux) ** 2 + (gy - uy) ** 2) / np.sum(ux ** 2 + uy ** 2))
        print("far field 2000x128 precision %d: relative L2 error %.3e" % (prec, err))
        assert err <= 1e-5, (prec, err)


def test_multipole_suspension_poiseuille_2000x64():
    wl = poiseuille_dense(2000, 64, seed=5)
    stream = torch.cuda.current_stream()
    kw = dict(kappa=wl.kappa, mu=wl.mu, dt=wl.dt, corr_tol=0.01, flow_kind=wl.flow_kind, flow_p=wl.flow_p,
              near_field=True, stream=stream, use_graph=True)
    g = binding.Suspension(wl.flat_xy(), wl.offsets, farfield_multipole=True, **kw)
    d = binding.Suspension(wl.flat_xy(), wl.offsets, **kw)
    off = wl.offsets
    g.step(1)
    d.step(1)
    g.sync()
    u_mp, u_pt = g.velocity(), d.velocity()
    assert g.counters()["near_pairs"] == d.counters()["near_pairs"]
    # against the oracle's all-pairs sum at sampled targets, at the oracle's own initial state (same
    # tolerance as the point-sum FP32 kernel)
    _, o, fx, fy = poiseuille_oracle_state()
    x0s, y0s = o.xs, o.ys
    rng = np.random.default_rng(22)
    tgt = np.sort(rng.choice(off[-1], 256, replace=False))
    ux, uy, near = far_field(x0s, y0s, fx, fy, wl.mu, near_mask=True, targets=tgt)
    assert not near
    owner = np.repeat(np.arange(wl.M), wl.counts)
    loc = tgt - off[owner[tgt]]
    X, Y = np.concatenate(x0s), np.concatenate(y0s)
    bx, by = background(wl.flow_kind, wl.flow_p, X[tgt], Y[tgt])
    for name, u0 in (("multipole", u_mp), ("point sums", u_pt)):
        gx = u0[2 * off[owner[tgt]] + loc] - bx
        gy = u0[2 * off[owner[tgt]] + wl.counts[owner[tgt]] + loc] - by
        err = np.sqrt(np.sum((gx - ux) ** 2 + (gy - uy) ** 2) / np.sum(ux ** 2 + uy ** 2))
        print("poiseuille 2000x64 far-field velocity, %s: relative L2 error %.3e" % (name, err))
        assert err <= 2e-5, (name, err)
    g.close()
    d.close()


def test_multipole_far_field_uneven_vesicles_and_near_lists():
    # point counts 16..128 in one box, some vesicles close (point sums and near test), most far
    from paper_2606_25569_b300.workloads import vesicle_outline
    rng = np.random.default_rng(23)
    xs, ys, fx, fy = [], [], [], []
    Ns = rng.choice([16, 32, 48, 64, 128], size=60)
    for v, N in enumerate(Ns):
        x, y = vesicle_outline(int(N), float(rng.uniform(0.6, 0.9)), 0.1, 1e-2, rng, rng.uniform(0, 2 * np.pi))
        xs.append(x + 0.25 * (v % 8) + 0.02 * rng.standard_normal())
        ys.append(y + 0.25 * (v // 8))
        fx.append(rng.standard_normal(int(N)))
        fy.append(rng.standard_normal(int(N)))
    off = np.concatenate([[0], np.cumsum(Ns)]).astype(np.int64)
    xy = np.concatenate([np.concatenate([a, b]) for a, b in zip(xs, ys)])
    f = np.concatenate([np.concatenate([a, b]) for a, b in zip(fx, fy)])
    got, counts = {}, {}
    for prec in (0, 2):
        plan = binding.FarFieldPlan(off, mu=1.0, near_mask=True, precision=prec)
        u = torch.empty(2 * off[-1], dtype=torch.float64, device="cuda")
        plan.eval(_dev(xy), _dev(f), u)
        got[prec] = u.cpu().numpy()
        counts[prec] = plan.counters()
        plan.close()
    assert counts[0] == counts[2] and counts[2]["near_pairs"] > 0 and counts[2]["err"] == 0  # same near pairs
    ux, uy, near = far_field(xs, ys, fx, fy, 1.0, near_mask=True)
    assert len(near) == counts[2]["near_pairs"]
    ref = np.concatenate([np.concatenate([ux[off[v]:off[v + 1]], uy[off[v]:off[v + 1]]]) for v in range(len(Ns))])
    err = np.linalg.norm(got[2] - ref) / np.linalg.norm(ref)
    print("uneven box, multipole: relative L2 error %.3e" % err)
    assert err <= 1e-5, err


def test_multipole_far_field_with_an_overflowing_source_list():
    # a large vesicle ringed by 220 small ones: more than 128 of them are too close to its centre for the
    # local expansion, so its target points take the fallback over all source vesicles
    from paper_2606_25569_b300.workloads import vesicle_outline
    rng = np.random.default_rng(31)
    x0, y0 = vesicle_outline(128, 0.9, 1.0, 1e-2, rng, 0.0)
    xs, ys, Ns = [x0], [y0], [128]
    for v in range(220):
        ring, ang = 1.6 + 0.25 * (v % 4), 2 * np.pi * (v // 4) / 55 + 0.3 * (v % 4)
        x, y = vesicle_outline(32, 0.8, 0.06, 1e-2, rng, rng.uniform(0, 2 * np.pi))
        xs.append(x + ring * np.cos(ang))
        ys.append(y + ring * np.sin(ang))
        Ns.append(32)
    fx = [rng.standard_normal(n) for n in Ns]
    fy = [rng.standard_normal(n) for n in Ns]
    off = np.concatenate([[0], np.cumsum(Ns)]).astype(np.int64)
    xy = np.concatenate([np.concatenate([a, b]) for a, b in zip(xs, ys)])
    f = np.concatenate([np.concatenate([a, b]) for a, b in zip(fx, fy)])
    plan = binding.FarFieldPlan(off, mu=1.0, near_mask=True, precision=2)
    u = torch.empty(2 * off[-1], dtype=torch.float64, device="cuda")
    plan.eval(_dev(xy), _dev(f), u)
    got = u.cpu().numpy()
    c = plan.counters()
    plan.close()
    ux, uy, near = far_field(xs, ys, fx, fy, 1.0, near_mask=True)
    assert c["err"] == 0 and c["near_pairs"] == len(near)
    ref = np.concatenate([np.concatenate([ux[off[v]:off[v + 1]], uy[off[v]:off[v + 1]]]) for v in range(len(Ns))])
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    err0 = np.linalg.norm(got[:256] - ref[:256]) / np.linalg.norm(ref[:256])
    print("ring, multipole: relative L2 error %.3e (large vesicle %.3e)" % (err, err0))
    assert err <= 1e-5 and err0 <= 1e-5, (err, err0)
