"""GPU checks of the cluster-tree multipole far field (VS_FLAG_FARFIELD_TREE / plan precision 4): against
the FP64 oracle's all-pairs sum at sampled targets, against the vesicle-by-vesicle multipole far field
(precision 2) everywhere, determinism, and a suspension stepped with it against one stepped with the
vesicle multipole far field."""
import numpy as np
import pytest

from oracle.farfield import far_field
from paper_2606_25569_b300 import binding
from paper_2606_25569_b300.workloads import farfield_box, poiseuille_dense, vesicle_outline

from .gpu_util import csr

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _eval(off, xy, f, precision, near_mask=False):
    plan = binding.FarFieldPlan(off, mu=1.0, near_mask=near_mask, precision=precision)
    u = torch.full((2 * int(off[-1]),), float("nan"), dtype=torch.float64, device="cuda")
    plan.eval(_dev(xy), _dev(f), u)
    torch.cuda.synchronize()
    out = u.cpu().numpy()
    plan.close()
    return out


def _sampled_error(got, wl_xs, wl_ys, fx, fy, off, counts, n, seed):
    rng = np.random.default_rng(seed)
    tgt = np.sort(rng.choice(int(off[-1]), n, replace=False))
    ux, uy, _ = far_field(wl_xs, wl_ys, fx, fy, 1.0, near_mask=False, targets=tgt)
    owner = np.repeat(np.arange(len(counts)), counts)
    loc = tgt - off[owner[tgt]]
    gx = got[2 * off[owner[tgt]] + loc]
    gy = got[2 * off[owner[tgt]] + counts[owner[tgt]] + loc]
    return np.sqrt(np.sum((gx - ux) ** 2 + (gy - uy) ** 2) / np.sum(ux ** 2 + uy ** 2))


def test_tree_far_field_2000x128_sampled_targets_and_against_vesicle_multipole():
    wl, fx, fy = farfield_box()
    off = wl.offsets
    xy, f = wl.flat_xy(), csr(fx, fy)
    tree = _eval(off, xy, f, 4)
    assert np.all(np.isfinite(tree))
    err = _sampled_error(tree, wl.xs, wl.ys, fx, fy, off, wl.counts, 256, 21)
    ves = _eval(off, xy, f, 2)
    d = np.linalg.norm(tree - ves) / np.linalg.norm(ves)
    print("tree far field 2000x128: against the oracle %.3e, against the vesicle multipole %.3e" % (err, d))
    assert err <= 1e-5, err
    assert d <= 1e-5, d
    again = _eval(off, xy, f, 4)
    assert np.array_equal(tree, again)  # deterministic


def test_tree_far_field_uneven_vesicles_with_near_lists():
    # 600 vesicles of 16 to 128 points, clustered so that the tree is deep on one side and some pairs are near
    rng = np.random.default_rng(8)
    xs, ys, fx, fy = [], [], [], []
    Ns = [16, 32, 64, 128, 48, 96]
    for v in range(600):
        N = Ns[v % len(Ns)]
        x, y = vesicle_outline(N, 0.7, 0.05, 1e-2, rng, rng.uniform(0, 2 * np.pi))
        if v < 400:
            cx, cy = 0.16 * (v % 20), 0.16 * (v // 20)  # a dense lattice
        else:
            cx, cy = rng.uniform(3.0, 30.0), rng.uniform(-10.0, 20.0)  # scattered far away
        xs.append(x + cx)
        ys.append(y + cy)
        fx.append(rng.standard_normal(N))
        fy.append(rng.standard_normal(N))
    counts = np.array([len(x) for x in xs])
    off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    xy, f = csr(xs, ys), csr(fx, fy)
    tree = _eval(off, xy, f, 4)
    ves = _eval(off, xy, f, 2)
    pts = _eval(off, xy, f, 0)
    assert np.all(np.isfinite(tree))
    err = _sampled_error(tree, xs, ys, fx, fy, off, counts, 300, 5)
    d = np.linalg.norm(tree - ves) / np.linalg.norm(ves)
    dp = np.linalg.norm(tree - pts) / np.linalg.norm(pts)
    print("tree far field, 600 uneven vesicles: oracle %.3e, vesicle multipole %.3e, point sums %.3e" % (err, d, dp))
    assert err <= 1e-5 and d <= 1e-5 and dp <= 1e-5, (err, d, dp)
    # with the near test: the near lists are those of the vesicle multipole far field
    tn = _eval(off, xy, f, 4, near_mask=True)
    vn = _eval(off, xy, f, 2, near_mask=True)
    assert np.linalg.norm(tn - vn) / np.linalg.norm(vn) <= 1e-5


def test_tree_suspension_poiseuille_2000x64_steps_like_the_vesicle_multipole():
    wl = poiseuille_dense(2000, 64, seed=5)
    stream = torch.cuda.current_stream()
    kw = dict(kappa=wl.kappa, mu=wl.mu, dt=wl.dt, corr_tol=0.01, flow_kind=wl.flow_kind, flow_p=wl.flow_p,
              near_field=True, stream=stream, use_graph=True)
    t = binding.Suspension(wl.flat_xy(), wl.offsets, farfield_tree=True, **kw)
    m = binding.Suspension(wl.flat_xy(), wl.offsets, farfield_multipole=True, **kw)
    t.step(5)
    m.step(5)
    t.sync()
    m.sync()
    assert t.counters()["near_pairs"] == m.counters()["near_pairs"]
    xt, xm = t.positions(), m.positions()
    err = np.linalg.norm(xt - xm) / np.linalg.norm(xm)
    ut, um = t.velocity(), m.velocity()
    du = np.linalg.norm(ut - um) / np.linalg.norm(um)
    print("tree against vesicle multipole after 5 steps: positions %.3e, velocity %.3e" % (err, du))
    t.close()
    m.close()
    # the two far fields differ by their truncation errors (velocity 1e-7 .. 1e-6 of its size); positions
    # take them through dt u, as with any FP32 far field (1e-7, the bar of the FP32 point-sum step test)
    assert err <= 1e-7 and du <= 1e-5, (err, du)


def test_tree_rejects_more_vesicles_than_it_holds():
    off = (np.arange(16385 + 1) * 8).astype(np.int64)
    with pytest.raises(Exception):
        binding.FarFieldPlan(off, mu=1.0, near_mask=False, precision=4)
