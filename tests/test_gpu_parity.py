"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances: FP64 parts 1e-10 relative per vesicle (the stated bar for FP64 steps); the self
matrix 1e-12 (a direct formula, no solve); FP32 compensated far field 1e-5 relative L2.
"""
import numpy as np
import pytest

from oracle.farfield import far_field
from oracle.step import Params, Suspension as OracleSuspension
from oracle.stokes import self_single_layer_matrix
from paper_2606_25569_b300 import binding
from paper_2606_25569_b300.workloads import farfield_box, single_shear, vesicle_outline

from .gpu_util import csr, offsets, rel_err_per_vesicle, sigma_error, sigma_tolerance, split

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _mixed(Ns, seed=0, spacing=3.0, R=1.0):
    rng = np.random.default_rng(seed)
    xs, ys = [], []
    for v, N in enumerate(Ns):
        x, y = vesicle_outline(N, float(rng.uniform(0.6, 0.9)), R, 2e-2, rng, rng.uniform(0, 2 * np.pi))
        xs.append(x + spacing * (v % 4))
        ys.append(y + spacing * (v // 4))
    return xs, ys


def test_self_matrices_uneven_N():
    Ns = [16, 32, 64, 128, 48, 8]
    xs, ys = _mixed(Ns, 1)
    off = offsets(xs)
    out = torch.zeros(int(sum(4 * n * n for n in Ns)), dtype=torch.float64, device="cuda")
    binding.self_matrices(_dev(csr(xs, ys)), off, 0.8, out)
    got = out.cpu().numpy()
    o = 0
    for x, y in zip(xs, ys):
        n = len(x)
        S = got[o:o + 4 * n * n].reshape(2 * n, 2 * n)
        ref = self_single_layer_matrix(x, y, 0.8)
        assert np.max(np.abs(S - ref)) <= 1e-12 * np.max(np.abs(ref)), n
        o += 4 * n * n


def _ff_case(M, N, near, seed):
    rng = np.random.default_rng(seed)
    xs, ys = _mixed([N] * M, seed, spacing=2.3)
    fx = [rng.standard_normal(N) for _ in range(M)]
    fy = [rng.standard_normal(N) for _ in range(M)]
    return xs, ys, fx, fy


@pytest.mark.parametrize("near", [False, True])
def test_farfield_fp64_matches_oracle(near):
    xs, ys, fx, fy = _ff_case(9, 32, near, 2)
    # pull one vesicle close to its neighbour so that the near mask has work
    xs[1] = xs[1] - 0.25
    off = offsets(xs)
    plan = binding.FarFieldPlan(off, mu=1.3, near_mask=near, precision=1)
    u = torch.empty(2 * off[-1], dtype=torch.float64, device="cuda")
    plan.eval(_dev(csr(xs, ys)), _dev(csr(fx, fy)), u)
    c = plan.counters()
    got = u.cpu().numpy()
    ux, uy, pairs = far_field(xs, ys, fx, fy, 1.3, near_mask=near)
    ref = csr(*_to_csr(ux, uy, xs))
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert c["near_pairs"] == len(pairs)
    if near:
        assert len(pairs) > 0


def _to_csr(ux, uy, xs):
    out, o = [], 0
    for x in xs:
        n = len(x)
        out.append(ux[o:o + n])
        out.append(uy[o:o + n])
        o += n
    return [out[0::2], out[1::2]]


def test_farfield_fp32_relative_l2():
    wl, fx, fy = farfield_box(M=300, N=64, seed=3, box=20.0 * np.sqrt(300 / 2000.0))
    off = wl.offsets
    plan = binding.FarFieldPlan(off, mu=1.0, near_mask=False, precision=0)
    u = torch.empty(2 * off[-1], dtype=torch.float64, device="cuda")
    plan.eval(_dev(wl.flat_xy()), _dev(csr(fx, fy)), u)
    got = u.cpu().numpy()
    rng = np.random.default_rng(0)
    tgt = np.sort(rng.choice(off[-1], 1024, replace=False))
    ux, uy, _ = far_field(wl.xs, wl.ys, fx, fy, 1.0, near_mask=False, targets=tgt)
    owner = np.repeat(np.arange(wl.M), wl.counts)
    loc = tgt - off[owner[tgt]]
    gx = got[2 * off[owner[tgt]] + loc]
    gy = got[2 * off[owner[tgt]] + wl.counts[owner[tgt]] + loc]
    err = np.sqrt(np.sum((gx - ux) ** 2 + (gy - uy) ** 2) / np.sum(ux ** 2 + uy ** 2))
    assert err <= 1e-5, err


def _oracle_and_gpu(xs, ys, kappa, mu, dt, flow_kind, flow_p, corr_tol, fp64=True, direct=False):
    o = OracleSuspension(xs, ys, Params(kappa=kappa, mu=mu, dt=dt, flow_kind=flow_kind, flow_p=flow_p,
                                        corr_tol=corr_tol))
    g = binding.Suspension(csr(xs, ys), offsets(xs), kappa=kappa, mu=mu, dt=dt, corr_tol=corr_tol,
                           flow_kind=flow_kind, flow_p=flow_p, farfield_fp64=fp64, direct_fp64=direct)
    return o, g


def _compare(o, g, tol_x=1e-10, tol_s=None):
    """Positions per vesicle at tol_x; tension at tol_s (None: the FP64 tolerance of gpu_util.SIGMA_TOL)."""
    counts = [len(x) for x in o.xs]
    gx, gy = split(g.positions(), counts)
    ex = rel_err_per_vesicle(gx, gy, o.xs, o.ys)
    es = sigma_error(g.tension(), o.sig)
    print("positions %.3e, tension %.3e" % (ex, es))
    assert ex <= tol_x, ex
    assert es <= sigma_tolerance(o.sig, tol_s), es
    return ex, es


def test_create_matches_oracle_init():
    wl = single_shear()
    o, g = _oracle_and_gpu(wl.xs, wl.ys, 1.0, 1.0, 1e-4, 1, (1.0, 0, 0, 0), 0.01)
    _compare(o, g, 1e-12, 1e-10)
    A0, L0 = g.reference()
    assert abs(A0[0] - o.A0[0]) <= 1e-13 * o.A0[0] and abs(L0[0] - o.L0[0]) <= 1e-13 * o.L0[0]


@pytest.mark.parametrize("direct", [False, True])
def test_single_vesicle_steps_match_oracle(direct):
    # default: FP32 factorisations refined to FP64 accuracy; direct: FP64 products and LU
    wl = single_shear()
    o, g = _oracle_and_gpu(wl.xs, wl.ys, 1.0, 1.0, 1e-4, 1, (1.0, 0, 0, 0), 0.01, direct=direct)
    for k in range(5):
        o.step()
        g.step()
        _compare(o, g)


@pytest.mark.parametrize("direct", [False, True])
def test_uneven_suspension_fp64_farfield_matches_oracle(direct):
    xs, ys = _mixed([32, 64, 32, 16], 5, spacing=2.6)
    o, g = _oracle_and_gpu(xs, ys, 1.0, 1.0, 1e-3, 2, (5.0, 8.0, 0, 0), 0.01, direct=direct)
    for k in range(3):
        o.step()
        g.step()
        _compare(o, g)
    vg = g.velocity()
    counts = [len(x) for x in xs]
    vx, vy = split(vg, counts)
    for v in range(len(xs)):
        n = counts[v]
        assert np.max(np.abs(vx[v] - o.velocity[v][:n])) <= 1e-10 * np.max(np.abs(o.velocity[v]))


def test_forced_correction_matches_oracle():
    xs, ys = _mixed([32, 32], 7, spacing=2.8)
    o, g = _oracle_and_gpu(xs, ys, 1.0, 1.0, 5e-3, 1, (2.0, 0, 0, 0), 0.0)
    for k in range(3):
        o.step()
        g.step()
        _compare(o, g)
    assert g.counters()["corrections"] == 6 and o.corrections == 6


def test_fp32_farfield_step_close_to_oracle():
    xs, ys = _mixed([32, 32, 32, 32], 9, spacing=2.6)
    o, g = _oracle_and_gpu(xs, ys, 1.0, 1.0, 1e-3, 1, (1.0, 0, 0, 0), 0.01, fp64=False)
    o.step()
    g.step()
    # FP32 velocities (relative 1e-5) enter X only through dt * u
    _compare(o, g, tol_x=1e-7, tol_s=1e-3)


def _close_pair(N=32, gap_h=0.5, seed=3):
    from oracle.spectral import Geometry
    rng = np.random.default_rng(seed)
    x0, y0 = vesicle_outline(N, 0.7, 1.0, 1e-2, rng, 0.0)
    x1, y1 = vesicle_outline(N, 0.8, 0.8, 1e-2, rng, 0.4)
    g0 = Geometry(x0, y0)
    shift = x0.max() - x1.min() + gap_h * g0.h
    x2, y2 = vesicle_outline(N, 0.75, 0.9, 1e-2, rng, 1.1)
    return [x0, x1 + shift, x2], [y0, y1 + 0.1, y2 + 2.6]


def test_near_field_step_matches_oracle():
    # FP64 far field, near-field correction on: FP32 RBF Cholesky on the GPU vs FP64 in the oracle
    xs, ys = _close_pair()
    o = OracleSuspension(xs, ys, Params(kappa=1.0, mu=1.0, dt=1e-3, flow_kind=1, flow_p=(0.5, 0, 0, 0),
                                        near_field=True))
    g = binding.Suspension(csr(xs, ys), offsets(xs), kappa=1.0, mu=1.0, dt=1e-3, flow_kind=1,
                           flow_p=(0.5, 0, 0, 0), near_field=True, farfield_fp64=True)
    for k in range(2):
        o.step()
        g.step()
        assert len(o.near_pairs) > 0
        assert g.counters()["near_pairs"] == len(o.near_pairs)
        counts = [len(x) for x in xs]
        vx, vy = split(g.velocity(), counts)
        ref = np.concatenate(o.velocity)
        got = np.concatenate([np.concatenate([a, b]) for a, b in zip(vx, vy)])
        # FP32 layer sums and FP32 RBF Cholesky: the FP32 bar of 1e-5 in relative L2, 5e-5 of the largest
        # velocity at any one point (as at 64 and 128 points)
        l2 = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        mx = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        print("near field N=32: velocity relative L2 %.3e, max %.3e" % (l2, mx))
        assert l2 <= 1e-5 and mx <= 5e-5, (l2, mx)
        _compare(o, g, tol_x=1e-8, tol_s=1e-4)


def _tips(N, gap_h=0.6, seed=4):
    """Vesicle 0 with the tips of two elongated vesicles 1 and 2 pointing at its point 0 from +-60 degrees
    (point 0 is within h of both: one target near two source vesicles), and vesicle 3 half a spacing from
    its other side."""
    from oracle.redistribute import redistribute
    from oracle.spectral import Geometry
    rng = np.random.default_rng(seed)
    x0, y0, _ = redistribute(*vesicle_outline(N, 0.7, 1.0, 1e-3, rng, 0.0))
    h0 = Geometry(x0, y0).h
    xs, ys = [x0], [y0]
    for th in (np.pi / 3, -np.pi / 3):
        x, y, _ = redistribute(*vesicle_outline(N, 0.65, 0.9, 1e-3, rng, th + np.pi))
        h = Geometry(x, y).h
        xs.append(x + x0[0] + gap_h * max(h, h0) * np.cos(th) - x[0])
        ys.append(y + y0[0] + gap_h * max(h, h0) * np.sin(th) - y[0])
    x3, y3, _ = redistribute(*vesicle_outline(N, 0.8, 0.8, 1e-3, rng, 1.3))
    y3 = y3 + 0.2
    x3 = x3 + x0.min() - x3.max()
    d = np.sqrt((x0[:, None] - x3[None, :]) ** 2 + (y0[:, None] - y3[None, :]) ** 2).min()
    x3 = x3 - (0.5 * Geometry(x3, y3).h - d) * 1.0
    xs.append(x3)
    ys.append(y3)
    return xs, ys


@pytest.mark.parametrize("N", [64, 128])
def test_near_field_at_64_and_128_points_matches_oracle(N):
    # 5N = 320 and 640 RBF systems (FP32 Cholesky on the GPU, FP64 in the oracle), four near source
    # vesicles, and a target point near two source vesicles at once
    xs, ys = _tips(N)
    kw = dict(kappa=1.0, mu=1.0, dt=1e-4, flow_kind=1, flow_p=(0.5, 0, 0, 0))
    o = OracleSuspension(xs, ys, Params(near_field=True, **kw))
    g = binding.Suspension(csr(xs, ys), offsets(xs), near_field=True, farfield_fp64=True, **kw)
    o.step()
    g.step()
    srcs = sorted(set(v for _, v in o.near_pairs))
    per_target = {}
    for t, v in o.near_pairs:
        per_target[t] = per_target.get(t, 0) + 1
    assert srcs == [0, 1, 2, 3] and max(per_target.values()) >= 2, (srcs, per_target)
    assert g.counters()["near_pairs"] == len(o.near_pairs)
    counts = [len(x) for x in xs]
    vx, vy = split(g.velocity(), counts)
    ref = np.concatenate(o.velocity)
    got = np.concatenate([np.concatenate([a, b]) for a, b in zip(vx, vy)])
    l2 = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    mx = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    print("near field N=%d: %d pairs, velocity relative L2 %.3e, max %.3e" % (N, len(o.near_pairs), l2, mx))
    # the layer sums and the RBF systems are FP32 (Cholesky, condition number about 3e4): the FP32 bar of
    # 1e-5 in relative L2, and 5e-5 of the largest velocity at any one point
    assert l2 <= 1e-5 and mx <= 5e-5, (l2, mx)
    _compare(o, g, tol_x=1e-8, tol_s=1e-4)


def test_graph_replay_matches_eager():
    # CUDA-graph replay of the step is bitwise identical to launching the kernels one by one,
    # including the near-field correction and the area/length correction paths
    xs, ys = _close_pair()
    xs.append(xs[2] + 3.0)
    ys.append(ys[2] - 1.0)
    kw = dict(kappa=1.0, mu=1.0, dt=1e-3, corr_tol=0.0, flow_kind=1, flow_p=(0.5, 0, 0, 0), near_field=True)
    stream = torch.cuda.Stream()
    a = binding.Suspension(csr(xs, ys), offsets(xs), stream=stream, use_graph=False, **kw)
    b = binding.Suspension(csr(xs, ys), offsets(xs), stream=stream, use_graph=True, **kw)
    for _ in range(5):
        a.step()
        b.step()
    assert np.array_equal(a.positions(), b.positions())
    assert np.array_equal(a.tension(), b.tension())
    ca, cb = a.counters(), b.counters()
    assert ca["corrections"] == cb["corrections"] > 0 and ca["near_pairs"] == cb["near_pairs"] > 0
    assert ca["launches"] == cb["launches"]


def test_farfield_launch_shapes_bitwise_identical():
    # every launch shape the autotuner may pick sums the same terms in the same order
    xs, ys = _mixed([64, 32, 64, 48, 64, 32, 64, 64], 9, spacing=2.4)
    g = binding.Suspension(csr(xs, ys), offsets(xs), kappa=1.0, mu=1.0, dt=1e-3, flow_kind=2,
                           flow_p=(5.0, 8.0, 0, 0), near_field=True)
    xy0, s0 = g.positions(), g.tension()
    ref = None
    k = 0
    while True:
        try:
            g.farfield_variant(k)
        except binding.VsError:
            break
        g.set_state(xy0, s0)
        g.step()
        u = g.velocity()
        if ref is None:
            ref = u
        assert np.array_equal(u, ref), k
        k += 1
    assert k >= 4
    g.close()


@pytest.mark.parametrize("Ns", [[64, 32, 64, 48, 64, 32, 64, 64], [128, 96, 128]])
def test_tensor_core_and_fma_operator_products_agree(Ns):
    # the preconditioners built on the tensor cores (three-part BF16 split, VS_FLAG_TC_GEMM) and with FP32
    # FMAs lead to the same FP64-accurate step (N = 128 also takes the 2 x 2 block inverse of A)
    xs, ys = _mixed(Ns, 10, spacing=2.6)
    kw = dict(kappa=1.0, mu=1.0, dt=1e-3, flow_kind=2, flow_p=(5.0, 8.0, 0, 0), farfield_fp64=True)
    a = binding.Suspension(csr(xs, ys), offsets(xs), **kw)
    b = binding.Suspension(csr(xs, ys), offsets(xs), tc_gemm=True, **kw)
    a.step(3)
    b.step(3)
    counts = [len(x) for x in xs]
    ax, ay = split(a.positions(), counts)
    bx, by = split(b.positions(), counts)
    assert rel_err_per_vesicle(ax, ay, bx, by) <= 1e-12
    assert np.max(np.abs(a.tension() - b.tension())) <= 1e-10 * np.max(np.abs(b.tension()))
    a.close()
    b.close()


@pytest.mark.parametrize("Ns", [[64, 62, 50, 34, 26, 18, 10, 64], [32, 32, 16, 8]])
def test_fused_operator_products_match_batched_and_oracle(Ns):
    # the FP32 preconditioners formed per vesicle in shared memory (k_fused_tl, k_fused_relax; N x N blocks
    # embedded in 64 x 64, point counts not multiples of 4 included) and by one batched GEMM launch per product
    # (VS_FLAG_OPS_BATCHED) lead to the same FP64-accurate steps, and those match the oracle
    xs, ys = _mixed(Ns, 12, spacing=2.6)
    kw = dict(kappa=1.0, mu=1.0, dt=1e-3, flow_kind=2, flow_p=(5.0, 8.0, 0, 0), corr_tol=0.01)
    o = OracleSuspension(xs, ys, Params(**kw))
    a = binding.Suspension(csr(xs, ys), offsets(xs), farfield_fp64=True, **kw)
    b = binding.Suspension(csr(xs, ys), offsets(xs), farfield_fp64=True, ops_batched=True, **kw)
    counts = [len(x) for x in xs]
    for k in range(3):
        o.step()
        a.step()
        b.step()
        _compare(o, a)
    ax, ay = split(a.positions(), counts)
    bx, by = split(b.positions(), counts)
    assert rel_err_per_vesicle(ax, ay, bx, by) <= 1e-12
    assert np.max(np.abs(a.tension() - b.tension())) <= 1e-10 * np.max(np.abs(b.tension()))
    a.close()
    b.close()


def test_set_state_keeps_operators_of_unchanged_vesicles():
    # vs_set_state only invalidates the cached operators of vesicles whose points changed; rebuilding the
    # others would give the same bits, so a suspension whose every vesicle was invalidated must agree
    xs, ys = _mixed([32, 64, 32, 48], 11, spacing=2.6)
    kw = dict(kappa=1.0, mu=1.0, dt=1e-3, corr_tol=0.01, flow_kind=1, flow_p=(0.5, 0, 0, 0), use_graph=True)
    a = binding.Suspension(csr(xs, ys), offsets(xs), **kw)
    b = binding.Suspension(csr(xs, ys), offsets(xs), **kw)
    a.step(2)
    b.step(2)
    xy, sg = a.positions(), a.tension()
    # unchanged state: stepping on from the cache equals stepping without the call
    b.set_state(xy, sg)
    a.step(1)
    b.step(1)
    assert np.array_equal(a.positions(), b.positions()) and np.array_equal(a.tension(), b.tension())
    # one vesicle moved: only its operators are rebuilt, with the same result as rebuilding all
    xy, sg = a.positions(), a.tension()
    new = xy.copy()
    o, n = 32, 64
    new[2 * o:2 * o + n] = 1.0001 * (new[2 * o:2 * o + n] - new[2 * o:2 * o + n].mean()) + new[2 * o:2 * o + n].mean()
    a.set_state(new, sg)
    b.set_state(xy + 1e-3, sg)  # every vesicle changed ...
    b.set_state(new, sg)        # ... and then set to the same state as a
    a.step(2)
    b.step(2)
    assert np.array_equal(a.positions(), b.positions()) and np.array_equal(a.tension(), b.tension())
    a.close()
    b.close()


def test_checkpoint_resume_is_bitwise():
    # a run resumed from a checkpoint continues with the same bits as the uninterrupted one
    xs, ys = _mixed([32, 64, 32, 48, 64, 32], 12, spacing=2.5)
    kw = dict(kappa=1.0, mu=1.0, dt=1e-3, corr_tol=0.0, flow_kind=1, flow_p=(0.5, 0, 0, 0), near_field=True,
              use_graph=True)
    a = binding.Suspension(csr(xs, ys), offsets(xs), **kw)
    a.step(3)
    ck = a.checkpoint()
    a.step(4)
    b = binding.Suspension(csr(xs, ys), offsets(xs), **kw)
    b.step(1)  # a different state, replaced by the restore
    b.restore(ck)
    b.step(4)
    assert np.array_equal(a.positions(), b.positions()) and np.array_equal(a.tension(), b.tension())
    ca, cb = a.counters(), b.counters()
    assert ca["steps"] == cb["steps"] == 7 and ca["corrections"] == cb["corrections"] > 0
    # a checkpoint of other point counts or parameters is refused
    c = binding.Suspension(csr(xs[:5], ys[:5]), offsets(xs[:5]), **kw)
    with pytest.raises(binding.VsError):
        c.restore(ck)
    d = binding.Suspension(csr(xs, ys), offsets(xs), **dict(kw, dt=2e-3))
    with pytest.raises(binding.VsError):
        d.restore(ck)
    with pytest.raises(binding.VsError):
        b.restore(ck[:100])
    for s in (a, b, c, d):
        s.close()


@pytest.mark.parametrize("multipole", [False, True])
def test_two_runs_are_bitwise_identical(multipole):
    # fixed-order reductions and no floating-point atomics: the same input gives the same bits
    xs, ys = _mixed([64, 32, 64, 48, 64, 32, 64, 64, 16, 128], 13, spacing=2.4)
    kw = dict(kappa=1.0, mu=1.0, dt=1e-3, corr_tol=0.0, flow_kind=1, flow_p=(0.5, 0, 0, 0), near_field=True,
              use_graph=True, farfield_multipole=multipole)
    runs = []
    for _ in range(2):
        s = binding.Suspension(csr(xs, ys), offsets(xs), **kw)
        s.step(4)
        runs.append((s.positions(), s.tension(), s.velocity(), s.counters()))
        s.close()
    (pa, ta, va, ca), (pb, tb, vb, cb) = runs
    assert np.array_equal(pa, pb) and np.array_equal(ta, tb) and np.array_equal(va, vb)
    assert ca["corrections"] == cb["corrections"] > 0 and ca["near_pairs"] == cb["near_pairs"]


def test_extreme_point_counts_step():
    # the smallest (8) and largest (128) point counts in one suspension, through the default path
    xs, ys = _mixed([8, 128, 8, 128], 14, spacing=2.6)
    o, g = _oracle_and_gpu(xs, ys, 1.0, 1.0, 1e-3, 1, (0.5, 0, 0, 0), 0.01)
    for _ in range(3):
        o.step()
        g.step()
        _compare(o, g)
    g.close()


def test_circle_makes_the_tension_system_singular_and_is_reported():
    # degenerate case of the method: on a circle a uniform tension gives a uniform normal force c n, and
    # S[c n] = 0, so the tension operator L = P S Ten annihilates constants and sigma is fixed only up to
    # one. The mixed-precision refinement notices (it cannot converge in the null direction) and the
    # suspension is refused with VS_ERR_NOT_CONVERGED instead of returning an arbitrary tension.
    N, R = 64, 0.7
    t = 2 * np.pi * np.arange(N) / N
    xs, ys = [R * np.cos(t)], [R * np.sin(t)]
    with pytest.raises(binding.VsError, match="NOT_CONVERGED"):
        binding.Suspension(csr(xs, ys), offsets(xs), kappa=1.3, mu=1.0, dt=1e-2, corr_tol=0.01, flow_kind=0)


@pytest.mark.parametrize("N", [32, 64])
def test_near_field_ying_zorin_matches_oracle(N):
    # the near field by the Ying-Zorin scheme (Sec. 2.2.2): closest point, on-curve value, FP32 sums at the
    # interpolation points (relative error about 1e-7 of the single layer there), FP64 interpolation
    from oracle.step import Suspension as OS
    xs, ys = _close_pair(N=N)
    kw = dict(kappa=1.0, mu=0.9, dt=1e-3, flow_kind=1, flow_p=(0.5, 0, 0, 0), near_field=True)
    o = OS(xs, ys, Params(near_yz=True, **kw))
    r = OS(xs, ys, Params(**kw))
    g = binding.Suspension(csr(xs, ys), offsets(xs), farfield_fp64=True, near_yz=True, **kw)
    u_o = o.interaction_velocity()
    u_r = r.interaction_velocity()
    assert o.near_pairs
    g.step()
    ug = g.velocity()
    counts = [len(x) for x in xs]
    uo = np.concatenate([np.concatenate(v) for v in u_o])
    ur = np.concatenate([np.concatenate(v) for v in u_r])
    err = np.max(np.abs(ug - uo)) / np.max(np.abs(uo))
    diff = np.max(np.abs(ur - uo)) / np.max(np.abs(uo))
    print("Ying-Zorin near field N=%d: GPU against the oracle %.2e (RBF scheme against Ying-Zorin %.2e)"
          % (N, err, diff))
    assert err <= 1e-6
    assert diff >= 100 * err
    # and the step that follows
    o.step()
    gx, gy = split(g.positions(), counts)
    assert rel_err_per_vesicle(gx, gy, o.xs, o.ys) <= 1e-9


@pytest.mark.parametrize("yz", [True, False])
def test_two_vesicles_sliding_past_each_other_in_shear(yz):
    # the two-vesicle shear interaction: vesicles on neighbouring streamlines of u = (y, 0), the upper one
    # behind and a fraction of a spacing above the lower one's top, slide past each other in near contact;
    # 30 steps with the near field (Ying-Zorin or layers + RBF) on both sides, FP64 far field. The near
    # velocities' FP32 parts (the Ying-Zorin sums, the RBF solve) set the tolerance (measured 2.7e-10 and
    # 2.8e-9)
    from oracle.spectral import Geometry
    rng = np.random.default_rng(17)
    N = 32
    x0, y0 = vesicle_outline(N, 0.7, 1.0, 1e-2, rng, 0.0)
    x1, y1 = vesicle_outline(N, 0.7, 1.0, 1e-2, rng, 0.0)
    h = Geometry(x0, y0).h
    x1 = x1 - 1.2
    y1 = y1 + (y0.max() - y1.min()) + 0.6 * h
    xs, ys = [x0, x1], [y0, y1]
    kw = dict(kappa=1.0, mu=1.0, dt=2e-3, flow_kind=1, flow_p=(1.0, 0, 0, 0), near_field=True)
    o = OracleSuspension(xs, ys, Params(near_yz=yz, **kw))
    g = binding.Suspension(csr(xs, ys), offsets(xs), farfield_fp64=True, near_yz=yz, **kw)
    near_steps, worst = 0, 0.0
    for k in range(30):
        o.step()
        g.step()
        near_steps += len(o.near_pairs) > 0
        gx, gy = split(g.positions(), [N, N])
        worst = max(worst, rel_err_per_vesicle(gx, gy, o.xs, o.ys))
    print("two vesicles in shear (%s): %d of 30 steps with near pairs, worst position difference %.2e"
          % ("Ying-Zorin" if yz else "RBF", near_steps, worst))
    assert near_steps >= 20
    assert worst <= (1e-9 if yz else 1e-8), worst
    g.close()
