"""GPU checks of the symmetric FP32 far field (k_farfield_sym: each unordered pair of points of different
vesicles evaluated once, both reactions added; the default FP32 far field) against the FP64 oracle's
all-pairs sum and against the per-target kernel.

Cases span one chunk of 16 vesicles with fewer column vesicles than warps (M = 2, 5), a partial last
chunk (M = 21, 37) and several chunks (M = 40), at N = 32, 64 and 128 (one, two and four points per lane),
and suspensions of uneven point counts (8 to 128 points: every pair of the three classes, padded
segments) with and without near pairs. Tolerance: the stated FP32 far-field bar, 1e-5 relative L2.
"""
import numpy as np
import pytest

from oracle.step import Params, Suspension as OracleSuspension
from paper_2606_25569_b300 import binding
from paper_2606_25569_b300.workloads import vesicle_outline

from .gpu_util import csr, offsets

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _grid(M, N, seed, spacing=3.2, close_pair=False):
    """M vesicles on a 7-wide grid; N an int or a list of point counts (cycled)."""
    rng = np.random.default_rng(seed)
    Ns = [N] * M if np.isscalar(N) else [N[v % len(N)] for v in range(M)]
    xs, ys = [], []
    for v in range(M):
        x, y = vesicle_outline(Ns[v], float(rng.uniform(0.6, 0.9)), 1.0, 2e-2, rng, rng.uniform(0, 2 * np.pi))
        xs.append(x + spacing * (v % 7))
        ys.append(y + spacing * (v // 7))
    if close_pair:  # vesicle 1's leftmost point moved to half a spacing (2 pi / N <= h) right of vesicle 0's rightmost
        h = 2 * np.pi / max(Ns[0], Ns[1])
        i0, i1 = int(np.argmax(xs[0])), int(np.argmin(xs[1]))
        xs[1] = xs[1] - xs[1][i1] + xs[0][i0] + 0.5 * h
        ys[1] = ys[1] - ys[1][i1] + ys[0][i0]
    return xs, ys


def _rel_l2(a, b):
    return np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2))


@pytest.mark.parametrize("M,N", [(2, 128), (5, 32), (21, 64), (37, 32), (40, 64), (18, 128)])
def test_symmetric_far_field_matches_oracle(M, N):
    xs, ys = _grid(M, N, seed=M + N)
    g = binding.Suspension(csr(xs, ys), offsets(xs), kappa=1.0, mu=1.3, dt=1e-4)
    assert g.farfield_variant()[0] == -1  # the symmetric kernel is in use
    g.step()
    got = g.velocity()  # u^n at X^0: the far field alone (no background flow, no near field)
    o = OracleSuspension(xs, ys, Params(kappa=1.0, mu=1.3, dt=1e-4))
    ref = np.concatenate([np.concatenate([ux, uy]) for ux, uy in o.interaction_velocity()])
    assert _rel_l2(got, ref) <= 1e-5
    g.close()


UNEVEN = [32, 128, 64, 48, 16, 100, 8, 96, 66, 34, 128, 20]


@pytest.mark.parametrize("M", [12, 45])
def test_symmetric_far_field_uneven_matches_oracle(M):
    xs, ys = _grid(M, UNEVEN, seed=M, spacing=3.4)
    g = binding.Suspension(csr(xs, ys), offsets(xs), kappa=1.0, mu=1.3, dt=1e-4)
    assert g.farfield_variant()[0] == -1  # the symmetric kernel is in use
    g.step()
    got = g.velocity()
    o = OracleSuspension(xs, ys, Params(kappa=1.0, mu=1.3, dt=1e-4))
    ref = np.concatenate([np.concatenate([ux, uy]) for ux, uy in o.interaction_velocity()])
    err = _rel_l2(got, ref)
    print("symmetric far field, %d vesicles of uneven N: relative L2 %.3e" % (M, err))
    assert err <= 1e-5, err
    g.close()


def test_symmetric_far_field_uneven_with_near_pairs_matches_oracle_and_per_target():
    xs, ys = _grid(30, [128, 32, 64, 48, 128, 16], seed=5, spacing=3.4, close_pair=True)
    kw = dict(kappa=1.0, mu=1.0, dt=1e-3, flow_kind=1, flow_p=(0.5, 0, 0, 0), near_field=True)
    a = binding.Suspension(csr(xs, ys), offsets(xs), **kw)
    b = binding.Suspension(csr(xs, ys), offsets(xs), farfield_per_target=True, **kw)
    assert a.farfield_variant()[0] == -1 and b.farfield_variant()[0] >= 0
    a.step()
    b.step()
    o = OracleSuspension(xs, ys, Params(**kw))
    ref = np.concatenate([np.concatenate([ux, uy]) for ux, uy in o.interaction_velocity()])
    assert a.counters()["near_pairs"] == b.counters()["near_pairs"] == len(o.near_pairs) > 0
    err, err_pt = _rel_l2(a.velocity(), ref), _rel_l2(a.velocity(), b.velocity())
    print("uneven with %d near pairs: against the oracle %.3e, against the per-target kernel %.3e"
          % (len(o.near_pairs), err, err_pt))
    assert err <= 1e-5 and err_pt <= 1e-5, (err, err_pt)
    a.close()
    b.close()


def test_symmetric_and_per_target_kernels_agree_with_near_pairs():
    xs, ys = _grid(21, 64, seed=4, close_pair=True)
    kw = dict(kappa=1.0, mu=1.0, dt=1e-3, flow_kind=1, flow_p=(0.5, 0, 0, 0), near_field=True)
    a = binding.Suspension(csr(xs, ys), offsets(xs), **kw)
    b = binding.Suspension(csr(xs, ys), offsets(xs), farfield_per_target=True, **kw)
    assert a.farfield_variant()[0] == -1 and b.farfield_variant()[0] >= 0
    for _ in range(2):
        a.step()
        b.step()
        assert _rel_l2(a.velocity(), b.velocity()) <= 1e-5
    ca, cb = a.counters(), b.counters()
    assert ca["near_pairs"] == cb["near_pairs"] > 0
    # the velocities differ by FP32 rounding (relative 1e-5 at most) and move the points by dt u a step
    dx = np.max(np.abs(a.positions() - b.positions()))
    assert dx <= 2 * 2 * kw["dt"] * 1e-5 * np.max(np.abs(b.velocity()))
    # an explicit per-target launch shape leaves the symmetric kernel
    a.farfield_variant(0)
    assert a.farfield_variant()[0] == 0
    a.step()
    b.step()
    assert _rel_l2(a.velocity(), b.velocity()) <= 1e-5
    a.close()
    b.close()


def test_symmetric_far_field_is_deterministic():
    # tiles are taken dynamically by the CTAs; every partial sum still has one fixed slot and order
    xs, ys = _grid(40, 64, seed=9, close_pair=True)
    kw = dict(kappa=1.0, mu=1.0, dt=1e-3, flow_kind=1, flow_p=(0.5, 0, 0, 0), near_field=True)
    runs = []
    for _ in range(2):
        g = binding.Suspension(csr(xs, ys), offsets(xs), **kw)
        for _ in range(3):
            g.step()
        runs.append((g.positions(), g.velocity(), g.counters()["near_pairs"]))
        g.close()
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    assert runs[0][2] == runs[1][2] > 0


@pytest.mark.parametrize("N", [128, UNEVEN])
def test_far_field_plan_symmetric_and_per_target_agree(N):
    # vs_farfield_eval: precision 0 (symmetric kernel) against 3 (per target), near mask on
    xs, ys = _grid(37, N, seed=12, close_pair=True)
    rng = np.random.default_rng(12)
    f = np.concatenate([np.concatenate([rng.standard_normal(len(x)), rng.standard_normal(len(x))]) for x in xs])
    off = offsets(xs)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    out = {}
    for prec in (0, 3):
        plan = binding.FarFieldPlan(off, mu=0.7, near_mask=True, precision=prec)
        u = torch.empty(2 * off[-1], dtype=torch.float64, device="cuda")
        plan.eval(dev(csr(xs, ys)), dev(f), u)
        out[prec] = (u.cpu().numpy(), plan.counters())
        plan.close()
    assert _rel_l2(out[0][0], out[3][0]) <= 1e-5
    assert out[0][1]["near_pairs"] == out[3][1]["near_pairs"] > 0


@pytest.mark.parametrize("precision", [0, 3])
def test_near_list_overflow_is_reported(precision):
    # ten small circles pass within 0.001 of one point of a larger vesicle: that target has ten near source
    # vesicles, more than a near list holds (8); both kernels flag the overflow (error bit 8)
    rng = np.random.default_rng(3)
    x0, y0 = vesicle_outline(32, 0.8, 1.0, 1e-2, rng, 0.0)
    xs, ys = [x0], [y0]
    th = 2 * np.pi * np.arange(32) / 32
    for v in range(10):
        phi = 2 * np.pi * v / 10
        cx, cy = x0[0] + 0.051 * np.cos(phi), y0[0] + 0.051 * np.sin(phi)
        xs.append(cx + 0.05 * np.cos(th + phi + np.pi))  # point 0 of each circle 0.001 from (x0[0], y0[0])
        ys.append(cy + 0.05 * np.sin(th + phi + np.pi))
    off = offsets(xs)
    f = np.ones(2 * off[-1])
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    plan = binding.FarFieldPlan(off, mu=1.0, near_mask=True, precision=precision)
    u = torch.empty(2 * off[-1], dtype=torch.float64, device="cuda")
    plan.eval(dev(csr(xs, ys)), dev(f), u)
    c = plan.counters()
    plan.close()
    assert c["err"] & 8


@pytest.mark.parametrize("N,slots", [(32, 4), (UNEVEN, 5)])
def test_phased_symmetric_far_field_matches_one_pass(N, slots, monkeypatch):
    # partial-sum memory bounded to `slots` chunk slots a point (VS_FFS_SLOT_BYTES below one slot per chunk):
    # the chunks are taken in groups of that many, phase by phase (each group pair's tiles, then their slots
    # reduced). The far field equals the one-pass evaluation's up to the grouping of the double-float sums,
    # with the same near pairs, and matches the oracle; the same through a far-field plan
    xs, ys = _grid(150, N, seed=21, close_pair=True)
    off = offsets(xs)
    P = int(off[-1])
    kw = dict(kappa=1.0, mu=1.0, dt=1e-3, flow_kind=1, flow_p=(0.5, 0, 0, 0), near_field=True, autotune=False)
    a = binding.Suspension(csr(xs, ys), off, **kw)
    monkeypatch.setenv("VS_FFS_SLOT_BYTES", str(slots * P * 16))
    b = binding.Suspension(csr(xs, ys), off, **kw)
    rng = np.random.default_rng(3)
    f = np.concatenate([np.concatenate([rng.standard_normal(len(x)), rng.standard_normal(len(x))]) for x in xs])
    dev = lambda v: torch.as_tensor(np.ascontiguousarray(v), dtype=torch.float64, device="cuda")
    plan_b = binding.FarFieldPlan(off, mu=0.7, near_mask=True, precision=0)
    monkeypatch.delenv("VS_FFS_SLOT_BYTES")
    plan_a = binding.FarFieldPlan(off, mu=0.7, near_mask=True, precision=0)
    assert a.farfield_variant()[0] == -1 and b.farfield_variant()[0] == -1
    a.step()
    b.step()
    o = OracleSuspension(xs, ys, Params(**{k: v for k, v in kw.items() if k != "autotune"}))
    ref = np.concatenate([np.concatenate([ux, uy]) for ux, uy in o.interaction_velocity()])
    d, e = _rel_l2(b.velocity(), a.velocity()), _rel_l2(b.velocity(), ref)
    print("phased against one pass %.3e, against the oracle %.3e" % (d, e))
    assert d <= 1e-12 and e <= 1e-5
    assert a.counters()["near_pairs"] == b.counters()["near_pairs"] == len(o.near_pairs) > 0
    ua = torch.empty(2 * P, dtype=torch.float64, device="cuda")
    ub = torch.empty_like(ua)
    plan_a.eval(dev(csr(xs, ys)), dev(f), ua)
    plan_b.eval(dev(csr(xs, ys)), dev(f), ub)
    assert _rel_l2(ub.cpu().numpy(), ua.cpu().numpy()) <= 1e-12
    assert plan_a.counters()["near_pairs"] == plan_b.counters()["near_pairs"] > 0
    for h in (a, b, plan_a, plan_b):
        h.close()


def test_fp32_rate_probes_bound_the_far_field():
    # the probes that measure the far field's FP32 denominators: paired FMA chains run near the FP32 pipe's
    # 128 lanes per clock per SM (at most ~2.1 GHz), the pair loop's instruction mix no faster than that, and the
    # symmetric far field itself (loads and lane exchanges added) no faster than its own instruction mix
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ffma2, ms0 = binding.fp32_rate(0)
    mix, ms1 = binding.fp32_rate(1)
    assert ms0 > 0 and ms1 > 0
    nominal = 128 * sms * 2.1e9 / 1e12
    assert 0.3 * nominal < ffma2 <= 1.02 * nominal, (ffma2, nominal)
    assert 0.2 * nominal < mix <= 1.02 * ffma2, (mix, ffma2)
    for bad in ((2, 16), (0, 0), (1, 1 << 21)):
        with pytest.raises(binding.VsError):
            binding.fp32_rate(*bad)
