"""GPU parity of the fully implicit step (mode 2; Sec. 2.2.3, Eq. time_step_sc1, preconditioned GMRES)
against the oracle's dense solve (oracle.implicit).

Tolerances. The coupled system is stiff: in the FP64 oracle itself a change of one input coordinate by
1e-16 of itself moves X^{n+1} by 1.3e-10 and sigma^{n+1} by 5e-9 of its size (tests/test_oracle_implicit.py
measures the mirror images to that level). The GPU path (GMRES to a relative residual of 1e-13, FP64 far
field, FP64 products) is held to 1e-9 in X and 1e-6 in sigma per step, and along five steps to five times
that; with the FP32 far field (relative error about 1e-5 of the interaction velocity, Sec. 4.1) to 1e-7 in
X and 1e-4 in sigma.
"""
import numpy as np
import pytest

from oracle.implicit import ImplicitSuspension
from oracle.step import Params
from paper_2606_25569_b300 import binding
from paper_2606_25569_b300.workloads import vesicle_outline

from .gpu_util import csr, offsets, rel_err_per_vesicle, split

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

KAPPA, MU = 1.0, 1.0


def _cluster(Ns, seed, spacing=2.6, R=1.0):
    rng = np.random.default_rng(seed)
    xs, ys = [], []
    for v, N in enumerate(Ns):
        x, y = vesicle_outline(N, float(rng.uniform(0.6, 0.9)), R, 2e-2, rng, rng.uniform(0, 2 * np.pi))
        xs.append(x + spacing * (v % 3) + 0.2 * rng.standard_normal())
        ys.append(y + spacing * (v // 3) + 0.2 * rng.standard_normal())
    return xs, ys


def _pair(xs, ys, dt, flow_kind, flow_p, tol=1e-13, **kw):
    p = Params(kappa=KAPPA, mu=MU, dt=dt, flow_kind=flow_kind, flow_p=flow_p, corr_tol=0.01)
    o = ImplicitSuspension(xs, ys, p)
    g = binding.Suspension(csr(xs, ys), offsets(xs), kappa=KAPPA, mu=MU, dt=dt, corr_tol=0.01, flow_kind=flow_kind,
                           flow_p=flow_p, mode=2, **kw)
    g.set_gmres(tol=tol, restart=30, max_iter=200)
    return o, g


def _errors(o, g):
    counts = [len(x) for x in o.xs]
    gx, gy = split(g.positions(), counts)
    ex = rel_err_per_vesicle(gx, gy, o.xs, o.ys)
    sg = g.tension()
    so = np.concatenate(o.sig)
    es = float(np.max(np.abs(sg - so)) / np.max(np.abs(so)))
    return ex, es


@pytest.mark.parametrize("direct", [False, True], ids=["fp32-preconditioner", "fp64-preconditioner"])
@pytest.mark.parametrize("Ns,flow", [([32] * 5, (3, (1.0, 6.0, 0, 0))), ([32, 24, 48, 32, 16, 64], (1, (1.0, 0, 0, 0)))])
def test_implicit_step_matches_oracle_fp64(Ns, flow, direct):
    # the preconditioner changes the iterations, not the solution (flexible GMRES, FP64 products)
    xs, ys = _cluster(Ns, 3)
    o, g = _pair(xs, ys, 1e-3, flow[0], flow[1], farfield_fp64=True, direct_fp64=direct)
    for k in range(5):
        o.step()
        g.step()
        ex, es = _errors(o, g)
        it, res, _ = g.gmres_stats()
        print("step %d: X %.3e sigma %.3e, GMRES %d iterations, residual %.2e" % (k + 1, ex, es, it, res))
        assert res <= 1e-13
        assert ex <= 1e-9 * (k + 1), ex
        assert es <= 1e-6 * (k + 1), es


def test_implicit_step_matches_oracle_fp32_far_field():
    xs, ys = _cluster([32] * 6, 4)
    o, g = _pair(xs, ys, 1e-3, 3, (1.0, 6.0, 0, 0), tol=1e-10)
    for k in range(3):
        o.step()
        g.step()
        ex, es = _errors(o, g)
        it, res, _ = g.gmres_stats()
        print("step %d: X %.3e sigma %.3e, GMRES %d iterations, residual %.2e" % (k + 1, ex, es, it, res))
        assert ex <= 1e-7 * (k + 1), ex
        assert es <= 1e-4 * (k + 1), es


def test_single_vesicle_converges_in_one_iteration():
    # with one vesicle the FP64 preconditioner is the exact inverse of the system
    xs, ys = _cluster([48], 5)
    o, g = _pair(xs, ys, 2e-3, 1, (1.5, 0, 0, 0), direct_fp64=True)
    o.step()
    g.step()
    it, res, tot = g.gmres_stats()
    assert it == 1 and tot == 1 and res <= 1e-13
    ex, es = _errors(o, g)
    assert ex <= 1e-9 and es <= 1e-6, (ex, es)


def test_gmres_reports_non_convergence():
    xs, ys = _cluster([32] * 4, 6, spacing=2.2)
    _, g = _pair(xs, ys, 1e-3, 3, (1.0, 6.0, 0, 0), farfield_fp64=True)
    before = g.positions()
    g.set_gmres(tol=1e-15, restart=2, max_iter=2)
    with pytest.raises(binding.VsError) as e:
        g.step()
    assert e.value.status == 4
    # the state is not advanced past the failing solve
    assert np.array_equal(g.positions(), before)
    with pytest.raises(binding.VsError):
        g.set_gmres(tol=0.0)


@pytest.mark.parametrize("yz", [False, True], ids=["layers-rbf", "ying-zorin"])
def test_implicit_step_with_near_field_matches_oracle(yz):
    # a close pair (gap about half a point spacing) and a third vesicle: U_near^{n+1} of Eq. time_step_sc1 by
    # the near-field rule (Sec. 3.3, or the Ying-Zorin evaluation of Sec. 2.2.2) in every GMRES product. The
    # GPU near field is FP32 (layer sums and the RBF solve, about 1e-5 of the correction; the Ying-Zorin sums
    # about 1e-7), so X is held to 1e-7 and sigma to 1e-4 per step.
    xs, ys = [], []
    for v, (cx, cy, th) in enumerate(((-0.36, 0.0, 1.5), (0.36, 0.05, 1.5), (0.0, 1.4, 0.2))):
        rng = np.random.default_rng(20 + v)
        x, y = vesicle_outline(32, 0.7, 0.5, 5e-2, rng, th)
        xs.append(x + cx)
        ys.append(y + cy)
    p = Params(kappa=KAPPA, mu=MU, dt=1e-3, flow_kind=1, flow_p=(1.0, 0, 0, 0), corr_tol=0.01, near_field=True,
               near_yz=yz)
    o = ImplicitSuspension(xs, ys, p)
    g = binding.Suspension(csr(xs, ys), offsets(xs), kappa=KAPPA, mu=MU, dt=1e-3, corr_tol=0.01, flow_kind=1,
                           flow_p=(1.0, 0, 0, 0), mode=2, near_field=True, farfield_fp64=True, near_yz=yz)
    g.set_gmres(tol=1e-8, restart=30, max_iter=200)
    for k in range(3):
        o.step()
        g.step()
        ex, es = _errors(o, g)
        it, res, _ = g.gmres_stats()
        print("near field, step %d: X %.3e sigma %.3e, GMRES %d iterations, residual %.2e" % (k + 1, ex, es, it, res))
        assert ex <= 1e-7 * (k + 1), ex
        assert es <= 1e-4 * (k + 1), es
