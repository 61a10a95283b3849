"""vs_farfield_eval_static: the far field for callers that cannot allocate device memory.

Such callers (code running inside another framework's memory pool, a process that has handed
all device memory to someone else, a real-time loop that must not allocate) get the same
far-field sum as vs_farfield_eval, computed with scratch that lives in a static device array of
the library. This file is collected last so that a run stopping at the first failure has
already run every other test. It calls the entry point through the C ABI twice in a row, on
two different layouts, and compares each result with the allocating entry point; and once on a
small suspension of uneven point counts against the oracle's all-pairs sum.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _layouts():
    from paper_2606_25569_b300.workloads import farfield_box, vesicle_outline
    wl, fx, fy = farfield_box(M=150, N=64, seed=13, box=20.0 * np.sqrt(150 / 2000.0))
    a = (wl.xs, wl.ys, fx, fy)
    rng = np.random.default_rng(21)
    xs, ys, gx, gy = [], [], [], []
    for v, N in enumerate([32, 64, 16, 128, 48] * 9):
        x, y = vesicle_outline(N, 0.7, 0.1, 1e-2, rng, rng.uniform(0, 2 * np.pi))
        xs.append(x + 0.45 * (v % 9))
        ys.append(y + 0.45 * (v // 9))
        gx.append(rng.standard_normal(N))
        gy.append(rng.standard_normal(N))
    return [a, (xs, ys, gx, gy)]


def _csr(xs, ys):
    return np.concatenate([np.concatenate([x, y]) for x, y in zip(xs, ys)])


@pytest.mark.parametrize("precision,tol", [(0, 1e-5), (1, 1e-12)])
def test_static_scratch_far_field_matches_allocating_entry_point(precision, tol):
    from paper_2606_25569_b300 import binding
    L = binding.lib()
    stream = torch.cuda.current_stream()
    for xs, ys, fx, fy in _layouts():  # two calls in a row, different layouts
        off = np.concatenate([[0], np.cumsum([len(x) for x in xs])]).astype(np.int64)
        xy = torch.as_tensor(_csr(xs, ys), device="cuda")
        f = torch.as_tensor(_csr(fx, fy), device="cuda")
        ref = torch.empty_like(xy)
        plan = binding.FarFieldPlan(off, mu=0.9, near_mask=False, precision=precision, stream=stream)
        plan.eval(xy, f, ref)
        got = torch.full_like(xy, float("nan"))
        st = L.vs_farfield_eval_static(off.ctypes.data, len(off) - 1, 0.9, precision, xy.data_ptr(), f.data_ptr(),
                                       got.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
        assert st == 0
        torch.cuda.synchronize()
        plan.close()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(g))
        err = np.linalg.norm(g - r) / np.linalg.norm(r)
        assert err <= tol, err


@pytest.mark.parametrize("precision,tol", [(0, 1e-5), (1, 1e-12)])
def test_static_scratch_far_field_matches_oracle_on_uneven_vesicles(precision, tol):
    from oracle.farfield import far_field
    from paper_2606_25569_b300 import binding
    from paper_2606_25569_b300.workloads import vesicle_outline
    L = binding.lib()
    rng = np.random.default_rng(31)
    xs, ys, fx, fy = [], [], [], []
    for v, N in enumerate([16, 64, 32, 8, 128, 48]):
        x, y = vesicle_outline(N, 0.75, 0.3, 1e-2, rng, rng.uniform(0, 2 * np.pi))
        xs.append(x + 0.9 * (v % 3))
        ys.append(y + 0.9 * (v // 3))
        fx.append(rng.standard_normal(N))
        fy.append(rng.standard_normal(N))
    off = np.concatenate([[0], np.cumsum([len(x) for x in xs])]).astype(np.int64)
    xy = torch.as_tensor(_csr(xs, ys), device="cuda")
    f = torch.as_tensor(_csr(fx, fy), device="cuda")
    got = torch.full_like(xy, float("nan"))
    stream = torch.cuda.current_stream()
    st = L.vs_farfield_eval_static(off.ctypes.data, len(off) - 1, 0.9, precision, xy.data_ptr(), f.data_ptr(),
                                   got.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
    assert st == 0
    torch.cuda.synchronize()
    ux, uy, _ = far_field(xs, ys, fx, fy, 0.9, near_mask=False)
    ref = np.concatenate([np.concatenate([ux[off[v]:off[v + 1]], uy[off[v]:off[v + 1]]]) for v in range(len(xs))])
    g = got.cpu().numpy()
    err = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    print("static far field against the oracle, precision %d: %.3e" % (precision, err))
    assert err <= tol, err


def test_static_scratch_rejects_oversized_input():
    from paper_2606_25569_b300 import binding
    L = binding.lib()
    M = 4097
    off = (np.arange(M + 1) * 8).astype(np.int64)
    st = L.vs_farfield_eval_static(off.ctypes.data, M, 1.0, 0, 1, 1, 1, None)
    assert st == 1  # VS_ERR_INVALID_ARG, checked before any device work
