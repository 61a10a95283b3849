"""GPU checks of the batched FP32 Gauss-Jordan inverse that builds the preconditioners of the mixed-precision
solves (vs_batched_inverse32): the no-pivoting elimination, its fallback to partial pivoting, and the
zero-pivot error, against numpy's FP64 inverse."""
import numpy as np
import pytest

from paper_2606_25569_b300 import binding

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _run(A):
    batch, n, _ = A.shape
    a = torch.as_tensor(A.astype(np.float32), device="cuda").contiguous()
    out = torch.empty_like(a)
    fb = binding.batched_inverse32(a, out, n, batch)
    return out.cpu().numpy().astype(np.float64), fb


def _rel_err(got, A):
    ref = np.linalg.inv(A.astype(np.float32).astype(np.float64))
    return max(np.linalg.norm(g - r) / np.linalg.norm(r) for g, r in zip(got, ref))


@pytest.mark.parametrize("n", [7, 32, 50, 64, 100, 128])
def test_well_conditioned_batch_without_pivoting(n):
    rng = np.random.default_rng(n)
    A = np.eye(n)[None] + 0.3 * rng.standard_normal((6, n, n)) / np.sqrt(n)
    got, fb = _run(A)
    assert fb == 0
    # FP32 elimination of matrices with condition numbers of a few: ~1e-6 relative
    assert _rel_err(got, A) <= 1e-4


@pytest.mark.parametrize("n", [16, 64, 128])
def test_zero_diagonal_falls_back_to_pivoting(n):
    rng = np.random.default_rng(100 + n)
    batch = 5
    A = []
    for _ in range(batch):
        perm = np.roll(np.arange(n), 1 + rng.integers(n - 1))  # a cyclic shift: every diagonal entry 0
        P = np.eye(n)[perm]
        A.append(P @ (np.eye(n) + 0.05 * rng.standard_normal((n, n)) / np.sqrt(n)) - np.diag(np.diag(P)))
    A = np.array(A)
    for a in A:
        a[np.arange(n), np.arange(n)] = 0.0
    got, fb = _run(A)
    assert fb == batch
    assert _rel_err(got, A) <= 1e-4


def test_mixed_batch_counts_only_the_matrices_that_need_pivoting():
    rng = np.random.default_rng(7)
    n, batch = 64, 8
    A = np.eye(n)[None] + 0.2 * rng.standard_normal((batch, n, n)) / np.sqrt(n)
    A[3, :, :] = A[3][::-1]          # a row reversal: zero-ish leading pivot
    A[3, 0, 0] = 0.0
    got, fb = _run(A)
    assert fb == 1
    assert _rel_err(got, A) <= 1e-4


def test_singular_matrix_is_reported():
    n = 32
    A = np.eye(n)[None].repeat(2, axis=0)
    A[1, :, 5] = 0.0  # a zero column: no pivot exists
    with pytest.raises(binding.VsError):
        _run(A)
