"""Host pin of the vesicle multipole expansion the FP32 far field can use (VS_FLAG_FARFIELD_MULTIPOLE):
with s_j the sources relative to the vesicle centre, g_j the weighted densities and zeta = 1/q, the
Stokeslet sum over a vesicle's points at a target q far from it equals
    -A_0 log|q| + A_0/2 + T1/2 + conj(E)/2 + q conj(S_A)/2
(series in zeta from the moments A_k, B_k, D_k; the library's kernels use this form). Written out here in
numpy and checked against the oracle's direct sum: the error decays like (R/|q|)^(P+1)."""
import numpy as np

from oracle.farfield import far_field, source_weights
from paper_2606_25569_b300.workloads import vesicle_outline


def _expansion(s, g, q, P):
    A = np.array([np.sum(g * s ** k) for k in range(P + 2)])
    B = np.array([np.sum(g * np.conj(s) ** k) for k in range(P + 2)])
    D = np.array([np.sum(np.conj(g) * s * np.conj(s) ** k) for k in range(P + 2)])
    z = 1.0 / q
    T1 = sum(A[k] / k * z ** k for k in range(1, P + 1))
    SA = sum(A[k - 1] * z ** k for k in range(1, P + 2))
    E = sum(((np.conj(B[k]) / k) if k <= P else 0.0) * z ** k - np.conj(D[k - 1]) * z ** k for k in range(1, P + 2))
    return -A[0] * np.log(abs(q)) + 0.5 * A[0] + 0.5 * T1 + 0.5 * np.conj(E) + 0.5 * q * np.conj(SA)


def test_expansion_matches_direct_sum_of_a_far_vesicle():
    rng = np.random.default_rng(3)
    N, R = 64, 0.1
    xs, ys = [], []
    x, y = vesicle_outline(N, 0.65, R, 1e-2, rng, 0.4)
    xs.append(x)
    ys.append(y)
    fx, fy = [rng.standard_normal(N)], [rng.standard_normal(N)]
    # a single target vesicle point far away: the oracle's velocity there from the source vesicle
    for dist, P, tol in ((4.0, 12, 1e-7), (3.0, 12, 2e-6), (3.0, 20, 1e-9)):
        ang = rng.uniform(0, 2 * np.pi)
        tx = np.array([dist * R * 1.3 * np.cos(ang)])
        ty = np.array([dist * R * 1.3 * np.sin(ang)])
        ux, uy, _ = far_field(xs + [tx + 0 * tx], ys + [ty], fx + [np.zeros(1)], fy + [np.zeros(1)], 1.0,
                              near_mask=False, targets=[N])
        w, _ = source_weights(xs, ys)
        c = np.array([x.mean(), y.mean()])
        s = (x - c[0]) + 1j * (y - c[1])
        g = (fx[0] + 1j * fy[0]) * w[0] / (4 * np.pi)
        u = _expansion(s, g, (tx[0] - c[0]) + 1j * (ty[0] - c[1]), P)
        scale = np.sqrt(np.mean(np.abs(g) ** 2)) * N
        assert abs(u - (ux[0] + 1j * uy[0])) <= tol * scale, (dist, P, abs(u - (ux[0] + 1j * uy[0])) / scale)
