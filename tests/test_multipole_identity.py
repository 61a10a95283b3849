"""Host pin of the vesicle multipole expansion the FP32 far field can use (VS_FLAG_FARFIELD_MULTIPOLE):
with s_j the sources relative to the vesicle centre, g_j the weighted densities and zeta = 1/q, the
Stokeslet sum over a vesicle's points at a target q far from it equals
    -A_0 log|q| + A_0/2 + T1/2 + conj(E)/2 + q conj(S_A)/2
(series in zeta from the moments A_k, B_k, D_k; the library's kernels use this form). Written out here in
numpy and checked against the oracle's direct sum: the error decays like (R/|q|)^(P+1). The translation to
a local expansion about a far target vesicle's centre (k_ff_local, k_farfield_loc) is written out and
checked the same way, and so are the cluster tree's exact shift of raw moments from the members of a box to
its centre (k_tree_moments) and the expansion of a whole cluster."""
from math import comb
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


def _local(s, g, d, P):
    """Local expansion about the target vesicle's centre of the source vesicle's expansion, d = c_A - c_B:
    u(w) = C + H(w)/2 + conj(K(w))/2 + w conj(S(w))/2 (coefficients of w^0 .. w^P)."""
    A = np.array([np.sum(g * s ** k) for k in range(P + 2)])
    B = np.array([np.sum(g * np.conj(s) ** k) for k in range(P + 2)])
    D = np.array([np.sum(np.conj(g) * s * np.conj(s) ** k) for k in range(P + 2)])
    t = [0] + [A[k] / k if k <= P else 0 for k in range(1, P + 2)]
    sa = [0] + [A[k - 1] for k in range(1, P + 2)]
    e = [0] + [(np.conj(B[k]) / k if k <= P else 0) - np.conj(D[k - 1]) for k in range(1, P + 2)]
    z = 1.0 / d

    def loc(f):  # sum_k f_k (d + w)^-k = sum_m L_m w^m
        return np.array([(-z) ** m * sum(comb(k + m - 1, m) * f[k] * z ** k for k in range(1, P + 2))
                         for m in range(P + 1)])

    ell = np.array([0] + [(-1) ** (m + 1) * z ** m / m for m in range(1, P + 1)])  # log(1 + w/d)
    LS = loc(sa)
    H = loc(t) - A[0] * ell
    K = loc(e) + np.conj(d) * LS - np.conj(A[0]) * ell
    C = -A[0] * np.log(abs(d)) + 0.5 * A[0]
    return C, H, K, LS


def test_local_expansion_matches_direct_sum_at_a_separated_vesicle():
    rng = np.random.default_rng(5)
    N, R, P = 64, 0.1, 12
    xb, yb = vesicle_outline(N, 0.65, R, 1e-2, rng, 0.4)
    xa, ya = vesicle_outline(N, 0.65, R, 1e-2, rng, 1.9)
    fx, fy = rng.standard_normal(N), rng.standard_normal(N)
    w, _ = source_weights([xb], [yb])
    cb = np.array([xb.mean(), yb.mean()])
    s = (xb - cb[0]) + 1j * (yb - cb[1])
    g = (fx + 1j * fy) * w[0] / (4 * np.pi)
    ca = np.array([xa.mean(), ya.mean()])
    wa = (xa - ca[0]) + 1j * (ya - ca[1])
    rho = np.abs(s).max() + np.abs(wa).max()
    scale = np.sqrt(np.mean(np.abs(g) ** 2)) * N
    # centre distance 2, 3, 4 and 6 times the sum of the two radii (the kernels take 2 and more)
    for sep, tol in ((2.0, 2e-8), (3.0, 1e-9), (4.0, 1e-11), (6.0, 1e-13)):
        d = sep * rho * np.exp(0.7j)
        X, Y = xa - ca[0] + cb[0] + d.real, ya - ca[1] + cb[1] + d.imag
        ux, uy, _ = far_field([xb, X], [yb, Y], [fx, np.zeros(N)], [fy, np.zeros(N)], 1.0, near_mask=False,
                              targets=np.arange(N, 2 * N))
        C, H, K, S = _local(s, g, d, P)
        pw = wa[:, None] ** np.arange(P + 1)[None, :]
        u = C + 0.5 * (pw @ H) + 0.5 * np.conj(pw @ K) + 0.5 * wa * np.conj(pw @ S)
        assert np.max(np.abs(u - (ux + 1j * uy))) <= tol * scale, (sep, np.max(np.abs(u - (ux + 1j * uy))) / scale)


def _moments(s, g, P):
    """The expansion's series about the sources' centre: (A0, t, e, sa) with t, e, sa the coefficients of
    zeta^1 .. zeta^(P+1) of T1, E and S_A (T1 and the B part of E truncated at P, as the kernels hold them)."""
    A = np.array([np.sum(g * s ** k) for k in range(P + 2)])
    B = np.array([np.sum(g * np.conj(s) ** k) for k in range(P + 2)])
    D = np.array([np.sum(np.conj(g) * s * np.conj(s) ** k) for k in range(P + 2)])
    t = np.array([A[k] / k if k <= P else 0.0 for k in range(1, P + 2)])
    sa = np.array([A[k - 1] for k in range(1, P + 2)])
    e = np.array([(np.conj(B[k]) / k if k <= P else 0.0) - np.conj(D[k - 1]) for k in range(1, P + 2)])
    return A[0], t, e, sa


def _field(A0, t, e, sa, q):
    """-A0 log|q| + A0/2 + T1/2 + conj(E)/2 + q conj(S_A)/2 at q (zeta = 1/q)."""
    z = 1.0 / q
    zk = z ** np.arange(1, len(t) + 1)
    return -A0 * np.log(abs(q)) + 0.5 * A0 + 0.5 * (t @ zk) + 0.5 * np.conj(e @ zk) + 0.5 * q * np.conj(sa @ zk)


def _shift(A0, t, e, sa, delta):
    """The expansion about c moved to c + delta (multipole-to-multipole): with q = q' + delta, each of
    Phi = -A0 log q + T1, Psi = -conj(A0) log q + E and S_A re-expanded in 1/q' by
    b_l = alpha (-delta)^l / l + sum_{k<=l} a_k C(l-1, k-1) (-delta)^(l-k), then E' += conj(delta) S_A'
    (the term q conj(S_A) = q' conj(S_A) + conj(conj(delta) S_A))."""
    n = len(t)

    def re(a, alpha):
        return np.array([alpha * (-delta) ** l / l + sum(a[k - 1] * comb(l - 1, k - 1) * (-delta) ** (l - k)
                                                         for k in range(1, l + 1)) for l in range(1, n + 1)])
    t2, e2, s2 = re(t, A0), re(e, np.conj(A0)), re(sa, 0.0)
    return A0, t2, e2 + np.conj(delta) * s2, s2


def test_shifted_expansion_matches_direct_sum():
    # two vesicles' expansions moved to a common centre and added reproduce the direct sum of both beyond the
    # disc that holds them; the error decays like (R/|q|)^(P+2)
    rng = np.random.default_rng(7)
    N, R, P = 64, 0.1, 12
    parts, xs, ys, fxs, fys = [], [], [], [], []
    for k, (ox, oy) in enumerate(((0.0, 0.0), (0.23, -0.11))):
        x, y = vesicle_outline(N, 0.65, R, 1e-2, rng, 0.3 + k)
        xs.append(x + ox)
        ys.append(y + oy)
        fxs.append(rng.standard_normal(N))
        fys.append(rng.standard_normal(N))
    w, _ = source_weights(xs, ys)
    cc = np.array([0.15, -0.02])  # the common centre
    rho, scale = 0.0, 0.0
    tot = None
    for v in range(2):
        cv = np.array([xs[v].mean(), ys[v].mean()])
        s = (xs[v] - cv[0]) + 1j * (ys[v] - cv[1])
        g = (fxs[v] + 1j * fys[v]) * w[v] / (4 * np.pi)
        rho = max(rho, np.abs((xs[v] - cc[0]) + 1j * (ys[v] - cc[1])).max())
        scale += np.sqrt(np.mean(np.abs(g) ** 2)) * N
        ex = _shift(*_moments(s, g, P), (cc[0] - cv[0]) + 1j * (cc[1] - cv[1]))
        tot = ex if tot is None else tuple(a + b for a, b in zip(tot, ex))
    for dist, tol in ((3.0, 1e-6), (6.0, 1e-10)):
        ang = rng.uniform(0, 2 * np.pi)
        q = dist * rho * np.exp(1j * ang)
        tx, ty = np.array([cc[0] + q.real]), np.array([cc[1] + q.imag])
        ux, uy, _ = far_field(xs + [tx], ys + [ty], fxs + [np.zeros(1)], fys + [np.zeros(1)], 1.0,
                              near_mask=False, targets=[2 * N])
        u = _field(*tot, q)
        err = abs(u - (ux[0] + 1j * uy[0])) / scale
        assert err <= tol, (dist, err)
    # and the shift by zero changes nothing; two shifts compose
    A0, t, e, sa = _moments(s, g, P)
    for a, b in zip(_shift(A0, t, e, sa, 0.0), (A0, t, e, sa)):
        assert np.allclose(a, b, rtol=0, atol=1e-15 * scale)
    d1, d2 = 0.03 - 0.02j, -0.05 + 0.04j
    one = _shift(*_shift(A0, t, e, sa, d1), d2)
    both = _shift(A0, t, e, sa, d1 + d2)
    for a, b in zip(one, both):
        assert np.allclose(a, b, rtol=0, atol=1e-12 * scale)


def _raw_moments(s, g, K):
    A = np.array([np.sum(g * s ** k) for k in range(K)])
    B = np.array([np.sum(g * np.conj(s) ** k) for k in range(K)])
    D = np.array([np.sum(np.conj(g) * s * np.conj(s) ** k) for k in range(K)])
    return A, B, D


def _shift_raw(A, B, D, delta):
    """Moments about a new centre from those about the old one, delta = old centre - new centre."""
    K = len(A)
    A2, B2, D2 = (np.zeros(K, complex) for _ in range(3))
    for k in range(K):
        for j in range(k + 1):
            c = comb(k, j)
            A2[k] += c * delta ** (k - j) * A[j]
            B2[k] += c * np.conj(delta) ** (k - j) * B[j]
            D2[k] += c * np.conj(delta) ** (k - j) * (D[j] + delta * np.conj(A[j]))
    return A2, B2, D2


def test_cluster_moments_follow_exactly_from_the_members():
    # the cluster tree's multipole-to-multipole shift: moments of three vesicles about their own centres,
    # shifted to the cluster centre and added, equal the moments of all their points about that centre
    rng = np.random.default_rng(12)
    K = 14
    pts, gs, tot = [], [], [np.zeros(K, complex) for _ in range(3)]
    centres = [0.3 + 0.1j, -0.2 + 0.25j, 0.05 - 0.3j]
    cc = np.mean(centres)
    for c in centres:
        x, y = vesicle_outline(64, 0.7, 0.1, 1e-2, rng, rng.uniform(0, 2 * np.pi))
        s = (x - x.mean()) + 1j * (y - y.mean())
        g = rng.standard_normal(64) + 1j * rng.standard_normal(64)
        pts.append(s + c)
        gs.append(g)
        for t, m in zip(tot, _shift_raw(*_raw_moments(s, g, K), c - cc)):
            t += m
    direct = _raw_moments(np.concatenate(pts) - cc, np.concatenate(gs), K)
    for t, d in zip(tot, direct):
        assert np.max(np.abs(t - d) / (np.abs(d) + 1e-300)) <= 1e-11


def test_cluster_expansion_matches_direct_sum_beyond_twice_its_radius():
    # the expansion of a whole cluster (three vesicles) about its centre, from the shifted moments, against
    # the oracle's direct sum at a target beyond twice the cluster's radius
    rng = np.random.default_rng(4)
    xs, ys, fx, fy = [], [], [], []
    for c in (0.0 + 0.0j, 0.35 + 0.1j, 0.1 + 0.4j):
        x, y = vesicle_outline(64, 0.7, 0.1, 1e-2, rng, rng.uniform(0, 2 * np.pi))
        xs.append(x - x.mean() + c.real)
        ys.append(y - y.mean() + c.imag)
        fx.append(rng.standard_normal(64))
        fy.append(rng.standard_normal(64))
    w, _ = source_weights(xs, ys)
    cen = [complex(x.mean(), y.mean()) for x, y in zip(xs, ys)]
    cc = np.mean(cen)
    K, P = 14, 12
    tot = [np.zeros(K, complex) for _ in range(3)]
    for v in range(3):
        s = (xs[v] + 1j * ys[v]) - cen[v]
        g = (fx[v] + 1j * fy[v]) * w[v] / (4 * np.pi)
        for t, m in zip(tot, _shift_raw(*_raw_moments(s, g, K), cen[v] - cc)):
            t += m
    allp = np.concatenate([x + 1j * y for x, y in zip(xs, ys)])
    radius = np.max(np.abs(allp - cc))
    q = 2.2 * radius * np.exp(1j * 0.7)
    ux, uy, _ = far_field(xs + [np.array([cc.real + q.real])], ys + [np.array([cc.imag + q.imag])],
                          fx + [np.zeros(1)], fy + [np.zeros(1)], 1.0, near_mask=False, targets=[3 * 64])
    # the expansion from the cluster moments (same series as _expansion, moments given)
    A, B, D = tot
    z = 1.0 / q
    T1 = sum(A[k] / k * z ** k for k in range(1, P + 1))
    SA = sum(A[k - 1] * z ** k for k in range(1, P + 2))
    E = sum(((np.conj(B[k]) / k) if k <= P else 0.0) * z ** k - np.conj(D[k - 1]) * z ** k for k in range(1, P + 2))
    u = -A[0] * np.log(abs(q)) + 0.5 * A[0] + 0.5 * T1 + 0.5 * np.conj(E) + 0.5 * q * np.conj(SA)
    scale = np.sqrt(np.mean(np.abs(np.concatenate([(a + 1j * b) * wv for a, b, wv in zip(fx, fy, w)])) ** 2)) \
        * 3 * 64 / (4 * np.pi)
    assert abs(u - (ux[0] + 1j * uy[0])) <= 1e-3 * scale, abs(u - (ux[0] + 1j * uy[0])) / scale
