"""Pins for oracle.standardize (Sec. 3.4.1)."""
import numpy as np

from oracle.spectral import Geometry
from oracle.standardize import (centroid, destandardize_disp, destandardize_points, fourier_filter, inertia,
                                standardize, to_frame_disp)
from paper_2606_25569_b300.workloads import vesicle_outline


def _shape(N=64, seed=0):
    rng = np.random.default_rng(seed)
    return vesicle_outline(N, 0.65, 1.0, 3e-2, rng, 0.7)


def test_centroid_is_polygon_area_centroid_and_translates():
    x, y = _shape()
    # polygon centroid of a finely resampled outline (shoelace), independent of the boundary formula
    from oracle.spectral import upsample
    X, Y = upsample(x, 32), upsample(y, 32)
    cr = X * np.roll(Y, -1) - np.roll(X, -1) * Y
    A = 0.5 * cr.sum()
    ref = np.array([((X + np.roll(X, -1)) * cr).sum(), ((Y + np.roll(Y, -1)) * cr).sum()]) / (6 * A)
    c = centroid(x, y)
    assert np.max(np.abs(c - ref)) < 1e-6
    assert np.max(np.abs(centroid(x + 3.0, y - 1.0) - (c + [3.0, -1.0]))) < 1e-12


def test_ellipse_inertia_closed_form():
    a, b, N = 1.7, 0.6, 128
    t = 2 * np.pi * np.arange(N) / N
    J = inertia(a * np.cos(t) + 0.4, b * np.sin(t) - 0.2, np.array([0.4, -0.2]))
    # int y^2 dA = pi a b^3 / 4, int x^2 dA = pi a^3 b / 4
    assert abs(J[0, 0] - np.pi * a * b ** 3 / 4) < 1e-12
    assert abs(J[1, 1] - np.pi * a ** 3 * b / 4) < 1e-12
    assert abs(J[0, 1]) < 1e-12


def test_standardized_shape_invariant_to_similarity_transforms():
    x, y = _shape(seed=1)
    xo, yo, p = standardize(x, y)
    assert abs(Geometry(xo, yo).length - 1.0) < 1e-12
    assert yo[-1] < 0 <= yo[0]
    th, sc, sh = 2.1, 3.7, np.array([5.0, -2.0])
    c, s = np.cos(th), np.sin(th)
    x2, y2 = sc * (c * x - s * y) + sh[0], sc * (s * x + c * y) + sh[1]
    for k in (0, 17):  # also a cyclic relabelling of the input points
        xo2, yo2, _ = standardize(np.roll(x2, k), np.roll(y2, k))
        assert np.max(np.abs(xo2 - xo)) + np.max(np.abs(yo2 - yo)) < 1e-12


def test_round_trips():
    x, y = _shape(seed=2)
    xo, yo, p = standardize(x, y)
    xb, yb = destandardize_points(xo, yo, p)
    assert np.max(np.abs(xb - x)) + np.max(np.abs(yb - y)) < 1e-13
    rng = np.random.default_rng(0)
    dx, dy = rng.standard_normal(64), rng.standard_normal(64)
    fx, fy = to_frame_disp(dx, dy, p)
    bx, by = destandardize_disp(fx, fy, p)
    assert np.max(np.abs(bx - dx)) + np.max(np.abs(by - dy)) < 1e-13


def test_filter_keeps_low_modes_only():
    N = 64
    t = 2 * np.pi * np.arange(N) / N
    v = np.cos(3 * t) + 0.5 * np.sin(16 * t) + 0.2 * np.cos(17 * t) + 0.1 * np.cos(32 * t)
    assert np.max(np.abs(fourier_filter(v) - (np.cos(3 * t) + 0.5 * np.sin(16 * t)))) < 1e-13


def test_fourier_features_of_single_modes_closed_form():
    from oracle.standardize import fourier_features
    N, K = 32, 7
    j = np.arange(N)
    # x = 3 + 2 cos(2 pi 3 j/N) - 5 sin(2 pi 5 j/N) has a_0 = 3, a_3 = 1, b_5 = 5/2 (v = a_0 + 2(a cos - b sin))
    vx = 3.0 + 2.0 * np.cos(2 * np.pi * 3 * j / N) - 5.0 * np.sin(2 * np.pi * 5 * j / N)
    vy = np.sin(2 * np.pi * 1 * j / N)
    f = fourier_features(vx, vy, K)
    expect = np.zeros(4 * K + 2)
    expect[0], expect[3], expect[K + 5] = 3.0, 1.0, 2.5
    expect[(2 * K + 1) + K + 1] = -0.5
    assert np.max(np.abs(f - expect)) < 1e-13


def test_feature_synthesis_equals_fft_lowpass():
    from oracle.standardize import features_to_samples, fourier_features
    x, y = _shape(64, 3)
    for K in (5, 16, 31):
        sx, sy = features_to_samples(fourier_features(x, y, K), K, 64)
        assert np.max(np.abs(sx - fourier_filter(x, K))) < 1e-13
        assert np.max(np.abs(sy - fourier_filter(y, K))) < 1e-13
