"""Redistribution of points to equal arclength (Sec. 4.2). Test infrastructure only.

Steps, in the paper's order:
1. upsample the curve by a factor of 6 (Fourier zero padding of the interpolant);
2. arclength l_m at the 6N upsampled parameters: cumulative trapezoid rule of the speed
   |X_alpha| (reading: the speed is the spectral derivative of the upsampled samples);
3. for each target arclength l~_k = k L / N, k = 0..N-1 (the paper's k/N assumes unit
   length), search the increasing sequence for the interval [l_m, l_{m+1}] holding l~_k
   (first m+1 with l_{m+1} >= l~_k) and interpolate linearly for alpha~_k;
4. reading: the new points are the trigonometric interpolant of X evaluated exactly at
   alpha~_k (the paper does not say how X is evaluated at alpha~).
Point 0 stays at alpha = 0.

Pins (tests/test_oracle_redistribute.py): a circle is a fixed point, the output is equally
spaced in arclength to within the linear-interpolation error, the curve itself is unchanged
(area/length preserved to spectral accuracy), resampling is idempotent to second order.
"""
import numpy as np

from .spectral import d_alpha, eval_interpolant, upsample

UPSAMPLE = 6


def arclength_parameters(x, y):
    """alpha~_k of the N equal-arclength targets on the curve (steps 1-3)."""
    N = len(x)
    Nu = UPSAMPLE * N
    xu, yu = upsample(x, UPSAMPLE), upsample(y, UPSAMPLE)
    sp = np.sqrt(d_alpha(xu) ** 2 + d_alpha(yu) ** 2)
    dal = 2.0 * np.pi / Nu
    l = np.concatenate([[0.0], np.cumsum(0.5 * dal * (sp + np.roll(sp, -1)))])
    total = l[-1]
    alpha_u = dal * np.arange(Nu + 1)
    out = np.zeros(N)
    for k in range(1, N):
        target = k * total / N
        m1 = int(np.searchsorted(l, target, side="left"))
        m0 = m1 - 1
        frac = (target - l[m0]) / (l[m1] - l[m0])
        out[k] = alpha_u[m0] + frac * dal
    return out


def redistribute(x, y):
    """Return (x~, y~, alpha~): the curve resampled at equal arclength (all four steps)."""
    a = arclength_parameters(x, y)
    return eval_interpolant(x, a), eval_interpolant(y, a), a
