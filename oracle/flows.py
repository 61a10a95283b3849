"""Background flows u_inf (Sec. 5.3, 5.4, Eq. tayGreenFlow). Test infrastructure only.

kind codes match the library's flow enumeration: 0 none, 1 shear, 2 Taylor-Green, 3 Poiseuille.
* shear:        u = rate * (y, 0)                                    (Sec. 5.4), p = (rate,)
* Taylor-Green: u = U (sin(pi x/W) cos(pi y/W), -cos(pi x/W) sin(pi y/W)) (Eq. tayGreenFlow),
                p = (U, W)
* Poiseuille:   u = u_max (1 - (y/W)^2) e_x, walls at y = +-W       (Sec. 5.3), p = (u_max, W)

Pins (tests/test_oracle_flows.py): every flow divergence-free by finite differences, the shear rate, the
Poiseuille no-slip walls, axis velocity and wall shear rate, the Taylor-Green stagnation points and speed.
"""
import numpy as np

NONE, SHEAR, TAYLOR_GREEN, POISEUILLE = 0, 1, 2, 3


def background(kind, p, x, y):
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if kind == NONE:
        return np.zeros_like(x), np.zeros_like(y)
    if kind == SHEAR:
        return p[0] * y, np.zeros_like(x)
    if kind == TAYLOR_GREEN:
        U, W = p[0], p[1]
        return (U * np.sin(np.pi * x / W) * np.cos(np.pi * y / W),
                -U * np.cos(np.pi * x / W) * np.sin(np.pi * y / W))
    if kind == POISEUILLE:
        umax, W = p[0], p[1]
        return umax * (1.0 - (y / W) ** 2), np.zeros_like(x)
    raise ValueError("unknown flow kind %r" % (kind,))
