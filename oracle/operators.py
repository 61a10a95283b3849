"""Per-vesicle boundary-integral operators (Eqs. totVelocity, bending_op, tension_op, PTop,
inextensib; Sec. 3.1). Test infrastructure only.

All operators are dense matrices over the stacked ordering [x_0..x_{N-1}, y_0..y_{N-1}]:
* D_s = diag(1/|X_alpha|) D_alpha, the arclength derivative (Sec. 2.2.1);
* S, the self single layer (oracle.stokes);
* B = -kappa S blockdiag(D_s^4, D_s^4), bending velocity B X (Eq. bending_op);
* Ten sigma = [D_s(sigma x_s); D_s(sigma y_s)] = (sigma X_s)_s, so T = S Ten (Eq. tension_op);
* P u = x_s D_s u_x + y_s D_s u_y, the surface divergence X_s . u_s (Eq. inextensib);
* L = P T (Eq. PTop);  M = T L^{-1} P (Sec. 3.1).

Pins (tests/test_oracle_operators.py): P(I - M) = 0, (I - M)^2 = I - M, circle force balance
sigma = -kappa/R^2 with S[c n] = 0, inextensibility of (I - M)u.
"""
import numpy as np

from .spectral import Geometry, d_alpha_matrix
from .stokes import self_single_layer_matrix


class Operators:
    def __init__(self, x, y, kappa, mu):
        g = Geometry(x, y)
        N = g.N
        self.geom = g
        self.N = N
        Da = d_alpha_matrix(N)
        Ds = Da / g.sa[:, None]
        self.Ds = Ds
        self.S = self_single_layer_matrix(x, y, mu)
        D4 = Ds @ Ds @ Ds @ Ds
        Z = np.zeros((N, N))
        self.B = -kappa * self.S @ np.block([[D4, Z], [Z, D4]])
        self.Ten = np.vstack([Ds * g.tx[None, :], Ds * g.ty[None, :]])
        self.T = self.S @ self.Ten
        self.P = np.hstack([g.tx[:, None] * Ds, g.ty[:, None] * Ds])
        self.L = self.P @ self.T

    def M(self):
        """M = T L^{-1} P (Sec. 3.1)."""
        return self.T @ np.linalg.solve(self.L, self.P)

    def project(self, u):
        """(I - M) u: the part of u compatible with inextensibility (Eq. membraneVelwoTen)."""
        s = np.linalg.solve(self.L, self.P @ u)
        return u - self.T @ s
