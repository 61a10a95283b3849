"""Area and length correction (Sec. 4.3). Test infrastructure only.

The paper defines the corrected configuration as
    X~ = argmin ||X~ - X||^2  subject to  A(X~) = A_0,  L(X~) = L_0,
and approximates it with an augmented-Lagrangian loop of Adam steps whose parameters it does
not print. Reading: compute the constrained minimiser itself. Its KKT conditions are
    X~ - X - J(X~)^T lam = 0,  c(X~) = (A(X~) - A_0, L(X~) - L_0) = 0,
solved here by Newton's method with exact Hessians of the discrete
    A = (2 pi/N) sum_j 1/2 (x_j y'_j - y_j x'_j),   L = (2 pi/N) sum_j |X'_j|,   X' = D_alpha X.
D_alpha is skew-symmetric, so grad_x A = (2 pi/N) y', grad_y A = -(2 pi/N) x',
grad L = -(2 pi/N) D_alpha (X'/|X'|).
The correction runs only when |A - A_0|/A_0 or |L - L_0|/L_0 exceeds tol (Sec. 4.3: 1%).

Pins (tests/test_oracle_correct.py): a uniformly scaled circle is mapped back to the circle of
area A_0 (closed form), constraints hold to 1e-12, KKT stationarity, no-op below the trigger.
"""
import numpy as np

from .spectral import d_alpha_matrix


def area_length(x, y):
    N = len(x)
    D = d_alpha_matrix(N)
    xa, ya = D @ x, D @ y
    dal = 2.0 * np.pi / N
    return dal * np.sum(0.5 * (x * ya - y * xa)), dal * np.sum(np.sqrt(xa ** 2 + ya ** 2))


def _constraints(z, D, A0, L0):
    N = len(z) // 2
    x, y = z[:N], z[N:]
    xa, ya = D @ x, D @ y
    s = np.sqrt(xa ** 2 + ya ** 2)
    tx, ty = xa / s, ya / s
    dal = 2.0 * np.pi / N
    A = dal * np.sum(0.5 * (x * ya - y * xa))
    L = dal * np.sum(s)
    gA = dal * np.concatenate([ya, -xa])
    gL = -dal * np.concatenate([D @ tx, D @ ty])
    Z = np.zeros((N, N))
    HA = dal * np.block([[Z, D], [D.T, Z]])
    Q = np.block([[np.diag(ty * ty / s), np.diag(-tx * ty / s)],
                  [np.diag(-tx * ty / s), np.diag(tx * tx / s)]])
    DD = np.block([[D, Z], [Z, D]])
    HL = dal * DD.T @ Q @ DD
    return np.array([A - A0, L - L0]), np.vstack([gA, gL]), (HA, HL)


def needs_correction(x, y, A0, L0, tol):
    A, L = area_length(x, y)
    return abs(A - A0) / abs(A0) > tol or abs(L - L0) / abs(L0) > tol


def correct(x, y, A0, L0, tol=0.01, max_iter=50, ctol=1e-13):
    """Return (x~, y~, fired, iterations); Newton stops once the step is below 1e-15 ||X||.

    Raises RuntimeError when Newton does not converge within max_iter.
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if not needs_correction(x, y, A0, L0, tol):
        return x.copy(), y.copy(), False, 0
    N = len(x)
    D = d_alpha_matrix(N)
    z0 = np.concatenate([x, y])
    z = z0.copy()
    lam = np.zeros(2)
    znorm = np.linalg.norm(z0)
    for it in range(1, max_iter + 1):
        c, J, (HA, HL) = _constraints(z, D, A0, L0)
        r = z - z0 - J.T @ lam
        K = np.zeros((2 * N + 2, 2 * N + 2))
        K[:2 * N, :2 * N] = np.eye(2 * N) - lam[0] * HA - lam[1] * HL
        K[:2 * N, 2 * N:] = -J.T
        K[2 * N:, :2 * N] = J
        # least squares so that a circle (rank-one J: both constraints act along n) still
        # takes the minimum-norm Newton step
        d = np.linalg.lstsq(K, -np.concatenate([r, c]), rcond=None)[0]
        z = z + d[:2 * N]
        lam = lam + d[2 * N:]
        if np.linalg.norm(d[:2 * N]) <= 1e-15 * znorm:
            c, _, _ = _constraints(z, D, A0, L0)
            if abs(c[0]) <= ctol * abs(A0) * 10 and abs(c[1]) <= ctol * abs(L0) * 10:
                return z[:N], z[N:], True, it
    raise RuntimeError("area/length correction did not converge")
