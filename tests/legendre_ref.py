"""Independent numpy restatements used by the oracle pins.

These helpers compute exact quantities of polynomials (Legendre coefficients of a
given function on a cell, derivatives of monomial sums) with numpy's own Legendre
and polynomial modules.  They share nothing with the oracle's C code.
"""
import numpy as np
from numpy.polynomial import legendre as L


def leg_coeffs_1d(fun, xa, xb, p, nquad=24):
    """Legendre coefficients c_m (m <= p) of fun on [xa, xb] (L2 projection)."""
    xi, w = L.leggauss(nquad)
    x = 0.5 * (xa + xb) + 0.5 * (xb - xa) * xi
    f = fun(x)
    out = np.zeros(p + 1)
    for m in range(p + 1):
        Pm = L.legval(xi, np.eye(p + 1)[m])
        out[m] = (2 * m + 1) / 2.0 * np.sum(w * f * Pm)
    return out


def leg_coeffs_2d(fun, xa, xb, ya, yb, p, nquad=16):
    """Tensor Legendre coefficients c[mx + (p+1) my] of fun(x, y) on a rectangle."""
    xi, w = L.leggauss(nquad)
    X = 0.5 * (xa + xb) + 0.5 * (xb - xa) * xi
    Y = 0.5 * (ya + yb) + 0.5 * (yb - ya) * xi
    F = fun(X[:, None], Y[None, :])  # [qx, qy]
    n = p + 1
    P = np.array([L.legval(xi, np.eye(n)[m]) for m in range(n)])  # [m, q]
    c = np.zeros(n * n)
    for my in range(n):
        for mx in range(n):
            c[mx + n * my] = (2 * mx + 1) * (2 * my + 1) / 4.0 * np.einsum("a,b,ab,a,b->", w, w, F, P[mx], P[my])
    return c


def project_state_1d(fun, nx, p, x0=0.0, x1=1.0):
    dx = (x1 - x0) / nx
    u = np.zeros((1, nx, p + 1))
    for i in range(nx):
        u[0, i] = leg_coeffs_1d(fun, x0 + i * dx, x0 + (i + 1) * dx, p)
    return u


def project_state_2d(fun, nx, ny, p, dom=(0.0, 1.0, 0.0, 1.0), nvar=1):
    """fun(x, y) -> scalar field, or a list of nvar fields."""
    x0, x1, y0, y1 = dom
    dx, dy = (x1 - x0) / nx, (y1 - y0) / ny
    funs = fun if isinstance(fun, (list, tuple)) else [fun]
    u = np.zeros((len(funs), nx * ny, (p + 1) ** 2))
    for v, f in enumerate(funs):
        for j in range(ny):
            for i in range(nx):
                u[v, i + nx * j] = leg_coeffs_2d(f, x0 + i * dx, x0 + (i + 1) * dx, y0 + j * dy, y0 + (j + 1) * dy, p)
    return u


class Poly2D:
    """p(x, y) = sum a[i, j] x^i y^j with exact derivatives."""

    def __init__(self, a):
        self.a = np.asarray(a, dtype=float)

    def __call__(self, x, y):
        x, y = np.broadcast_arrays(np.asarray(x, dtype=float), np.asarray(y, dtype=float))
        return np.polynomial.polynomial.polyval2d(x, y, self.a)

    def deriv(self, kx, ky):
        a = self.a
        if kx:
            a = np.polynomial.polynomial.polyder(a, kx, axis=0)
        if ky:
            a = np.polynomial.polynomial.polyder(a, ky, axis=1)
        if a.size == 0:
            a = np.zeros((1, 1))
        return Poly2D(a)

    def ic_params(self):
        """Layout of the IC_POLY initial datum: params[i + 5 j] = a[i, j]."""
        prm = np.zeros(25)
        for i in range(self.a.shape[0]):
            for j in range(self.a.shape[1]):
                prm[i + 5 * j] = self.a[i, j]
        return prm
