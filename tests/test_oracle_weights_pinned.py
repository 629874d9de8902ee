"""Hand-derived values of the sensor's nonlinear weights (Sec. 3.2, Sec. 2.2).

Polynomial reproduction makes every candidate equal, so it passes whatever the
weights are.  These cases fix the weights themselves: piecewise-linear (1D P1) and
piecewise-bilinear (2D Q1) data on transmissive meshes, scaled so that the
smoothness indicators are a few times eps = 1e-6.  There every parameter of the
weights moves gamma_e by 1e-4 or more:

  * eps = 1e-6 and r = 2 in the vertex weights (eq. taylorcand) and in the cell
    weights (eq. finalweno);
  * the linear weights gamma_l = 1e-3 of the vertex candidates and
    gamma_0 = 1 - v_e 1e-3 of the cell's own polynomial (v_e = 2 in 1D, 4 in 2D);
  * the factor h^(2|k|) of the pointwise indicator (eq. pointsnorm) and
    h^(2|k|-d) of the element semi-norm (eq. snorm);
  * gamma_e = 1 - min(1, ||u - u*||_e / ||u||_e) (eq. gamma, q = 1).

The expected values are computed here in closed form.  For linear and bilinear
functions every semi-norm integral has an exact expression in the polynomial's
coefficients about the cell centre, so the test needs no quadrature, no Taylor
evaluation at quadrature points and no Legendre routine: it shares no step with
the oracle, which integrates every derivative of every candidate by tensor Gauss
quadrature.  Changing any one of eps, r, gamma_0, gamma_l or either h exponent in
the oracle turns at least one of these tests red (checked by planting each change
in the oracle's C source).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2601_16911_gb300 import inputs as I

EPS, R, GV = 1e-6, 2.0, 1e-3


# --------------------------------------------------------------------------- 1D P1

DX1 = 0.25                          # three cells on [0, 0.75]; h_e = dx in 1D (reading A3)
SLOPES1 = 4e-6 * np.array([0.2, 10.0, -0.3])   # a kink: flat, steep, flat
U_LEFT1 = 0.3                       # value at x = 0 of the continuous broken line


def _broken_line_1d():
    """Legendre P1 coefficients (mean, b) of the continuous broken line with SLOPES1.
    On a cell, u = mean + b xi with xi = 2 (x - x_e)/dx, so the slope is 2 b / dx."""
    nodes = U_LEFT1 + np.concatenate([[0.0], np.cumsum(SLOPES1 * DX1)])
    mean = 0.5 * (nodes[:-1] + nodes[1:])
    b = SLOPES1 * DX1 / 2.0
    u = np.zeros((1, 3, 2))
    u[0, :, 0], u[0, :, 1] = mean, b
    return u, nodes


def expected_1d():
    """Work-through of the sensor on the 1D kink.

    (a) Taylor data (eq. taylorsol) of cell e at its vertex x_i: (u^e(x_i), s_e),
        s_e the cell's slope.  Pointwise indicator (eq. pointsnorm, q = 1, only
        k = 1): beta = sqrt(h^2 s_e^2) = h |s_e|.  With h = 0.25 and
        s = (0.8, 40, -1.2) 1e-6 these are 0.2, 10 and 0.3 times 1e-6.
    (b) Vertex weights w = (eps + beta)^-r, normalised over the patch; the
        vertex candidate is T* = sum w T / sum w.  Interior vertex 1 joins cells
        0 and 1: w = (1.2e-6)^-2 and (11e-6)^-2, normalised 0.9882 and 0.0118,
        so T*_x = 1.261e-6, near the flat cell's 0.8e-6.  Vertex 2 (weights
        0.0138, 0.9862) gives T*_x = -6.32e-7, near the right cell's -1.2e-6.
        Boundary vertices hold one cell (transmissive, A15).
    (c) Candidates of cell e: its own slope s_e and the slopes T*_x of its left
        and right vertex candidates.  For a linear v on a cell of length dx the
        element semi-norm (eq. snorm, d = 1) is sqrt(h^(2-1) dx v'^2).  Cell
        weights omega_l = gamma_l (eps + beta_l)^-r / sum, gamma_0 = 1 - 2e-3,
        gamma_1 = gamma_2 = 1e-3.  u* has slope sum omega_l slope_l, and
        gamma_e = 1 - min(1, |s_e - slope*| / |s_e|).  The steep middle cell:
        omega = (0.8617, 0.0604, 0.0779) to four places, gamma_1 = 0.862383, so it
        is troubled (gamma < 0.9); the flat cells stay near 1 (0.99952, 0.99940).
    nu_e = lambda_e h / (2p) (eq. lostab) with lambda_e = max |u| over the cell's
    Gauss and face nodes (Burgers, reading A2): the right end of each cell here
    (the data are positive and the middle cell's slope dominates), about 0.3, so
    nu_e = 0.3 * 0.25 / 2 = 0.0375 to five places.
    """
    _, nodes = _broken_line_1d()
    h = DX1
    s = SLOPES1
    taylor = {}  # (cell, corner) -> (value, slope)
    for e in range(3):
        taylor[(e, 0)] = (nodes[e], s[e])
        taylor[(e, 1)] = (nodes[e + 1], s[e])
    tstar = np.zeros((4, 2))
    for v in range(4):
        patch = [(v - 1, 1)] if v > 0 else []
        patch += [(v, 0)] if v < 3 else []
        w = np.array([(EPS + h * abs(taylor[c][1])) ** (-R) for c in patch])
        tstar[v] = sum(wi * np.array(taylor[c]) for wi, c in zip(w, patch)) / w.sum()
    gamma, omega = np.zeros(3), np.zeros((3, 3))
    for e in range(3):
        slopes = np.array([s[e], tstar[e, 1], tstar[e + 1, 1]])
        beta = np.sqrt(h ** (2 - 1) * DX1 * slopes ** 2)
        lin = np.array([1.0 - 2 * GV, GV, GV])
        om = lin / (EPS + beta) ** R
        om /= om.sum()
        omega[e] = om
        gamma[e] = 1.0 - min(1.0, abs(s[e] - om @ slopes) / abs(s[e]))
    lam = np.abs(nodes[1:])            # max |u| of an increasing or decreasing line: an end
    lam = np.maximum(lam, np.abs(nodes[:-1]))
    nu = lam * h / 2.0
    return tstar, gamma, omega, nu


def _mesh_1d():
    return I.mesh(1, 3, degree=1, system=I.BURGERS, bc=I.TRANSMISSIVE, domain=(0.0, 3 * DX1, 0.0, 1.0))


def test_1d_kink_vertex_candidates():
    u, _ = _broken_line_1d()
    tstar, _, _, _ = expected_1d()
    got = O.vertex_average(_mesh_1d(), u)
    np.testing.assert_allclose(got[:, 0], tstar[:, 0], rtol=1e-12, atol=0)
    np.testing.assert_allclose(got[:, 1], tstar[:, 1], rtol=1e-12, atol=0)


def test_1d_kink_sensor_and_viscosity():
    u, _ = _broken_line_1d()
    tstar, gamma, omega, nu = expected_1d()
    out = O.residual(_mesh_1d(), u)
    np.testing.assert_allclose(out["gamma"], gamma, rtol=0, atol=1e-12)
    np.testing.assert_allclose(out["nu"], nu, rtol=1e-12, atol=0)
    # the worked numbers of the docstring
    assert abs(gamma[1] - 0.862383) < 5e-7
    np.testing.assert_allclose(omega[1], [0.8617, 0.0604, 0.0779], atol=5e-5)
    np.testing.assert_allclose(tstar[1:3, 1], [1.261e-6, -6.32e-7], rtol=1e-3)
    assert list(out["troubled"]) == [0, 1, 0]


# --------------------------------------------------------------------------- 2D Q1

DX2, DY2 = 0.25, 0.125               # 2 x 2 cells on [0, 0.5] x [0, 0.25]
# Legendre Q1 coefficients (c00, c10, c01, c11) per cell (cell = i + 2 j):
# u = c00 + c10 xi + c01 eta + c11 xi eta; the non-mean ones scaled by 1e-6.
COEF2 = np.array([[0.3, 0.2, 0.1, 0.05],
                  [0.1, 8.0, 3.0, 2.0],
                  [0.2, -0.3, 0.2, 0.1],
                  [0.4, 0.1, -0.2, 0.05]])
COEF2[:, 1:] *= 1e-6


def _state_2d():
    u = np.zeros((1, 4, 4))
    u[0] = COEF2  # Legendre mode order k = kx + 2 ky: (0,0), (1,0), (0,1), (1,1)
    return u


def _centre_form(c):
    """u about the cell centre: u = A + B X + C Y + D X Y, X = x - x_c, Y = y - y_c."""
    c00, c10, c01, c11 = c
    return np.array([c00, 2 * c10 / DX2, 2 * c01 / DY2, 4 * c11 / (DX2 * DY2)])


def _snorm2(B, C, D, h):
    """||v||_e^2 of eq. snorm (d = 2, q = 1) for v = A + B X + C Y + D X Y on a
    dx x dy cell, tensor set {0,1}^2 without k = 0 (reading A5):
      k = (1,0): h^0 int (B + D Y)^2 = dx (B^2 dy + D^2 dy^3 / 12)
      k = (0,1): h^0 int (C + D X)^2 = dy (C^2 dx + D^2 dx^3 / 12)
      k = (1,1): h^2 int D^2         = h^2 dx dy D^2
    (the odd moments of X and Y vanish about the centre)."""
    return (DX2 * (B * B * DY2 + D * D * DY2 ** 3 / 12.0) + DY2 * (C * C * DX2 + D * D * DX2 ** 3 / 12.0)
            + h ** 2 * DX2 * DY2 * D * D)


def expected_2d():
    """Work-through of the sensor on the 2 x 2 Q1 case (h = sqrt(dx^2 + dy^2), A3).

    (a) At corner (xi_c, eta_c) in {-1, 1}^2 of cell e the Taylor data
        (eq. taylorsol, tensor set A5) are u, u_x = (2/dx)(c10 + c11 eta_c),
        u_y = (2/dy)(c01 + c11 xi_c), u_xy = 4 c11 / (dx dy).  Pointwise
        indicator (eq. pointsnorm): beta^2 = h^2 (u_x^2 + u_y^2) + h^4 u_xy^2.
    (b) Vertex weights (eps + beta)^-2 over the patch: four cells at the centre
        vertex, two on the edge midpoints, one at the domain corners.
    (c) The candidate from vertex x_i is T*_0 + T*_x (x-x_i) + T*_y (y-y_i) +
        T*_xy (x-x_i)(y-y_i).  About the cell centre this is B = T*_x + T*_xy o_y,
        C = T*_y + T*_xy o_x, D = T*_xy with (o_x, o_y) = x_c - x_i; its
        semi-norm is `_snorm2`.  Cell weights with gamma_0 = 1 - 4e-3 and
        gamma_l = 1e-3; u - u* has the coefficients of the cell's own minus the
        weighted sum, and gamma_e = 1 - min(1, ||u - u*||_e / ||u||_e).
        The steep cell 1 gets gamma_1 = 0.691587 (troubled), the others stay
        above 0.996.
    """
    h = math.hypot(DX2, DY2)
    taylor = {}
    for e in range(4):
        c00, c10, c01, c11 = COEF2[e]
        for c in range(4):
            xi, eta = (1.0 if c & 1 else -1.0), (1.0 if c >> 1 else -1.0)
            taylor[(e, c)] = np.array([c00 + c10 * xi + c01 * eta + c11 * xi * eta,
                                       2.0 / DX2 * (c10 + c11 * eta), 2.0 / DY2 * (c01 + c11 * xi),
                                       4.0 / (DX2 * DY2) * c11])
    patches = {}
    for e in range(4):
        i, j = e % 2, e // 2
        for c in range(4):
            patches.setdefault((i + (c & 1), j + (c >> 1)), []).append((e, c))
    tstar = {}
    for v, patch in patches.items():
        acc, wsum = np.zeros(4), 0.0
        for key in patch:
            T = taylor[key]
            beta = math.sqrt(h ** 2 * (T[1] ** 2 + T[2] ** 2) + h ** 4 * T[3] ** 2)
            w = (EPS + beta) ** (-R)
            acc += w * T
            wsum += w
        tstar[v] = acc / wsum
    gamma = np.zeros(4)
    for e in range(4):
        i, j = e % 2, e // 2
        xc, yc = (i + 0.5) * DX2, (j + 0.5) * DY2
        cands = [_centre_form(COEF2[e])[1:]]
        for c in range(4):
            V = (i + (c & 1), j + (c >> 1))
            ox, oy = xc - V[0] * DX2, yc - V[1] * DY2
            T = tstar[V]
            cands.append(np.array([T[1] + T[3] * oy, T[2] + T[3] * ox, T[3]]))
        beta = np.array([math.sqrt(_snorm2(*x, h)) for x in cands])
        lin = np.array([1.0 - 4 * GV] + [GV] * 4)
        om = lin / (EPS + beta) ** R
        om /= om.sum()
        diff = cands[0] - sum(o * x for o, x in zip(om, cands))
        gamma[e] = 1.0 - min(1.0, math.sqrt(_snorm2(*diff, h)) / beta[0])
    return tstar, gamma


def _mesh_2d():
    return I.mesh(2, 2, 2, degree=1, system=I.BURGERS, bc=I.TRANSMISSIVE, domain=(0.0, 2 * DX2, 0.0, 2 * DY2))


def test_2d_q1_vertex_candidates():
    d = _mesh_2d()
    tstar, _ = expected_2d()
    got = O.vertex_average(d, _state_2d())
    # transmissive 2 x 2: vertices in row-major order of the 3 x 3 lattice
    for v in range(9):
        exp = tstar[(v % 3, v // 3)]
        np.testing.assert_allclose(got[v], exp, rtol=1e-12, atol=1e-12 * np.abs(exp).max())


def test_2d_q1_sensor():
    _, gamma = expected_2d()
    out = O.residual(_mesh_2d(), _state_2d())
    np.testing.assert_allclose(out["gamma"], gamma, rtol=0, atol=1e-12)
    assert abs(gamma[1] - 0.691587) < 5e-7
    assert list(out["troubled"]) == [0, 1, 0, 0]


@pytest.mark.parametrize("which", ["eps", "r", "gamma_vertex"])
def test_parameters_reach_the_sensor(which):
    """The descriptor's eps, r and gamma_vertex are the ones the sensor uses: a
    changed value moves gamma_e of the steep cells by more than 1e-5."""
    d = _mesh_1d()
    base = O.residual(d, _broken_line_1d()[0])["gamma"]
    d2 = dict(d, **{which: {"eps": 1e-5, "r": 1.0, "gamma_vertex": 2e-3}[which]})
    moved = O.residual(d2, _broken_line_1d()[0])["gamma"]
    assert np.abs(moved - base).max() > 1e-5
