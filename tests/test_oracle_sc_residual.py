"""Pins of the oracle's stages (d) and (e) and of its SSP-RK3 driver.

  * (d) the nonlinear weights preserve each cell's dissipation rate (Sec. 4, the
    identity D^scaled = D^orig), are all 1 for p = 1 in 1D (Sec. 4 remark), and
    follow the pointwise indicator of eq. alpha_prelim (Fig. quadweights set-up);
  * (e) for global polynomial data the residual is the exact time derivative
    (linear advection, Burgers for exactly integrated degrees, the Euler density
    wave), DG cell mass is conserved (eq. convop, zero-sum of s_h), gamma = 0 gives
    LLF plus the low-order viscosity of eq. lostab, and SC leaves s_h(u, u) unchanged;
  * SSP-RK3 on a linear operator is the cubic Taylor polynomial of exp(dt L).
"""
import math

import numpy as np
import pytest
from numpy.polynomial import legendre as L

from oracle import oracle as O
from paper_2601_16911_gb300 import inputs as I
from tests.legendre_ref import Poly2D, leg_coeffs_1d, project_state_1d, project_state_2d


def grad_at_gauss_2d(u_cell, p, dx, dy):
    """grad u at the (p+1)^2 Gauss points of a cell, numpy Legendre evaluation."""
    n = p + 1
    xi, w = L.leggauss(n)
    c = u_cell.reshape(n, n)  # [my, mx]
    P = np.array([L.legval(xi, np.eye(n)[m]) for m in range(n)])
    dP = np.array([L.legval(xi, L.legder(np.eye(n)[m])) for m in range(n)])
    gx = np.einsum("yx,xa,yb->ab", c, dP, P) * 2 / dx  # [qx, qy]
    gy = np.einsum("yx,xa,yb->ab", c, P, dP) * 2 / dy
    W = np.outer(w, w) * dx * dy / 4
    return gx, gy, W


def test_sc_preserves_cell_dissipation_rate():
    d, ic = I.kpp(1, n=10, degree=3)
    u = O.project(d, *ic)
    out = O.residual(d, u)
    tr = out["troubled"].astype(bool)
    assert tr.sum() > 5
    p, n = 3, 10
    dx = dy = 4.0 / n
    for e in np.nonzero(tr)[0]:
        gx, gy, W = grad_at_gauss_2d(u[0, e], p, dx, dy)
        f = (1 - out["gamma"][e]) * (gx ** 2 + gy ** 2)  # [qx, qy]
        a = out["alpha"][e, 0].reshape(p + 1, p + 1).T  # stored q = qx + n qy -> [qx, qy]
        orig = np.sum(W * f)
        scaled = np.sum(W * a * f)
        assert abs(scaled - orig) <= 1e-13 * abs(orig)
        assert np.all(a >= 0)
    assert np.all(out["alpha"][~tr] == 1.0)


def test_sc_p1_1d_all_ones():
    d = I.mesh(1, 12, degree=1)
    u = np.zeros((1, 12, 2))
    u[0, :6, 0] = 1.0  # a jump at x = 0.5 and at the periodic boundary
    u[0, 5, 1] = 0.4
    u[0, 6, 1] = -0.3
    out = O.residual(d, u)
    assert out["troubled"].any()
    np.testing.assert_allclose(out["alpha"], 1.0, atol=1e-14)


def test_sc_weights_follow_pointwise_indicator():
    """1D, p = 4, step at the centre of one cell (the set-up of Fig. quadweights).
    eq. alphaq makes alpha_q proportional to the pointwise indicator ||u||_{x_q}
    (eq. alpha_prelim), with the factor fixed by dissipation preservation; the
    indicator is recomputed here from numpy's Legendre derivatives.  The symmetric
    step gives symmetric, non-uniform weights."""
    p, nx = 4, 8
    d = I.mesh(1, nx, degree=p, bc=I.TRANSMISSIVE)
    dx = 1.0 / nx
    xc = 3.5 * dx
    u = project_state_1d(lambda x: (x >= xc).astype(float), nx, p)
    out = O.residual(d, u)
    assert out["troubled"][3] == 1
    a = out["alpha"][3, 0]
    np.testing.assert_allclose(a, a[::-1], rtol=1e-12)
    assert np.ptp(a) > 1e-2
    xi, w = L.leggauss(p + 1)
    c = u[0, 3]
    ind = np.zeros(p + 1)
    grad = L.legval(xi, L.legder(c)) * 2 / dx
    for k in range(1, p + 1):
        dk = L.legval(xi, L.legder(c, k)) * (2 / dx) ** k
        ind += dx ** (2 * k) * dk ** 2  # h_e = dx in 1D
    ind = np.sqrt(ind)
    ratio = a / ind
    np.testing.assert_allclose(ratio, ratio[0], rtol=1e-12)
    f = grad ** 2
    assert abs(np.sum(w * a * f) - np.sum(w * f)) < 1e-13 * np.sum(w * f)


# ---- stage (e): exact residuals on polynomial data -----------------------------------------


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_linear_advection_residual_is_exact_derivative(p):
    rng = np.random.default_rng(p)
    P = Poly2D(rng.standard_normal((p + 1, p + 1)))
    a = (0.7, -1.3)
    nx, ny = 3, 4
    d = I.mesh(2, nx, ny, degree=p, system=I.LINADV, bc=I.TRANSMISSIVE, adv_vx=a[0], adv_vy=a[1])
    u = project_state_2d(P, nx, ny, p)
    dPx, dPy = P.deriv(1, 0), P.deriv(0, 1)
    exact = project_state_2d(lambda x, y: -(a[0] * dPx(x, y) + a[1] * dPy(x, y)), nx, ny, p)
    r = O.residual(d, u)["dudt"]
    np.testing.assert_allclose(r, exact, rtol=0, atol=1e-9 * np.abs(exact).max())


@pytest.mark.parametrize("p", [1, 2])
def test_burgers_1d_residual_exact_for_low_degree(p):
    rng = np.random.default_rng(20 + p)
    coef = rng.standard_normal(p + 1)
    f = lambda x: np.polynomial.polynomial.polyval(x, coef)
    df = lambda x: np.polynomial.polynomial.polyval(x, np.polynomial.polynomial.polyder(coef))
    nx = 5
    d = I.mesh(1, nx, degree=p, system=I.BURGERS, bc=I.TRANSMISSIVE)
    u = project_state_1d(f, nx, p)
    exact = project_state_1d(lambda x: -f(x) * df(x), nx, p)
    r = O.residual(d, u)["dudt"]
    np.testing.assert_allclose(r, exact, rtol=0, atol=1e-10 * np.abs(exact).max())


def test_burgers_2d_residual_exact_q1():
    rng = np.random.default_rng(3)
    P = Poly2D(rng.standard_normal((2, 2)))
    nx, ny = 4, 3
    d = I.mesh(2, nx, ny, degree=1, system=I.BURGERS, bc=I.TRANSMISSIVE)
    u = project_state_2d(P, nx, ny, 1)
    Px, Py = P.deriv(1, 0), P.deriv(0, 1)
    exact = project_state_2d(lambda x, y: -P(x, y) * (Px(x, y) + Py(x, y)), nx, ny, 1)
    r = O.residual(d, u)["dudt"]
    np.testing.assert_allclose(r, exact, rtol=0, atol=1e-10 * np.abs(exact).max())


@pytest.mark.parametrize("p", [1, 2, 3])
def test_euler_density_wave_residual_is_exact(p):
    """Constant velocity and pressure: the Euler flux is affine in rho and
    dU/dt = -(v . grad rho) (1, vx, vy, |v|^2/2) exactly (HLL of equal states = f)."""
    rng = np.random.default_rng(40 + p)
    a = 0.05 * rng.standard_normal((p + 1, p + 1))
    a[0, 0] = 1.0
    R = Poly2D(a)
    vx, vy, p0, g = 0.6, -0.4, 0.8, 1.4
    nx, ny = 3, 3
    d = I.mesh(2, nx, ny, degree=p, system=I.EULER, bc=I.TRANSMISSIVE)
    U = [R, lambda x, y: vx * R(x, y), lambda x, y: vy * R(x, y),
         lambda x, y: p0 / (g - 1) + 0.5 * (vx * vx + vy * vy) * R(x, y)]
    u = project_state_2d(U, nx, ny, p, nvar=4)
    Rx, Ry = R.deriv(1, 0), R.deriv(0, 1)
    adv = lambda x, y: -(vx * Rx(x, y) + vy * Ry(x, y))
    exact = project_state_2d([adv, lambda x, y: vx * adv(x, y), lambda x, y: vy * adv(x, y),
                              lambda x, y: 0.5 * (vx * vx + vy * vy) * adv(x, y)], nx, ny, p, nvar=4)
    r = O.residual(d, u)["dudt"]
    np.testing.assert_allclose(r, exact, rtol=0, atol=1e-9 * np.abs(exact).max())


@pytest.mark.parametrize("bc", [I.PERIODIC, I.TRANSMISSIVE])
def test_euler_constant_state_is_steady(bc):
    d = I.mesh(2, 4, 3, degree=2, system=I.EULER, bc=bc)
    u = O.project(d, I.IC_QUADRANTS, [0.5, 0.5] + [1.2, 0.3, -0.2, 0.9] * 4)
    r = O.residual(d, u)["dudt"]
    assert np.abs(r).max() < 1e-12


@pytest.mark.parametrize("case", ["kpp", "burgers1d", "euler", "linadv2d"])
def test_dg_mass_conservation(case):
    if case == "kpp":
        d, ic = I.kpp(2, n=8, degree=2)
    elif case == "burgers1d":
        d, ic = I.burgers1d_step(4, nx=16, degree=3)
    elif case == "euler":
        d, ic = I.euler_quadrants(5, n=6, degree=2)
        d["bc"] = (I.PERIODIC,) * 4
    else:
        d = I.mesh(2, 6, 5, degree=3, system=I.LINADV, adv_vx=0.4, adv_vy=0.9)
        ic = (I.IC_CIRCLE, [0.5, 0.5, 0.3, 2.0, -1.0])
    u = O.project(d, *ic)
    out = O.residual(d, u)
    r = out["dudt"]
    if case in ("kpp", "linadv2d"):
        assert out["troubled"].any()
    # int_Omega du_h/dt = sum_e |K_e| * (mode-0 coefficient of dudt)
    tot = r[:, :, 0].sum(axis=1)
    scale = np.abs(r[:, :, 0]).sum(axis=1) + 1e-30
    assert np.all(np.abs(tot) <= 1e-12 * scale)


def test_gamma_zero_is_llf_plus_low_order_viscosity():
    """1D linear advection, gamma forced to 0, SC off:
    dudt = -a u' - nu M^{-1} int phi' u', nu = |a| h / (2p) (eq. lostab)."""
    p, nx, a = 3, 5, 0.8
    coef = np.array([0.2, -1.0, 0.7, 0.3])
    f = lambda x: np.polynomial.polynomial.polyval(x, coef)
    df = lambda x: np.polynomial.polynomial.polyval(x, np.polynomial.polynomial.polyder(coef))
    d = I.mesh(1, nx, degree=p, system=I.LINADV, bc=I.TRANSMISSIVE, adv_vx=a, sensor_mode=2, sc_quadrature=0)
    u = project_state_1d(f, nx, p)
    dx = 1.0 / nx
    nu = abs(a) * dx / (2 * p)
    n = p + 1
    dP = [L.legder(np.eye(n)[m]) for m in range(n)]
    xi, w = L.leggauss(n + 2)
    K = np.array([[np.sum(w * L.legval(xi, dP[m]) * L.legval(xi, dP[k])) for k in range(n)] for m in range(n)])
    M = np.array([dx / (2 * m + 1) for m in range(n)])
    exact = project_state_1d(lambda x: -a * df(x), nx, p)
    for i in range(nx):
        exact[0, i] -= nu * (2.0 / dx) * (K @ u[0, i]) / M
    r = O.residual(d, u)["dudt"]
    np.testing.assert_allclose(r, exact, rtol=0, atol=1e-11 * np.abs(exact).max())


def test_sc_keeps_dissipation_rate_of_each_cell():
    """s_h(u, u) per cell is unchanged by the quadrature redistribution: the
    residuals with and without SC differ only in the viscous term, whose pairing
    with u (mass-weighted) must vanish cell by cell."""
    d, ic = I.kpp(4, n=8, degree=3)
    u = O.project(d, *ic)
    on = O.residual(d, u)
    d_off = dict(d, sc_quadrature=0)
    off = O.residual(d_off, u)
    assert on["troubled"].any()
    n = 4
    M = np.array([1.0 / ((2 * mx + 1) * (2 * my + 1)) for my in range(n) for mx in range(n)])
    pair = np.einsum("ek,ek,k->e", u[0], on["dudt"][0] - off["dudt"][0], M)
    scale = np.einsum("ek,ek,k->e", np.abs(u[0]), np.abs(on["dudt"][0] - off["dudt"][0]), M) + 1e-30
    assert np.all(np.abs(pair) <= 1e-10 * scale)
    assert np.abs(on["dudt"] - off["dudt"]).max() > 1e-6  # SC does change the residual


def test_ssprk3_is_cubic_taylor_polynomial_for_linear_operator():
    """Linear advection with gamma forced to 1 (no viscosity) is linear: one SSP-RK3
    step equals (1 + dtL + dt^2 L^2/2 + dt^3 L^3/6) u."""
    rng = np.random.default_rng(11)
    d = I.mesh(2, 5, 4, degree=2, system=I.LINADV, adv_vx=0.9, adv_vy=0.5, sensor_mode=1)
    u = rng.standard_normal(O.state_shape(d))
    Lop = lambda v: O.residual(d, v)["dudt"]
    dt = 0.01
    L1 = Lop(u)
    L2 = Lop(L1)
    L3 = Lop(L2)
    ref = u + dt * L1 + dt ** 2 / 2 * L2 + dt ** 3 / 6 * L3
    got = O.ssprk3(d, u, dt, 1)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.abs(u).max())
