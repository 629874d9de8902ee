"""Pins of the oracle's stages (a)-(c): Hermite data, vertex averaging and the
cell-vertex WENO sensor (Sec. 3.2, Sec. 2.2 eq. gamma).

What fixes them without an implementation to compare against:
  * polynomial reproduction: for a global tensor polynomial of degree <= p every
    Taylor expansion (eq. taylorsol) is exact, so the vertex candidates, the WENO
    reconstruction and u^e coincide and gamma_e = 1 (no viscosity);
  * the Taylor data equal the exact derivatives at the cell corners, and the vertex
    smoothness indicators equal the pointwise semi-norm (eq. pointsnorm) of those;
  * equal indicators give equal weights (the vertex value is the patch mean);
  * a perfectly flat neighbour dominates a steep one (WENO stencil selection);
  * gamma_e in [0, 1], and invariance/equivariance under symmetries.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2601_16911_gb300 import inputs as I
from tests.legendre_ref import Poly2D, project_state_1d, project_state_2d


def rand_poly(rng, p, dim):
    a = rng.standard_normal((p + 1, p + 1 if dim == 2 else 1))
    return Poly2D(a)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_projection_matches_numpy(p):
    rng = np.random.default_rng(p)
    P = rand_poly(rng, p, 2)
    d = I.mesh(2, 3, 2, degree=p, bc=I.TRANSMISSIVE, domain=(0.0, 1.0, -0.5, 0.5))
    u_or = O.project(d, I.IC_POLY, P.ic_params())
    u_np = project_state_2d(P, 3, 2, p, dom=(0.0, 1.0, -0.5, 0.5))
    np.testing.assert_allclose(u_or, u_np, rtol=0, atol=1e-12)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_hermite_data_exact_derivatives_2d(p):
    rng = np.random.default_rng(10 + p)
    P = rand_poly(rng, p, 2)
    nx, ny, dom = 3, 4, (0.0, 1.5, 0.0, 1.0)
    d = I.mesh(2, nx, ny, degree=p, bc=I.TRANSMISSIVE, domain=dom)
    u = project_state_2d(P, nx, ny, p, dom=dom)
    T, beta = O.hermite(d, u)
    dx, dy = 1.5 / nx, 1.0 / ny
    h = math.hypot(dx, dy)
    n = p + 1
    for e in range(nx * ny):
        i, j = e % nx, e // nx
        for c in range(4):
            X, Y = (i + (c & 1)) * dx, (j + (c >> 1)) * dy
            s2 = 0.0
            for ky in range(n):
                for kx in range(n):
                    ex = P.deriv(kx, ky)(X, Y)
                    assert abs(T[e, c, kx + n * ky] - ex) < 1e-7 * (1 + abs(ex))  # (2/dx)^kx (2/dy)^ky amplifies rounding
                    if kx + ky:
                        s2 += h ** (2 * (kx + ky)) * ex * ex
            assert abs(beta[e, c] - math.sqrt(s2)) < 1e-7 * (1 + math.sqrt(s2))


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("dim", [1, 2])
def test_polynomial_reproduction(p, dim):
    rng = np.random.default_rng(100 * dim + p)
    P = rand_poly(rng, p, dim)
    if dim == 1:
        nx = 6
        d = I.mesh(1, nx, degree=p, bc=I.TRANSMISSIVE)
        u = project_state_1d(lambda x: P(x, 0.0 * x), nx, p)
    else:
        nx, ny = 4, 3
        d = I.mesh(2, nx, ny, degree=p, bc=I.TRANSMISSIVE)
        u = project_state_2d(P, nx, ny, p)
    Ts = O.vertex_average(d, u)
    n = p + 1
    vx = nx + 1
    for v in range(Ts.shape[0]):
        X = (v % vx) / nx
        Y = (v // vx) / (d["ny"]) if dim == 2 else 0.0
        for t in range(Ts.shape[1]):
            kx, ky = (t % n, t // n) if dim == 2 else (t, 0)
            ex = P.deriv(kx, ky)(X, Y)
            amp = (2.0 * nx) ** kx * ((2.0 * d["ny"]) ** ky if dim == 2 else 1.0)  # rounding of D^k
            assert abs(Ts[v, t] - ex) < 1e-11 * amp * np.abs(u).max() + 1e-9 * abs(ex)
    out = O.residual(d, u)
    assert np.all(np.abs(1.0 - out["gamma"]) < 1e-9)
    assert not out["troubled"].any()


@pytest.mark.parametrize("dim", [1, 2])
def test_equal_indicators_give_patch_mean(dim):
    """Same slope in every cell, random cell means: every corner indicator is equal,
    so the vertex value is the plain mean of the patch's corner values."""
    rng = np.random.default_rng(7)
    p = 2
    nx, ny = 5, 4
    if dim == 1:
        d = I.mesh(1, nx, degree=p)
        u = np.zeros((1, nx, p + 1))
        u[0, :, 0] = rng.standard_normal(nx)
        u[0, :, 1] = 0.3  # slope in every cell, P_1 coefficient
    else:
        d = I.mesh(2, nx, ny, degree=p)
        u = np.zeros((1, nx * ny, (p + 1) ** 2))
        u[0, :, 0] = rng.standard_normal(nx * ny)
        u[0, :, 1] = 0.3
        u[0, :, p + 1] = -0.2
    T, _ = O.hermite(d, u)
    Ts = O.vertex_average(d, u)
    cnt, cell, cor, _ = O.vertex_patches(d)
    for v in range(len(cnt)):
        vals = [T[cell[v, s], cor[v, s], 0] for s in range(cnt[v])]
        assert abs(Ts[v, 0] - np.mean(vals)) < 1e-12
        assert abs(Ts[v, 1] - T[cell[v, 0], cor[v, 0], 1]) < 1e-12


def test_flat_neighbour_dominates_steep_one():
    """1D: a flat cell next to a steep cell; at the shared vertex the vertex
    candidate follows the flat cell (stencil selection of the Jiang-Shu weights)."""
    p, nx = 2, 6
    d = I.mesh(1, nx, degree=p)
    u = np.zeros((1, nx, p + 1))
    u[0, :, 0] = 1.0
    u[0, 3, 1] = 5.0  # cell 3 steep, cell 2 flat
    T, _ = O.hermite(d, u)
    Ts = O.vertex_average(d, u)
    # vertex 3 joins cell 2 (right corner) and cell 3 (left corner)
    flat, steep = T[2, 1], T[3, 0]
    assert np.all(np.abs(Ts[3] - flat) <= 1e-6 * np.abs(steep - flat) + 1e-14)


def _kpp_state(n=10, p=2, seed=3):
    d, ic = I.kpp(seed, n=n, degree=p)
    return d, O.project(d, *ic)


def test_gamma_in_unit_interval_and_detects_jump():
    d, u = _kpp_state()
    g = O.residual(d, u)["gamma"]
    assert np.all(g >= 0.0) and np.all(g <= 1.0)
    # cells that the circle crosses are troubled, cells far from it are smooth
    # (their data is constant up to projection rounding, so gamma is near, not at, 1)
    n = d["nx"]
    assert g.min() < 0.5
    corner_cells = [0, n - 1, n * (n - 1), n * n - 1]
    assert np.all(g[corner_cells] > 0.99)


def test_sensor_invariant_under_constant_shift_and_sign():
    d, u = _kpp_state()
    g0 = O.residual(d, u)["gamma"]
    u2 = u.copy()
    u2[:, :, 0] += 0.37  # adds a constant: derivatives unchanged
    np.testing.assert_allclose(O.residual(d, u2)["gamma"], g0, atol=1e-12)
    np.testing.assert_allclose(O.residual(d, -u)["gamma"], g0, atol=1e-12)


def test_sensor_translation_equivariance():
    d, u = _kpp_state(n=8)
    n, nd = d["nx"], u.shape[2]
    g = O.residual(d, u)["gamma"].reshape(n, n)
    us = np.roll(u.reshape(1, n, n, nd), shift=(1, 2), axis=(1, 2)).reshape(u.shape)
    gs = O.residual(d, us)["gamma"].reshape(n, n)
    np.testing.assert_allclose(gs, np.roll(g, shift=(1, 2), axis=(0, 1)), atol=1e-12)


def test_sensor_mirror_symmetry():
    """x -> -x: cell i -> nx-1-i and Legendre mode mx picks up (-1)^mx."""
    rng = np.random.default_rng(5)
    p, n = 3, 6
    d = I.mesh(2, n, n, degree=p, domain=(-1.0, 1.0, -1.0, 1.0))
    u = rng.standard_normal((1, n * n, (p + 1) ** 2)) * 0.1
    g = O.residual(d, u)["gamma"].reshape(n, n)
    um = u.reshape(1, n, n, p + 1, p + 1)[:, :, ::-1, :, :].copy()  # [var, j, i, my, mx]
    sign = np.array([(-1.0) ** mx for mx in range(p + 1)])
    um = um * sign[None, None, None, None, :]
    gm = O.residual(d, um.reshape(u.shape))["gamma"].reshape(n, n)
    np.testing.assert_allclose(gm, g[:, ::-1], atol=1e-12)
