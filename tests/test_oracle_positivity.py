"""Pins of the oracle's positivity limiter for the Euler equations (readings P1-P4; the
scaling limiter of Zhang and Shu restated with a relative floor, not part of the paper): admissible data pass
unchanged, limited data are admissible at every volume and face Gauss node and keep
their cell means, the limiting is tight (the pressure touches eps at the binding node),
and an inadmissible mean is reported."""
import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import oracle as O
from paper_2601_16911_gb300 import inputs as I

G = 1.4


def euler_mesh(n=5, p=2):
    return I.mesh(2, n, n, degree=p, system=I.EULER, bc=I.TRANSMISSIVE)


def random_state(d, rng, amp):
    """Cell means admissible (rho ~ 1, p ~ 0.5), non-mean modes of size amp."""
    nd = (d["degree"] + 1) ** 2
    ne = d["nx"] * d["ny"]
    u = rng.uniform(-amp, amp, (4, ne, nd)) / np.arange(1, nd + 1)
    rho = rng.uniform(0.8, 1.2, ne)
    mx, my = rng.uniform(-0.3, 0.3, ne), rng.uniform(-0.3, 0.3, ne)
    p = rng.uniform(0.3, 0.7, ne)
    u[0, :, 0], u[1, :, 0], u[2, :, 0] = rho, mx, my
    u[3, :, 0] = p / (G - 1) + 0.5 * (mx * mx + my * my) / rho
    return u


def point_values(d, u):
    """Every variable at the volume and face Gauss nodes of every cell, evaluated here
    from the Legendre coefficients (numpy), independently of the oracle."""
    n = d["degree"] + 1
    x, _ = np.polynomial.legendre.leggauss(n)
    pts = [(a, b) for b in x for a in x] + [(1.0, t) for t in x] + [(-1.0, t) for t in x] + \
          [(t, 1.0) for t in x] + [(t, -1.0) for t in x]
    xs = np.array([q[0] for q in pts])
    ys = np.array([q[1] for q in pts])
    Vx = npleg.legvander(xs, n - 1)
    Vy = npleg.legvander(ys, n - 1)
    B = np.einsum("pi,pj->pji", Vx, Vy).reshape(len(pts), n * n)  # mode mx + n my
    return np.einsum("pm,vem->vep", B, u)


def pressure(U):
    return (G - 1) * (U[3] - 0.5 * (U[1] ** 2 + U[2] ** 2) / U[0])


def test_admissible_data_pass_unchanged():
    d = euler_mesh()
    u = random_state(d, np.random.default_rng(0), 0.05)
    out, th, code = O.positivity(d, u)
    assert code == 0 and np.all(th == 1.0)
    assert np.array_equal(out, u)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_limited_state_is_admissible_tight_and_conservative(p):
    d = euler_mesh(p=p)
    rng = np.random.default_rng(p)
    u = random_state(d, rng, 1.6)
    V0 = point_values(d, u)
    assert (V0[0] < 0).any() and (pressure(V0) < 0).any()  # the data need limiting
    out, th, code = O.positivity(d, u)
    assert code == 0
    assert np.array_equal(out[:, :, 0], u[:, :, 0])  # means kept
    V = point_values(d, out)
    rho, pr = V[0], pressure(V)
    eps = 1e-3 * np.minimum(u[0, :, 0], pressure(u[:, :, 0]))
    assert np.all(rho >= eps[:, None] * (1 - 1e-9) - 1e-12)
    assert np.all(pr >= eps[:, None] - 1e-9)
    limited = th < 1.0
    assert limited.sum() >= 3
    # tight: in each cell limited for pressure, the binding node sits at p = eps
    for e in np.nonzero(limited)[0]:
        if (pressure(V0[:, e, :]) < eps[e]).any() and pr[e].min() < 1.001 * eps[e]:
            assert abs(pr[e].min() - eps[e]) < 1e-9
    # cells whose nodes were admissible are untouched
    ok = (V0[0] >= eps[:, None]).all(1) & (pressure(V0) >= eps[:, None]).all(1)
    assert np.array_equal(out[:, ok], u[:, ok])
    assert np.all(th[ok] == 1.0)


def test_density_only_violation_scales_only_the_density():
    """A cell with a negative density node but positive pressure after the density
    step: only the density's non-mean modes are scaled, to rho_min = eps."""
    d = euler_mesh(n=1, p=1)
    u = np.zeros((4, 1, 4))
    u[0, 0] = [1.0, 1.3, 0.0, 0.0]  # rho = 1 + 1.3 xi: negative at xi = -1
    u[3, 0, 0] = 2.5
    out, th, code = O.positivity(d, u)
    V = point_values(d, out)
    eps = 1e-3 * min(1.0, 0.4 * 2.5)
    assert abs(V[0].min() - eps) < 1e-12
    assert np.array_equal(out[1:], u[1:])
    th1 = (1.0 - eps) / (1.0 - (1.0 - 1.3))  # rho_min = 1 - 1.3 at the face xi = -1
    assert abs(th[0] - th1) < 1e-15
    assert np.allclose(out[0, 0, 1:], th1 * u[0, 0, 1:], rtol=1e-15, atol=0)


def test_inadmissible_mean_is_reported_and_left_alone():
    d = euler_mesh(n=2, p=1)
    u = random_state(d, np.random.default_rng(5), 0.01)
    u[0, 2, 0] = -0.1
    out, th, code = O.positivity(d, u)
    assert code == 4
    assert np.array_equal(out[:, 2], u[:, 2])


def test_limited_ssprk3_survives_a_near_vacuum():
    """Two halves moving apart fast at low pressure: the plain scheme reaches a
    non-positive pressure within a few steps; with the limiter in every stage the run
    completes and stays admissible at every node."""
    d = I.mesh(2, 12, 4, degree=2, system=I.EULER, bc=I.TRANSMISSIVE, domain=(-1, 1, 0, 0.5))
    # quadrants: left (rho, vx, vy, p) = (1, -3, 0, 0.01), right (1, 3, 0, 0.01)
    prm = [0.0, 0.25, 1.0, -3.0, 0.0, 0.01, 1.0, 3.0, 0.0, 0.01, 1.0, -3.0, 0.0, 0.01, 1.0, 3.0, 0.0, 0.01]
    u0 = O.project(d, I.IC_QUADRANTS, prm)
    dt = 0.05 * (2.0 / 12) / (3.0 + np.sqrt(1.4 * 0.01)) / 5
    with pytest.raises(RuntimeError):
        O.ssprk3(d, u0.copy(), dt, 10)
    dp = dict(d, positivity=1)
    u = O.ssprk3(dp, u0.copy(), dt, 40)
    V = point_values(d, u)
    assert np.all(V[0] > 0) and np.all(pressure(V) > 0)
    assert np.all(u[0, :, 0] > 0.5)
