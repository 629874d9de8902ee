"""Pins of the oracle's HWENO limiter (Sec. 3: the cell-vertex reconstruction u^{e,*}
overwrites u^e; readings A27, A28): exactness on polynomial data, conservation of
cell means, the blend of the four average-corrected vertex candidates recomputed here
by a least-squares fit of their Taylor forms, the identity when the vertex candidates
carry no weight, the troubled set of the sensor, and the effect of limiting every
stage on a shock."""
import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle import oracle as O
from paper_2601_16911_gb300 import inputs as I


def poly_params(rng, p):
    """IC_POLY coefficients of a polynomial in Q_p (x^i y^j with i, j <= p)."""
    P = np.zeros(25)
    for j in range(p + 1):
        for i in range(p + 1):
            P[i + 5 * j] = rng.uniform(-1, 1)
    return list(P)


@pytest.mark.parametrize("dim,p", [(1, 1), (1, 3), (2, 1), (2, 2), (2, 3), (2, 4)])
def test_polynomial_data_is_left_unchanged(dim, p):
    """Every candidate reproduces a polynomial of Q_p exactly (its vertex data are the
    polynomial's own derivatives), so limiting every cell changes nothing."""
    rng = np.random.default_rng(10 * dim + p)
    d = I.mesh(dim, 5, 4, degree=p, system=I.BURGERS, bc=I.TRANSMISSIVE, domain=(-0.3, 0.9, 0.2, 1.4))
    u = O.project(d, I.IC_POLY, poly_params(rng, p) if dim == 2 else
                  [rng.uniform(-1, 1) if (i < p + 1) else 0.0 for i in range(25)])
    out, tr = O.limit(d, u, all_cells=True)
    assert tr.all()
    assert np.abs(out - u).max() <= 1e-9 * np.abs(u).max()


@pytest.mark.parametrize("dim,p", [(1, 2), (2, 2), (2, 4)])
def test_cell_means_are_conserved(dim, p):
    rng = np.random.default_rng(3 + p)
    d = I.mesh(dim, 6, 5, degree=p, system=I.BURGERS)
    u = rng.standard_normal(O.state_shape(d))
    out, _ = O.limit(d, u, all_cells=True)
    assert np.array_equal(out[..., 0], u[..., 0])
    assert np.abs(out - u).max() > 1e-3  # the rest did change


def taylor_value(Ts, p, dim, ox, oy):
    v = np.zeros_like(ox)
    n = p + 1
    from math import factorial
    for t in range(n ** dim):
        kx, ky = t % n, (t // n if dim == 2 else 0)
        term = Ts[t] * ox ** kx / factorial(kx)
        if dim == 2:
            term = term * oy ** ky / factorial(ky)
        v = v + term
    return v


@pytest.mark.parametrize("dim,p", [(1, 2), (2, 1), (2, 3)])
def test_equal_weights_blend_of_vertex_candidates(dim, p):
    """With eps huge every Jiang-Shu weight equals its linear weight; with the vertex
    linear weight 1/ncorner the cell candidate drops out and u^{e,*} is the plain mean
    of the vertex candidates, each average-corrected.  Recomputed here from the
    oracle's vertex data by sampling each Taylor form and fitting Legendre modes."""
    rng = np.random.default_rng(7 * p + dim)
    nc = 4 if dim == 2 else 2
    d = I.mesh(dim, 4, 3, degree=p, system=I.BURGERS, domain=(0.0, 1.2, 0.0, 0.9), eps=1e30, gamma_vertex=1.0 / nc)
    u = rng.standard_normal(O.state_shape(d))
    out, _ = O.limit(d, u, all_cells=True)
    Ts = O.vertex_average(d, u)
    _, _, _, cvert = O.vertex_patches(d)
    dx = (d["x1"] - d["x0"]) / d["nx"]
    dy = (d["y1"] - d["y0"]) / d["ny"]
    n = p + 1
    xi = rng.uniform(-1, 1, 200)
    eta = rng.uniform(-1, 1, 200) if dim == 2 else np.zeros(200)
    if dim == 2:
        V = npleg.legvander2d(xi, eta, [p, p])  # column index = my + (p+1) mx
        perm = [mx * n + my for my in range(n) for mx in range(n)]  # our index mx + n my
        V = V[:, perm]
    else:
        V = npleg.legvander(xi, p)
    for e in range(O.counts(d)["ncell"]):
        fit = np.zeros(n ** dim)
        for c in range(nc):
            cx, cy = (1.0 if c & 1 else -1.0), (1.0 if c >> 1 else -1.0)
            ox, oy = 0.5 * dx * (xi - cx), 0.5 * dy * (eta - cy)
            vals = taylor_value(Ts[cvert[e, c]], p, dim, ox, oy if dim == 2 else 0 * ox)
            coef, *_ = np.linalg.lstsq(V, vals, rcond=None)
            fit += coef / nc
        fit[0] = u[0, e, 0]
        assert np.abs(out[0, e] - fit).max() <= 1e-9 * max(1.0, np.abs(fit).max()), e


def test_no_vertex_weight_is_identity():
    rng = np.random.default_rng(1)
    d = I.mesh(2, 5, 5, degree=2, system=I.BURGERS, gamma_vertex=0.0)
    u = rng.standard_normal(O.state_shape(d))
    out, _ = O.limit(d, u, all_cells=True)
    assert np.abs(out - u).max() <= 1e-14 * np.abs(u).max()


def test_limits_exactly_the_sensors_troubled_cells():
    d, ic = I.kpp(0, n=16, degree=2)
    u = O.project(d, *ic)
    out, tr = O.limit(d, u)
    ref = O.residual(d, u)
    expect = (ref["gamma"] < d["c_gamma"]).astype(np.int32)
    assert np.array_equal(tr, expect)
    assert 0 < tr.sum() < tr.size
    keep = tr == 0
    assert np.array_equal(out[:, keep], u[:, keep])


def test_limiter_in_every_stage_tames_the_shock():
    """1D Burgers step to t = 0.3 (past the sine's shock time 1/(2 pi)) without
    artificial viscosity (sensor forced smooth): plain DG overshoots the initial range
    at the shocks; limiting every stage (A27) cuts the overshoot several-fold."""
    d0, ic = I.burgers1d_step(0, nx=64, degree=2)
    xs = np.linspace(0.0, 1.0, 4001)
    u_ic = np.array([O.ic_point(d0, ic[0], ic[1], x, 0.0)[0] for x in xs])
    lo, hi = u_ic.min(), u_ic.max()
    u0 = O.project(d0, *ic)
    nst = 576
    dt = 0.3 / nst
    res = {}
    for lim in (0, 1):
        d = dict(d0, sensor_mode=1, hweno_limiter=lim)
        u = O.ssprk3(d, u0.copy(), dt, nst)
        v = O.eval_points(d, u, 0, 5)[0]
        res[lim] = max(v.max() - hi, lo - v.min(), 0.0)
    assert res[0] > 0.05 * (hi - lo), res
    assert res[1] < 0.3 * res[0], res
