"""Pins of the oracle's continuous Galerkin (CG) variant.

The CG details are readings (lumped-mass projection P_h, A13; lumped mass with two
defect-correction sweeps, A12), so they are pinned by what the mathematics and the
paper fix:
  * the GLL Lagrange basis reproduces the Legendre-basis sensor data of the same cell
    polynomials (the sensor is basis independent);
  * DG-to-CG consistency of the Taylor data at vertices (u is continuous: the vertex
    values of all cells at a vertex agree);
  * conservation: the integral of du/dt vanishes on a periodic mesh;
  * the paper's printed L1 errors of Table tab:bur2 (CG, 1D Burgers, t = 0.1) and their
    convergence orders, reproduced within a stated factor (tests/golden/).
"""
import math
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as L

from oracle import oracle as O
from paper_2601_16911_gb300 import inputs as I
from tests.test_oracle_convergence import burgers_exact

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "tab_bur2_cvweno_cg.txt")


def gll(p):
    """GLL nodes from numpy: the endpoints and the roots of P_p'."""
    inner = np.sort(np.real(L.legroots(L.legder(np.eye(p + 1)[p])))) if p > 1 else np.array([])
    return np.concatenate([[-1.0], inner, [1.0]])


def lagrange_to_legendre(p):
    """Matrix V with c_legendre = V @ u_nodes for one 1D cell (interpolation, numpy)."""
    x = gll(p)
    # nodal values of Legendre polynomials: A[a, m] = P_m(x_a); c = A^{-1} u
    A = np.array([[L.legval(xa, np.eye(p + 1)[m]) for m in range(p + 1)] for xa in x])
    return np.linalg.inv(A)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_cg_sensor_equals_dg_sensor_of_same_polynomials(p):
    """2D periodic: convert every cell's GLL nodal values to Legendre coefficients with
    numpy; the oracle's CG and DG sensor outputs must then agree."""
    n = 6
    d_cg = I.mesh(2, n, n, degree=p, system=I.KPP, kind=I.CG, domain=(-2, 2, -2, 2), lambda_const=1.0)
    d_dg = dict(d_cg, kind=I.DG)
    rng = np.random.default_rng(p)
    uc = rng.standard_normal(O.state_shape(d_cg))  # nodal values, (1, (p n)^2)
    V = lagrange_to_legendre(p)
    NN = p * n
    ug = np.zeros(O.state_shape(d_dg))
    for j in range(n):
        for i in range(n):
            loc = np.array([[uc[0, ((p * i + a) % NN) + NN * ((p * j + b) % NN)] for a in range(p + 1)]
                            for b in range(p + 1)])  # [b, a]
            coef = V @ loc @ V.T  # [my, mx]
            ug[0, i + n * j] = coef.reshape(-1)
    a = O.residual(d_cg, uc)
    b = O.residual(d_dg, ug)
    np.testing.assert_allclose(a["gamma"], b["gamma"], atol=1e-10)
    np.testing.assert_allclose(a["nu"], b["nu"], rtol=1e-12)
    Ta, _ = O.hermite(d_cg, uc)
    Tb, _ = O.hermite(d_dg, ug)
    np.testing.assert_allclose(Ta, Tb, rtol=1e-9, atol=1e-9 * np.abs(Tb).max())


def test_cg_vertex_values_continuous():
    d = I.mesh(2, 5, 4, degree=3, system=I.KPP, kind=I.CG, domain=(-2, 2, -2, 2), lambda_const=1.0)
    u = np.random.default_rng(1).standard_normal(O.state_shape(d))
    T, _ = O.hermite(d, u)
    cnt, cell, cor, _ = O.vertex_patches(d)
    for v in range(len(cnt)):
        vals = [T[cell[v, s], cor[v, s], 0] for s in range(cnt[v])]
        assert np.ptp(vals) < 1e-12


@pytest.mark.parametrize("case", ["kpp", "burgers1d"])
def test_cg_conservation(case):
    if case == "kpp":
        d, ic = I.kpp(3, n=10, degree=2, kind=I.CG)
    else:
        d, ic = I.burgers1d_step(2, nx=24, degree=3)
        d["kind"] = I.CG
    u = O.project(d, *ic)
    out = O.residual(d, u)
    assert out["troubled"].any()
    tot = O.mass_total(d, out["dudt"])[0]
    scale = O.mass_total(d, np.abs(out["dudt"]))[0]
    assert abs(tot) <= 1e-12 * scale


def cg_burgers_l1(nx, p, cfl=0.05):
    d = I.mesh(1, nx, degree=p, system=I.BURGERS, kind=I.CG)
    u = O.project(d, I.IC_SINE_STEP, [1.0, 1.0, 0.0, 2.0])
    nst = int(math.ceil(0.1 / (cfl * (1.0 / nx) / p)))
    u = O.ssprk3(d, u, 0.1 / nst, nst)
    vals, xs, _, ws = O.eval_points(d, u, 0, 8)
    return float(np.sum(np.abs(vals - burgers_exact(xs, 0.1)) * ws))


def test_cg_burgers_matches_paper_table():
    """Table tab:bur2: within a factor 1.5 for p = 1 and 15 % for p = 2, 3; the
    convergence orders between E_h = 64 and 128 within 0.3 of the paper's (0.5 for
    p = 1, whose printed errors are still pre-asymptotic: EOC 3.06, 2.59, 2.11
    falling towards 2)."""
    rows = [tuple(float(x) for x in ln.split()) for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    got = {}
    for eh, p, ref in rows:
        e = cg_burgers_l1(int(eh), int(p))
        got[(int(eh), int(p))] = (e, ref)
        tol = math.log(1.5) if p == 1 else math.log(1.15)
        assert abs(math.log(e / ref)) <= tol, (eh, p, e, ref)
    for p in (1, 2, 3):
        eoc = math.log(got[(64, p)][0] / got[(128, p)][0]) / math.log(2.0)
        eoc_ref = math.log(got[(64, p)][1] / got[(128, p)][1]) / math.log(2.0)
        assert abs(eoc - eoc_ref) <= (0.5 if p == 1 else 0.3), (p, eoc, eoc_ref)
