"""GPU parity of every stage of the path against the FP64 oracle, through the C ABI.

Each case feeds both sides the same FP32-rounded coefficients.  Bars:
  * integer tables (vertex patches, cell corners) bit-exact against the oracle's
    geometric search; the colouring valid;
  * (a)+(b) vertex candidates, (c) gamma_e / nu_e, (d) alpha_q and (e) dudt within
    the FP32 tolerances of tests/gpu_common.py (residual: max relative error 1e-5);
  * where FP32 rounding takes the SC decision (gamma_e within 1e-4 of C_gamma) the
    GPU is given the oracle's decision, and gamma is compared only on cells whose
    data are not flat to rounding level.
Meshes are ragged against the 16x8 (2D) and 128 (1D) tiles, periodic and
transmissive, from 1x1 to several tiles, degree 1..4.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2601_16911_gb300 import cvweno as cv
from paper_2601_16911_gb300 import inputs as I
from tests.gpu_common import (ALPHA_TOL, GAMMA_TOL, RES_TOL, borderline_override, nonflat_mask, rel_err, residual_pair, rounded,
                              to_gpu)

pytestmark = pytest.mark.gpu


def case(name):
    if name == "burgers1d_cfg1":
        return I.burgers1d_step(0, nx=128, degree=2)
    if name.startswith("burgers1d_p"):
        p = int(name[-1])
        return I.burgers1d_step(1, nx=37, degree=p)
    if name.startswith("kpp_p"):
        p = int(name[-1])
        return I.kpp(2, n=20, degree=p)
    if name.startswith("burgers2d_p"):
        p = int(name[-1])
        g = I.SplitMix64(3)
        d = I.mesh(2, 24, 19, degree=p, system=I.BURGERS, bc=I.TRANSMISSIVE)
        return d, (I.IC_FOURIER, I.fourier_modes(g))
    if name == "linadv_circle":
        d = I.mesh(2, 17, 9, degree=2, system=I.LINADV, adv_vx=0.7, adv_vy=-0.4)
        return d, (I.IC_CIRCLE, [0.4, 0.5, 0.3, 2.0, -1.0])
    if name.startswith("euler_p"):
        p = int(name[-1])
        return I.euler_quadrants(4, n=20, degree=p)
    if name == "euler_wave":
        d = I.mesh(2, 18, 11, degree=2, system=I.EULER)
        return d, (I.IC_DENSITY_WAVE, [0.3, 1.0, 2.0, 0.7, -0.4, 0.9])
    if name.startswith("tiny"):
        nx, ny, bc = {"tiny11p": (1, 1, I.PERIODIC), "tiny23p": (2, 3, I.PERIODIC),
                      "tiny31t": (3, 1, I.TRANSMISSIVE), "tiny22t": (2, 2, I.TRANSMISSIVE)}[name]
        d = I.mesh(2, nx, ny, degree=2, system=I.KPP, bc=bc, domain=(-2, 2, -2, 2), lambda_const=1.0)
        rng = np.random.default_rng(nx * 10 + ny)
        return d, ("random", rng)
    raise KeyError(name)


def initial(d, ic):
    if ic[0] == "random":
        return ic[1].standard_normal(O.state_shape(d)) * 0.5
    return O.project(d, *ic)


ALL = (["burgers1d_cfg1"] + [f"burgers1d_p{p}" for p in (1, 3, 4)] + [f"kpp_p{p}" for p in (1, 2, 3, 4)]
       + ["burgers2d_p2", "burgers2d_p3", "linadv_circle", "tiny11p", "tiny23p", "tiny31t", "tiny22t"]
       + ["euler_p1", "euler_p2", "euler_p3", "euler_p4", "euler_wave"])


@pytest.mark.parametrize("name", ALL)
def test_tables_bit_exact(name):
    d, _ = case(name)
    mesh = cv.Mesh(d)
    cvert, vcells, colour = mesh.tables()
    cnt, cell, cor, ocv = O.vertex_patches(d)
    assert np.array_equal(cvert, ocv)
    nc = cvert.shape[1]
    ref = np.full((len(cnt), nc), -1, np.int32)
    for v in range(len(cnt)):
        for s in range(cnt[v]):
            ref[v, nc - 1 - cor[v, s]] = cell[v, s]  # the cell touching with corner c sits in slot (2^d-1) - c
    assert np.array_equal(vcells, ref)
    # colouring: no two distinct cells sharing a vertex have one colour
    for v in range(vcells.shape[0]):
        cs = [c for c in vcells[v] if c >= 0]
        cols = {}
        for c in cs:
            if c in cols:
                continue
            cols[c] = colour[c]
        assert len(set(cols.values())) == len(cols)
    mesh.close()


@pytest.mark.parametrize("name", ALL)
def test_projection_parity(name):
    d, ic = case(name)
    if ic[0] == "random":
        pytest.skip("random coefficients, no analytic datum")
    mesh = cv.Mesh(d)
    got = mesh.project(*ic).cpu().numpy()
    ref = O.project(d, *ic)
    # the 12-point projection rule (reading A17) evaluated in FP32: a few ulps of the
    # largest coefficient
    assert rel_err(got, ref) < 2e-6
    mesh.close()


@pytest.mark.parametrize("name", ALL)
def test_vertex_candidates_parity(name):
    """Stages (a)+(b): the vertex candidates' derivatives, per derivative order."""
    d, ic = case(name)
    u = rounded(initial(d, ic))
    ref = O.vertex_average(d, u)
    mesh = cv.Mesh(d)
    got = mesh.vertex_data(to_gpu(u)).cpu().numpy()
    mesh.close()
    scale = np.abs(ref).max(axis=0) + 1e-30
    err = (np.abs(got - ref) / scale).max()
    assert err < 1e-5, err


@pytest.mark.parametrize("name", ALL)
def test_full_stage_parity(name):
    """Stages (a)-(e): gamma, nu, alpha, troubled flags and dudt."""
    d, ic = case(name)
    u, ref, got, nflip = residual_pair(d, initial(d, ic))
    mask = nonflat_mask(u)
    gerr = np.abs(got["gamma"] - ref["gamma"])[mask]
    assert gerr.size == 0 or gerr.max() < GAMMA_TOL, gerr.max()
    assert rel_err(got["nu"], ref["nu"]) < 1e-6
    # SC decisions agree wherever they are not decided by rounding
    dec = np.abs(ref["gamma"] - d["c_gamma"]) >= 1e-4
    assert np.array_equal(got["troubled"][dec & mask], ref["troubled"][dec & mask])
    both = (got["troubled"] == 1) & (ref["troubled"] == 1) & mask
    if both.any():
        aerr = np.abs(got["alpha"][both] - ref["alpha"][both]).max() / np.abs(ref["alpha"][both]).max()
        assert aerr < ALPHA_TOL, aerr
    # the smooth Euler density wave (not one of the workloads) sits on the FP32 floor
    # of the flux evaluation: reading A26 -- the error is the same with gamma taken
    # from the GPU (pure arithmetic), bounded here by 1e-4
    tol = 1e-4 if name == "euler_wave" else RES_TOL
    assert rel_err(got["dudt"], ref["dudt"]) < tol


@pytest.mark.parametrize("name", ["kpp_p3", "burgers1d_cfg1", "burgers2d_p2"])
def test_sensor_entry_point_matches_full_stage(name):
    d, ic = case(name)
    u = to_gpu(rounded(initial(d, ic)))
    mesh = cv.Mesh(d)
    g, nu = mesh.sensor(u)
    full = mesh.residual_ex(u)
    assert torch.equal(g, full["gamma"]) and torch.equal(nu, full["nu"])
    r = mesh.residual(u)
    assert torch.equal(r, full["dudt"])
    mesh.close()


@pytest.mark.parametrize("name", ["kpp_p2", "burgers1d_cfg1", "linadv_circle", "burgers2d_p3", "euler_p3"])
def test_ssprk3_step_parity(name):
    d, ic = case(name)
    u = rounded(initial(d, ic))
    lam = O.max_wavespeed(d, u)
    h = min((d["x1"] - d["x0"]) / d["nx"], (d["y1"] - d["y0"]) / d["ny"] if d["dim"] == 2 else 1e9)
    dt = 0.1 * h / (d["dim"] * lam)
    ref = O.ssprk3(d, u, dt, 1)
    mesh = cv.Mesh(d)
    ug = to_gpu(u)
    mesh.step(ug, dt=dt)
    mesh.status_check()
    assert rel_err(ug.cpu().numpy(), ref) < RES_TOL
    # CFL path: the FP64 max wave speed agrees and the step size follows from it
    assert abs(mesh.max_wavespeed(to_gpu(u)) - lam) <= 1e-6 * lam
    mesh.close()


def test_mass_total_matches_oracle():
    d, ic = I.kpp(5, n=24, degree=3)
    u = rounded(O.project(d, *ic))
    mesh = cv.Mesh(d)
    tot = mesh.mass_total(to_gpu(u))
    ref = O.mass_total(d, u)
    assert abs(tot[0] - ref[0]) <= 1e-12 * abs(ref[0])
    mesh.close()
