"""GPU parity of the CG variant (continuous Q_p, GLL nodal values, periodic meshes)
against the FP64 oracle, through the C ABI: projection, every stage output (gamma, nu,
troubled flags, alpha, nodal du/dt), the SSP-RK3 step, FP64 mass totals, and the
final-time L1 error of 1D Burgers against the exact solution next to the paper's
Table tab:bur2 value."""
import math
import os

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2601_16911_gb300 import cvweno as cv
from paper_2601_16911_gb300 import inputs as I
from tests.gpu_common import ALPHA_TOL, GAMMA_TOL, RES_TOL, borderline_override, rel_err, rounded, to_gpu

pytestmark = pytest.mark.gpu


def case(name):
    if name.startswith("kpp_cg_p"):
        return I.kpp(2, n=20, degree=int(name[-1]), kind=I.CG)
    if name.startswith("burgers1d_cg_p"):
        d, ic = I.burgers1d_step(1, nx=37, degree=int(name[-1]))
        d["kind"] = I.CG
        return d, ic
    if name == "burgers2d_cg_p2":
        g = I.SplitMix64(3)
        return I.mesh(2, 24, 19, degree=2, system=I.BURGERS, kind=I.CG), (I.IC_FOURIER, I.fourier_modes(g))
    raise KeyError(name)


ALL = [f"kpp_cg_p{p}" for p in (1, 2, 3, 4)] + [f"burgers1d_cg_p{p}" for p in (1, 2, 3)] + ["burgers2d_cg_p2"]


def cg_nonflat(d, u, rel=1e-6):
    """Cells whose nodal values are not constant to rounding level."""
    c = O.counts(d)
    n = d["degree"] + 1
    # spread of the nodal values of each cell, via the oracle's Taylor data at corners
    T, _ = O.hermite(d, u)
    spread = np.abs(T[:, :, 1:]).max(axis=(1, 2))
    return spread > rel * max(spread.max(), 1e-300)


@pytest.mark.parametrize("name", ALL)
def test_cg_projection_parity(name):
    d, ic = case(name)
    mesh = cv.Mesh(d)
    got = mesh.project(*ic).cpu().numpy()
    ref = O.project(d, *ic)
    assert got.shape == ref.shape
    # GLL interpolation of the datum in FP32 (reading A25): a few ulps; measured 9.7e-7
    assert rel_err(got, ref) < 2e-6
    mesh.close()


@pytest.mark.parametrize("name", ALL)
def test_cg_full_stage_parity(name):
    d, ic = case(name)
    u = rounded(O.project(d, *ic))
    ref = O.residual(d, u)
    ov, _ = borderline_override(d, ref["gamma"], ref["troubled"])
    mesh = cv.Mesh(d)
    out = mesh.residual_ex(to_gpu(u), troubled_override=torch.from_numpy(ov).cuda())
    mesh.status_check()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    mesh.close()
    mask = cg_nonflat(d, u)
    assert np.abs(got["gamma"] - ref["gamma"])[mask].max() < GAMMA_TOL
    assert rel_err(got["nu"], ref["nu"]) < 1e-6
    dec = (np.abs(ref["gamma"] - d["c_gamma"]) >= 1e-4) & mask
    assert np.array_equal(got["troubled"][dec], ref["troubled"][dec])
    both = (got["troubled"] == 1) & (ref["troubled"] == 1) & mask
    if both.any():
        assert np.abs(got["alpha"][both] - ref["alpha"][both]).max() / np.abs(ref["alpha"][both]).max() < ALPHA_TOL
    assert rel_err(got["dudt"], ref["dudt"]) < RES_TOL


@pytest.mark.parametrize("name", ["kpp_cg_p2", "burgers1d_cg_p3"])
def test_cg_step_and_mass(name):
    d, ic = case(name)
    u = rounded(O.project(d, *ic))
    lam = O.max_wavespeed(d, u)
    h = (d["x1"] - d["x0"]) / d["nx"]
    dt = 0.05 * h / (d["dim"] * d["degree"] * lam)
    ref = O.ssprk3(d, u, dt, 1)
    mesh = cv.Mesh(d)
    ug = to_gpu(u)
    m0 = mesh.mass_total(ug)[0]
    assert abs(m0 - O.mass_total(d, u)[0]) <= 1e-10 * max(1.0, abs(m0))
    mesh.step(ug, dt=dt)
    mesh.status_check()
    assert rel_err(ug.cpu().numpy(), ref) < RES_TOL
    assert abs(mesh.mass_total(ug)[0] - m0) <= 1e-6 * max(1.0, abs(m0))
    mesh.close()


def test_cg_burgers_final_time_matches_oracle_and_paper():
    """1D Burgers CG p = 2, E_h = 128, t = 0.1: the GPU run agrees with the oracle run to
    1e-5 (relative L1 of the difference) and its error against the exact solution is
    the paper's Table tab:bur2 entry 2.32e-6 within 15 %."""
    from tests.test_oracle_convergence import burgers_exact
    d = I.mesh(1, 128, degree=2, system=I.BURGERS, kind=I.CG)
    u0 = rounded(O.project(d, I.IC_SINE_STEP, [1.0, 1.0, 0.0, 2.0]))
    nst = int(math.ceil(0.1 / (0.05 * (1.0 / 128) / 2)))
    dt = 0.1 / nst
    ref = O.ssprk3(d, u0, dt, nst)
    mesh = cv.Mesh(d)
    ug = to_gpu(u0)
    mesh.advance(ug, dt, nst)
    mesh.status_check()
    got = ug.cpu().numpy().astype(np.float64)
    mesh.close()
    assert O.l1_diff(d, got, ref) <= 1e-5 * O.l1_diff(d, ref, np.zeros_like(ref))
    vals, xs, _, ws = O.eval_points(d, got, 0, 8)
    err = float(np.sum(np.abs(vals - burgers_exact(xs, 0.1)) * ws))
    assert abs(math.log(err / 2.32e-6)) <= math.log(1.15), err
