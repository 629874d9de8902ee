"""The tensor-core form of the 2D Q3 stage kernel (cvweno_mesh_set_tensor_cores).

Stage (c)'s corner products -- the four vertex candidates mapped into the cell's
semi-norm coordinates (Sec. 3.2 eq. finalweno, semi-norm of Sec. 2.2 eq. snorm) -- run
on tcgen05 in split TF32 over 8 x 16 tiles.  The same bars as the CUDA-core form:
  * every stage output against the FP64 oracle (tests/gpu_common.py tolerances;
    residual max relative error 1e-5), on meshes ragged against the 8 x 16 tile,
    periodic and transmissive, from one cell to several tiles, for every scalar law;
  * SSP-RK3 steps against the oracle;
  * against the CUDA-core form on the same input: the vertex data bit for bit (stages
    a-b are the same code), gamma and dudt to FP32 rounding;
  * the sensor-only and limiter modes, which read the same corner products.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2601_16911_gb300 import cvweno as cv
from paper_2601_16911_gb300 import inputs as I
from tests.gpu_common import ALPHA_TOL, GAMMA_TOL, RES_TOL, nonflat_mask, rel_err, residual_pair, rounded, to_gpu

pytestmark = pytest.mark.gpu


def case(name):
    if name == "kpp20":
        return I.kpp(2, n=20, degree=3)
    if name == "kpp_ragged":
        d, ic = I.kpp(7, n=16, degree=3)
        return dict(d, nx=13, ny=37), ic
    if name == "burgers_t":
        g = I.SplitMix64(3)
        d = I.mesh(2, 24, 19, degree=3, system=I.BURGERS, bc=I.TRANSMISSIVE)
        return d, (I.IC_FOURIER, I.fourier_modes(g))
    if name == "linadv":
        d = I.mesh(2, 17, 9, degree=3, system=I.LINADV, adv_vx=0.7, adv_vy=-0.4)
        return d, (I.IC_CIRCLE, [0.4, 0.5, 0.3, 2.0, -1.0])
    if name.startswith("tiny"):
        nx, ny, bc = {"tiny11p": (1, 1, I.PERIODIC), "tiny23t": (2, 3, I.TRANSMISSIVE),
                      "tiny9x17p": (9, 17, I.PERIODIC)}[name]
        d = I.mesh(2, nx, ny, degree=3, system=I.KPP, bc=bc, domain=(-2, 2, -2, 2), lambda_const=1.0)
        return d, ("random", np.random.default_rng(nx * 100 + ny))
    raise KeyError(name)


def initial(d, ic):
    if ic[0] == "random":
        return ic[1].standard_normal(O.state_shape(d)) * 0.5
    return O.project(d, *ic)


def tc_mesh(d):
    m = cv.Mesh(d)
    m.set_tensor_cores(True)
    return m


CASES = ["kpp20", "kpp_ragged", "burgers_t", "linadv", "tiny11p", "tiny23t", "tiny9x17p"]


@pytest.mark.parametrize("name", CASES)
def test_full_stage_parity_tensor_cores(name):
    d, ic = case(name)
    mesh = tc_mesh(d)
    u, ref, got, _ = residual_pair(d, initial(d, ic), mesh=mesh)
    mesh.close()
    mask = nonflat_mask(u)
    gerr = np.abs(got["gamma"] - ref["gamma"])[mask]
    assert gerr.size == 0 or gerr.max() < GAMMA_TOL, gerr.max()
    assert rel_err(got["nu"], ref["nu"]) < 1e-6
    dec = np.abs(ref["gamma"] - d["c_gamma"]) >= 1e-4
    assert np.array_equal(got["troubled"][dec & mask], ref["troubled"][dec & mask])
    both = (got["troubled"] == 1) & (ref["troubled"] == 1) & mask
    if both.any():
        aerr = np.abs(got["alpha"][both] - ref["alpha"][both]).max() / np.abs(ref["alpha"][both]).max()
        assert aerr < ALPHA_TOL, aerr
    assert rel_err(got["dudt"], ref["dudt"]) < RES_TOL


@pytest.mark.parametrize("name", ["kpp20", "kpp_ragged", "burgers_t"])
def test_tensor_cores_against_cuda_cores(name):
    d, ic = case(name)
    u = to_gpu(rounded(initial(d, ic)))
    plain, tcm = cv.Mesh(d), tc_mesh(d)
    assert torch.equal(plain.vertex_data(u), tcm.vertex_data(u))
    a, b = plain.residual_ex(u), tcm.residual_ex(u)
    ga, nu_a = plain.sensor(u)
    gb, nu_b = tcm.sensor(u)
    torch.cuda.synchronize()
    plain.status_check()
    tcm.status_check()
    mask = nonflat_mask(u.cpu().numpy().astype(np.float64))
    assert (a["gamma"] - b["gamma"]).abs().cpu().numpy()[mask].max() < 1e-5
    assert torch.equal(gb, b["gamma"]) and torch.equal(nu_b, nu_a)
    assert rel_err(b["dudt"].cpu().numpy(), a["dudt"].cpu().numpy()) < 1e-6
    plain.close()
    tcm.close()


@pytest.mark.parametrize("name", ["kpp20", "burgers_t"])
def test_ssprk3_steps_tensor_cores(name):
    d, ic = case(name)
    u = rounded(initial(d, ic))
    lam = O.max_wavespeed(d, u)
    h = min((d["x1"] - d["x0"]) / d["nx"], (d["y1"] - d["y0"]) / d["ny"])
    dt = 0.1 * h / (d["dim"] * lam)
    ref = O.ssprk3(d, u, dt, 2)
    mesh = tc_mesh(d)
    ug = to_gpu(u)
    mesh.advance(ug, dt, 2)
    mesh.status_check()
    assert rel_err(ug.cpu().numpy(), ref) < RES_TOL
    mesh.close()


def test_limiter_tensor_cores():
    d, ic = case("kpp20")
    u = to_gpu(rounded(initial(d, ic)))
    plain, tcm = cv.Mesh(d), tc_mesh(d)
    la, ta = plain.limit(u)
    lb, tb = tcm.limit(u)
    torch.cuda.synchronize()
    # the limited set agrees except where gamma sits at C_gamma to rounding
    assert (ta != tb).sum().item() <= 2
    same = (ta == tb).cpu().numpy()
    diff = np.abs(la.cpu().numpy()[0] - lb.cpu().numpy()[0])[same].max()
    assert diff <= 1e-5 * np.abs(la.cpu().numpy()).max()
    plain.close()
    tcm.close()


def test_setter_rejects_other_meshes():
    for d in (I.kpp(0, n=8, degree=2)[0], I.kpp(0, n=8, degree=3, kind=I.CG)[0],
              I.euler_quadrants(0, n=8, degree=3)[0], I.burgers1d_step(0, nx=16, degree=3)[0]):
        m = cv.Mesh(d)
        with pytest.raises(cv.CvwenoError) as e:
            m.set_tensor_cores(True)
        assert e.value.code == cv.ERR_UNSUPPORTED
        m.set_tensor_cores(False)
        m.close()
    m = cv.Mesh(I.kpp(0, n=8, degree=3)[0])
    with pytest.raises(cv.CvwenoError) as e:
        load = cv.load()
        code = load.cvweno_mesh_set_tensor_cores(m.handle, 2)
        cv._check(code, "cvweno_mesh_set_tensor_cores")
    assert e.value.code == cv.ERR_ARG
    m.close()
