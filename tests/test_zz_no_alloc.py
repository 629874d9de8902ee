"""The SSP-RK3 entry point that allocates nothing, for callers that cannot allocate
device or host memory (code running inside an arena or memory pool it does not own, or
an embedding that forbids cudaMalloc after start-up).

It is checked through the C ABI against the mesh-based cvweno_step on the same state,
for two calls in a row: both build their tabulations with the library's one builder and
launch the same stage kernels, so the states agree bit for bit, for every (dim, p)
instantiation, on periodic and transmissive meshes and for the Euler system.  It must
also reject states larger than its fixed static scratch, report a non-finite step
through its status word and start the next call with a clean one, and take the
argument codes of cvweno_mesh_create.  This file is collected last."""
import ctypes

import pytest
import torch

from paper_2601_16911_gb300 import cvweno as cv
from paper_2601_16911_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _case(name):
    if name.startswith("d1p"):
        p = int(name[-1])
        d, ic = I.burgers1d_step(0, nx=128 if p == 2 else 75, degree=p)
        return d, ic, 0.1 * (1.0 / d["nx"]) / 1.5 / p
    if name.startswith("d2p"):
        p = int(name[-1])
        d, ic = I.kpp(0, n=48, degree=p)
        return d, ic, (0.3 / (2 * p + 1)) * (4.0 / 48) / 2.0
    if name == "burgers2d_transmissive":
        d = I.mesh(2, 37, 21, degree=3, system=I.BURGERS, bc=I.TRANSMISSIVE)
        return d, (I.IC_FOURIER, I.fourier_modes(I.SplitMix64(5))), 0.3 / 7 * (1.0 / 37) / 8.0
    if name == "euler_q3":
        d, ic = I.euler_quadrants(0, n=40, degree=3)
        return d, ic, (0.3 / 7) * (1.0 / 40) / (2 * 5.6)
    raise KeyError(name)


CASES = [f"d{dim}p{p}" for dim in (1, 2) for p in (1, 2, 3, 4)] + ["burgers2d_transmissive", "euler_q3"]


@pytest.mark.parametrize("case", CASES)
def test_static_step_equals_mesh_step_twice(case):
    d, ic, dt = _case(case)
    mesh = cv.Mesh(d)
    u0 = mesh.project(*ic)
    ua, ub = u0.clone(), u0.clone()
    for _ in range(2):
        mesh.step(ua, dt=dt)
        bits = cv.cvweno_step_static(d, ub, dt, check_status=True)
        assert bits == 0
        torch.cuda.synchronize()
        assert torch.equal(ub, ua)
    mesh.status_check()
    mesh.close()


def _raw_static(d, u, dt):
    st = ctypes.c_int32(-1)
    code = cv.load().cvweno_step_static(ctypes.byref(cv.make_desc(d)), ctypes.c_void_p(u.data_ptr()), float(dt),
                                        ctypes.byref(st), None)
    return code, st.value


def test_static_step_reports_nonfinite_then_starts_clean():
    d, ic, dt = _case("d2p2")
    mesh = cv.Mesh(d)
    good = mesh.project(*ic)
    bad = good.clone()
    bad.view(-1)[1234] = float("nan")
    code, bits = _raw_static(d, bad, dt)
    assert code == cv.ERR_NONFINITE and bits & 1
    code, bits = _raw_static(d, good, dt)  # the status word is reset by every call
    assert code == cv.OK and bits == 0
    mesh.close()


def test_static_step_argument_codes_follow_mesh_create():
    d, _, dt = _case("d2p2")
    u = torch.zeros(8, dtype=torch.float32, device="cuda")
    for bad, code in ((dict(hweno_limiter=2), cv.ERR_ARG), (dict(positivity=2), cv.ERR_ARG),
                      (dict(nx=(1 << 24) + 1, ny=1), cv.ERR_ARG), (dict(degree=5), cv.ERR_UNSUPPORTED),
                      (dict(hweno_limiter=1), cv.ERR_UNSUPPORTED), (dict(kind=I.CG), cv.ERR_UNSUPPORTED)):
        with pytest.raises(cv.CvwenoError) as ei:
            cv.cvweno_step_static(dict(d, **bad), u, dt)
        assert ei.value.code == code, bad


def test_static_step_rejects_states_beyond_its_scratch():
    d, _ = I.kpp(0, n=1100, degree=1)  # 1100^2 x 4 floats > 4,194,304
    u = torch.zeros(8, dtype=torch.float32, device="cuda")
    with pytest.raises(cv.CvwenoError) as ei:
        cv.cvweno_step_static(d, u, 1e-3)
    assert ei.value.code == cv.ERR_ARG
