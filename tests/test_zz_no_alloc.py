"""The SSP-RK3 entry point that allocates nothing, for callers that cannot allocate
device or host memory (code running inside an arena it does not own, or an embedding
that forbids cudaMalloc after start-up).  It is checked through the C ABI against the
mesh-based cvweno_step on the same state, for two calls in a row, and it must reject
states larger than its fixed static scratch.  This file is collected last."""
import numpy as np
import pytest
import torch

from paper_2601_16911_gb300 import cvweno as cv
from paper_2601_16911_gb300 import inputs as I
from tests.gpu_common import RES_TOL

pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = a.double(), b.double()
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("case", ["kpp_q3", "burgers1d_p2"])
def test_static_step_matches_mesh_step_twice(case):
    if case == "kpp_q3":
        d, ic = I.kpp(0, n=64, degree=3)
        dt = (0.3 / 7) * (4.0 / 64) / 2.0
    else:
        d, ic = I.burgers1d_step(0, nx=128, degree=2)
        dt = 0.1 * (1.0 / 128) / 1.5
    mesh = cv.Mesh(d)
    u0 = mesh.project(*ic)
    ua, ub = u0.clone(), u0.clone()
    for _ in range(2):
        mesh.step(ua, dt=dt)
        bits = cv.cvweno_step_static(d, ub, dt, check_status=True)
        assert bits == 0
        torch.cuda.synchronize()
        assert rel(ub, ua) < RES_TOL
    mesh.status_check()
    mesh.close()


def test_static_step_rejects_states_beyond_its_scratch():
    d, _ = I.kpp(0, n=1100, degree=1)  # 1100^2 x 4 floats > 4,194,304
    u = torch.zeros(8, dtype=torch.float32, device="cuda")
    with pytest.raises(cv.CvwenoError) as ei:
        cv.cvweno_step_static(d, u, 1e-3)
    assert ei.value.code == cv.ERR_ARG
