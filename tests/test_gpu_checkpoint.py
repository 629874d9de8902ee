"""Resume from a checkpoint reproduces the uninterrupted run bit for bit (DG, CG and
Euler meshes): n steps straight through against k steps, save, a fresh mesh from the
file, and n - k more steps."""
import pytest
import torch

from paper_2601_16911_gb300 import checkpoint as ck
from paper_2601_16911_gb300 import cvweno as cv
from paper_2601_16911_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("case", ["kpp_dg_q3", "kpp_cg_q2", "euler_q2", "burgers1d_p3"])
def test_resume_equals_uninterrupted_run(tmp_path, case):
    d, ic = {"kpp_dg_q3": lambda: I.kpp(2, n=24, degree=3),
             "kpp_cg_q2": lambda: I.kpp(2, n=20, degree=2, kind=I.CG),
             "euler_q2": lambda: I.euler_quadrants(1, n=24, degree=2),
             "burgers1d_p3": lambda: I.burgers1d_step(4, nx=90, degree=3)}[case]()
    dt, n, k = 2e-4, 6, 2
    m = cv.Mesh(d)
    u0 = m.project(*ic)
    straight = u0.clone()
    m.advance(straight, dt, n)
    part = u0.clone()
    m.advance(part, dt, k)
    torch.cuda.synchronize()
    m.status_check()
    path = str(tmp_path / "ck.npz")
    ck.save(path, d, part, t=k * dt, step=k)
    m.close()
    m2, u, t, step = ck.resume(path)
    assert step == k and t == k * dt
    m2.advance(u, dt, n - k)
    torch.cuda.synchronize()
    m2.status_check()
    assert torch.equal(u, straight)
    m2.close()
