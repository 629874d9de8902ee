"""Whole SSP-RK3 steps of a one-tile 1D mesh in one launch.

A 1D scalar DG mesh of at most 128 cells is one CTA, so cvweno_step and cvweno_advance
run all its stages (and all the steps of one advance call) in one kernel, with block
barriers in place of the launch boundaries. With kernel timing on, the mesh runs one
launch per stage instead. Both run the same stage code on the same block, so their
results must agree bit for bit. The cases cover P1-P4, Burgers and linear advection,
periodic and transmissive boundaries, a 3-cell mesh, a ragged 37-cell tile and a full
128-cell tile. They also check that one advance of several steps gives the same bits as
the same steps taken one call at a time.
"""
import pytest
import torch

from paper_2601_16911_gb300 import cvweno as cv
from paper_2601_16911_gb300 import inputs as I

pytestmark = pytest.mark.gpu

CASES = [(p, system, bc, nx)
         for p in (1, 2, 3, 4)
         for system, bc in ((I.BURGERS, I.PERIODIC), (I.BURGERS, I.TRANSMISSIVE), (I.LINADV, I.PERIODIC))
         for nx in (3, 37, 128)]


def make(p, system, bc, nx):
    d = I.mesh(1, nx, degree=p, system=system, bc=bc)
    ic = (I.IC_SINE_STEP, [1.0, 1.0, 0.5, 0.43])
    dt = 0.05 * (1.0 / nx) / 1.5  # CFL 0.05: inside the SSP-RK3 DG limit at p = 4 (about 0.09)
    return d, ic, dt


@pytest.mark.parametrize("p,system,bc,nx", CASES,
                         ids=["p%d-%s-%s-n%d" % (p, "burgers" if s == I.BURGERS else "linadv",
                                                 "per" if b == I.PERIODIC else "tra", n) for p, s, b, n in CASES])
def test_one_launch_steps_match_stage_launches(p, system, bc, nx):
    d, ic, dt = make(p, system, bc, nx)
    fused = cv.Mesh(d)
    staged = cv.Mesh(d)
    staged.set_kernel_timing(True)  # one launch per stage
    u0 = fused.project(*ic)
    ua, ub, uc = u0.clone(), u0.clone(), u0.clone()
    fused.advance(ua, dt, 6)
    staged.advance(ub, dt, 6)
    for _ in range(6):
        fused.step(uc, dt=dt)
    torch.cuda.synchronize()
    assert len(staged.kernel_times()) == 3  # the staged mesh did launch stage by stage
    assert torch.equal(ua, ub)
    assert torch.equal(ua, uc)
    assert not torch.equal(ua, u0)
    fused.status_check()
    staged.status_check()
    fused.close()
    staged.close()


def test_one_launch_steps_leave_larger_meshes_to_stage_launches():
    # 129 cells are two tiles: the step runs as stage launches and still agrees with a
    # mesh timed stage by stage
    d, ic, dt = make(2, I.BURGERS, I.PERIODIC, 129)
    a, b = cv.Mesh(d), cv.Mesh(d)
    b.set_kernel_timing(True)
    u0 = a.project(*ic)
    ua, ub = u0.clone(), u0.clone()
    a.advance(ua, dt, 3)
    b.advance(ub, dt, 3)
    torch.cuda.synchronize()
    assert torch.equal(ua, ub)
    a.close()
    b.close()
