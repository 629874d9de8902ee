"""Tile loads on 16-byte-aligned and misaligned states.

The stage kernels copy an aligned state in 16-byte pieces: whole cells where a cell is a
multiple of 4 floats (Q1, Q3), runs of halo cells by rows otherwise (Q2, Q4, 1D), nodal
rows for CG. A state that is not 16-byte aligned goes float by float. Both paths must
give the same bits. The cases cover DG Q1-Q4 and CG Q1-Q3 in 2D, DG P1-P4 and CG in 1D,
periodic and transmissive, and the Euler kernel at Q1-Q3 (two variables staged at a time
where cells are whole chunks). Every mesh size is a non-multiple of the tile, so there
are ragged tiles and wrapped halo columns. Each case checks the residual and two full
SSP-RK3 steps, so u_n of stages 2 and 3 is read in both layouts.
"""
import pytest
import torch

from paper_2601_16911_gb300 import cvweno as cv
from paper_2601_16911_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def misaligned_copy(u):
    """The same values at a data pointer 4 bytes past a 16-byte boundary."""
    buf = torch.empty(u.numel() + 4, dtype=u.dtype, device=u.device)
    v = buf[1:1 + u.numel()].view(u.shape)
    v.copy_(u)
    assert v.data_ptr() % 16 == 4
    return v


def kpp(p, kind):
    return I.kpp(3, n=37, degree=p, kind=kind), 1e-4


def burgers2d_transmissive(p):
    d = I.mesh(2, 21, 19, degree=p, system=I.BURGERS, bc=I.TRANSMISSIVE)
    return (d, (I.IC_FOURIER, I.fourier_modes(I.SplitMix64(7)))), 2e-5


def burgers1d(p, bc, kind=I.DG):
    d, ic = I.burgers1d_step(5, nx=141, degree=p)
    return (dict(d, bc=(bc,) * 4, kind=kind), ic), 1e-4


CASES = ([("dg2d-kpp-q%d" % p, lambda p=p: kpp(p, I.DG)) for p in (1, 2, 3, 4)]
         + [("cg2d-kpp-q%d" % p, lambda p=p: kpp(p, I.CG)) for p in (1, 2, 3)]
         + [("dg2d-burgers-transmissive-q%d" % p, lambda p=p: burgers2d_transmissive(p)) for p in (2, 3)]
         + [("dg1d-p%d-%s" % (p, name), lambda p=p, bc=bc: burgers1d(p, bc))
            for p in (1, 2, 3, 4) for name, bc in (("periodic", I.PERIODIC), ("transmissive", I.TRANSMISSIVE))]
         + [("cg1d-p%d" % p, lambda p=p: burgers1d(p, I.PERIODIC, I.CG)) for p in (2, 3)]
         + [("euler-q%d" % p, lambda p=p: (I.euler_quadrants(2, n=37, degree=p), 1e-4)) for p in (1, 2, 3)])


@pytest.mark.parametrize("make", [c[1] for c in CASES], ids=[c[0] for c in CASES])
def test_aligned_and_misaligned_states_agree(make):
    (d, ic), dt = make()
    m = cv.Mesh(d)
    u = m.project(*ic)
    ua = u.clone()
    um = misaligned_copy(u)
    ra = m.residual(ua)
    rm = m.residual(um)
    torch.cuda.synchronize()
    m.status_check()
    assert torch.equal(ra, rm)
    m.advance(ua, dt, 2)
    m.advance(um, dt, 2)
    torch.cuda.synchronize()
    m.status_check()
    assert torch.equal(ua, um)
    assert not torch.equal(ua, u)  # the steps did something
    m.close()
