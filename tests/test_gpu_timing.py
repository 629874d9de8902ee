"""Per-launch kernel timing (cvweno_mesh_set_kernel_timing / cvweno_kernel_times): one
duration per launch of a step, in launch order, directly and from a captured graph."""
import pytest
import torch

from paper_2601_16911_gb300 import cvweno as cv
from paper_2601_16911_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,dim,per_stage", [(I.DG, 2, 1), (I.CG, 2, 2), (I.CG, 1, 4)])
def test_kernel_times_direct_and_in_graph(kind, dim, per_stage):
    if dim == 2:
        d, ic = I.kpp(0, n=64, degree=2, kind=kind)
    else:
        d, ic = I.burgers1d_step(0, nx=64, degree=2)
        d = dict(d, kind=kind)
    mesh = cv.Mesh(d)
    u = mesh.project(*ic)
    assert mesh.kernel_times() == []
    mesh.set_kernel_timing(True)
    mesh.advance(u, 1e-3, 1)
    t = mesh.kernel_times()
    assert len(t) == 3 * per_stage and all(x > 0 for x in t)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        mesh.advance(u, 1e-3, 1)
    torch.cuda.current_stream().wait_stream(s)
    with torch.cuda.graph(g):
        mesh.advance(u, 1e-3, 1)
    mesh.set_kernel_timing(False)
    for _ in range(2):
        g.replay()
        t = mesh.kernel_times()
        assert len(t) == 3 * per_stage and all(x > 0 for x in t)
    mesh.status_check()
    mesh.close()
