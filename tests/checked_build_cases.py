"""Workloads run through the bounds-checked library and through the normal one.

``run_all()`` runs every kernel form of the path on small meshes (ragged against every
tile, periodic and transmissive, 16-byte-aligned and misaligned states) with whatever
library the process loaded, and returns every output as named arrays.
``narrowed_extents()`` (checked library only) narrows a mesh's check extents below its
buffers and returns the status each launch then reports; every access stays within the
real buffers, so nothing faults whatever the checks do.

Run as a module (``python -m tests.checked_build_cases OUT.npz`` with CVWENO_CHECKED=1)
it saves both into OUT.npz for tests/test_gpu_checked_build.py.
"""
import sys

import numpy as np
import torch

from paper_2601_16911_gb300 import cvweno as cv
from paper_2601_16911_gb300 import inputs as I


def misaligned_copy(u):
    """The same values at a data pointer 4 bytes past a 16-byte boundary."""
    buf = torch.empty(u.numel() + 4, dtype=u.dtype, device=u.device)
    v = buf[1:1 + u.numel()].view(u.shape)
    v.copy_(u)
    return v


def _meshes():
    """(name, desc, initial condition, dt, options)."""
    out = []
    for p in (1, 2, 3, 4):
        d, ic = I.kpp(3, n=21, degree=p)
        out.append((f"dg2d-kpp-q{p}", d, ic, 1e-4, {}))
    d = I.mesh(2, 19, 13, degree=3, system=I.BURGERS, bc=I.TRANSMISSIVE)
    out.append(("dg2d-burgers-transmissive-q3", d, (I.IC_FOURIER, I.fourier_modes(I.SplitMix64(7))), 2e-5, {}))
    d, ic = I.kpp(4, n=19, degree=3)
    out.append(("dg2d-kpp-q3-tensor-cores", d, ic, 1e-4, {"tc": True}))
    d, ic = I.kpp(5, n=18, degree=2)
    out.append(("dg2d-kpp-q2-surrogate", d, ic, 1e-4, {"mlp": True}))
    for p in (1, 2, 3):
        d, ic = I.kpp(3, n=17, degree=p, kind=I.CG)
        out.append((f"cg2d-kpp-q{p}", d, ic, 1e-4, {}))
    for p in (1, 2, 3, 4):
        for bc_name, bc in (("periodic", I.PERIODIC), ("transmissive", I.TRANSMISSIVE)):
            d, ic = I.burgers1d_step(5, nx=141, degree=p)
            out.append((f"dg1d-p{p}-{bc_name}", dict(d, bc=(bc,) * 4), ic, 1e-4, {}))
        d, ic = I.burgers1d_step(5, nx=100, degree=p)
        out.append((f"dg1d-p{p}-one-tile", d, ic, 1e-4, {}))
    for p in (2, 3):
        d, ic = I.burgers1d_step(5, nx=141, degree=p)
        out.append((f"cg1d-p{p}", dict(d, kind=I.CG), ic, 1e-4, {}))
    for p in (1, 2, 3):
        d, ic = I.euler_quadrants(2, n=23, degree=p)
        out.append((f"euler-q{p}", d, ic, 1e-4, {"euler": True}))
    return out


def _arr(t):
    return t.detach().cpu().numpy().copy()


def run_all():
    res = {}
    for name, d, ic, dt, opt in _meshes():
        m = cv.Mesh(d)
        if opt.get("tc"):
            m.set_tensor_cores(True)
        net = None
        if opt.get("mlp"):
            net = cv.Mlp(I.mlp_init(0))
            m.set_surrogate(net, 0.5)
        u = m.project(*ic)
        for layout, v in (("aligned", u.clone()), ("misaligned", misaligned_copy(u))):
            key = f"{name}/{layout}"
            res[key + "/residual"] = _arr(m.residual(v))
            m.advance(v, dt, 2)
            res[key + "/steps"] = _arr(v)
        if d["dim"] == 2 and d.get("kind", I.DG) == I.DG and not opt.get("euler"):
            ex = m.residual_ex(u)
            for k, t in ex.items():
                res[f"{name}/ex/{k}"] = _arr(t)
            res[f"{name}/tstar"] = _arr(m.vertex_data(u))
            g, nu = m.sensor(u)
            res[f"{name}/sensor_gamma"], res[f"{name}/sensor_nu"] = _arr(g), _arr(nu)
            lim, troubled = m.limit(u)
            res[f"{name}/limit"], res[f"{name}/limit_troubled"] = _arr(lim), _arr(troubled)
        if opt.get("mlp"):
            f, gf, nrm = m.features(u, with_norm=True)
            res[f"{name}/features"], res[f"{name}/features_gamma"], res[f"{name}/features_norm"] = (
                _arr(f), _arr(gf), _arr(nrm))
        if opt.get("euler"):
            pu, theta = m.positivity(u)
            res[f"{name}/positivity"], res[f"{name}/theta"] = _arr(pu), _arr(theta)
        torch.cuda.synchronize()
        m.status_check()
        m.close()
        if net is not None:
            net.close()
    # batched stages: ragged meshes of every degree
    g = I.SplitMix64(3)
    probs = []
    for k in range(6):
        n = g.randint(5, 17)
        probs.append((I.mesh(2, n, n, degree=1 + k % 4, system=I.BURGERS), (I.IC_FOURIER, I.fourier_modes(g))))
    b = cv.Batch([p[0] for p in probs])
    u = b.empty_state()
    for k, (d, ic) in enumerate(probs):
        m = cv.Mesh(d)
        m.project(*ic, out=b.view(u, k).view(m.state_shape))
        m.close()
    res["batch/residual"] = _arr(b.residual(u))
    b.advance(u, [1e-5] * b.count, 2)
    res["batch/steps"] = _arr(u)
    assert b.status_check() == -1
    b.close()
    # the allocation-free step
    d, ic = I.burgers1d_step(5, nx=141, degree=2)
    m = cv.Mesh(d)
    u = m.project(*ic)
    m.close()
    st = cv.cvweno_step_static(d, u, 1e-4, check_status=True)
    res["step_static/steps"] = _arr(u)
    res["step_static/status"] = np.array([st], np.int32)
    torch.cuda.synchronize()
    return res


def _status_of(fn):
    try:
        fn()
        return cv.OK
    except cv.CvwenoError as e:
        return e.code


def narrowed_extents():
    """Status codes after launches whose check extents are narrowed by one float or one
    cell (the real buffers are untouched and every access stays inside them)."""
    out = {}
    cases = [("dg2d-q2", I.kpp(3, n=21, degree=2)), ("dg2d-q3", I.kpp(3, n=21, degree=3)),
             ("cg2d-q2", I.kpp(3, n=17, degree=2, kind=I.CG)), ("dg1d-p3", I.burgers1d_step(5, nx=141, degree=3)),
             ("euler-q2", I.euler_quadrants(2, n=23, degree=2))]
    for name, (d, ic) in cases:
        m = cv.Mesh(d)
        u = m.project(*ic)
        torch.cuda.synchronize()
        n_state, n_cell = u.numel(), d["nx"] * d.get("ny", 1)
        for tag, ext in (("state", (n_state - 1, n_cell)), ("cells", (n_state, n_cell - 1)),
                         ("restored", (-1, -1))):
            m.set_check_extents(*ext)
            v = u.clone()
            m.advance(v, 1e-5, 1)
            out[f"{name}/{tag}"] = _status_of(m.status_check)
        m.close()
    return out


def main(path):
    assert cv.checked(), "CVWENO_CHECKED=1 must select the checked library"
    lib = cv.load(build_if_missing=True)
    res = run_all()
    res.update({"narrowed/" + k: np.array([v], np.int32) for k, v in narrowed_extents().items()})
    res["library"] = np.array([cv.library_path()])
    del lib
    np.savez(path, **res)


if __name__ == "__main__":
    main(sys.argv[1])
