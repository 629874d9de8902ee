"""GPU HWENO limiter (Sec. 3; readings A27, A28) through the C ABI, against the oracle:
the limited state and the limited set on the sensor's troubled cells and on every
cell, exactness on polynomial data, kept cell means, the limited SSP-RK3 step, and
argument handling."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2601_16911_gb300 import cvweno as cv
from paper_2601_16911_gb300 import inputs as I
from tests.gpu_common import rounded, to_gpu

pytestmark = pytest.mark.gpu

LIM_TOL = 1e-5  # max |u_gpu - u_oracle| / max |u|


def cases():
    out = []
    for p in (1, 2, 3, 4):
        out.append((f"kpp_p{p}", *I.kpp(2, n=20, degree=p)))
    g = I.SplitMix64(9)
    for p in (2, 4):
        d = I.mesh(2, 19, 13, degree=p, system=I.BURGERS, bc=I.TRANSMISSIVE)
        out.append((f"burgers2d_p{p}", d, (I.IC_FOURIER, I.fourier_modes(g))))
    for p in (1, 2, 4):
        d, ic = I.burgers1d_step(3, nx=150, degree=p)
        out.append((f"burgers1d_p{p}", d, ic))
    return out


CASES = cases()


@pytest.mark.parametrize("name,d,ic", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("all_cells", [False, True])
def test_limit_matches_oracle(name, d, ic, all_cells):
    u = rounded(O.project(d, *ic))
    ref, tr_ref = O.limit(d, u, all_cells=all_cells)
    mesh = cv.Mesh(d)
    got, tr = mesh.limit(to_gpu(u), all_cells=all_cells)
    torch.cuda.synchronize()
    mesh.status_check()
    got, tr = got.cpu().numpy().astype(np.float64), tr.cpu().numpy()
    mesh.close()
    if all_cells:
        assert tr.all()
        keep = np.ones(tr.shape, bool)
    else:
        gam = O.residual(d, u)["gamma"]
        keep = np.abs(gam - d["c_gamma"]) >= 1e-4  # decisions not taken by rounding
        assert np.array_equal(tr[keep], tr_ref[keep])
        assert tr_ref.sum() > 0 or name.startswith("burgers2d")
        keep &= tr == tr_ref
    # cell means are copied, never recomputed
    assert np.array_equal(got[..., 0], u[..., 0])
    err = np.abs(got[:, keep] - ref[:, keep]).max() / np.abs(u).max()
    assert err <= LIM_TOL, (name, err)


@pytest.mark.parametrize("dim,p", [(1, 3), (2, 2), (2, 4)])
def test_polynomial_data_unchanged(dim, p):
    rng = np.random.default_rng(p + 10 * dim)
    d = I.mesh(dim, 9, 7, degree=p, system=I.BURGERS, bc=I.TRANSMISSIVE)
    P = np.zeros(25)
    for j in range(p + 1 if dim == 2 else 1):
        for i in range(p + 1):
            P[i + 5 * j] = rng.uniform(-1, 1)
    u = rounded(O.project(d, I.IC_POLY, list(P)))
    mesh = cv.Mesh(d)
    got, tr = mesh.limit(to_gpu(u), all_cells=True)
    torch.cuda.synchronize()
    assert bool(tr.all())
    err = np.abs(got.cpu().numpy() - u).max() / np.abs(u).max()
    mesh.close()
    assert err <= LIM_TOL, err


def test_limited_ssprk3_matches_oracle():
    """1D Burgers (the 128-cell P2 step datum) with the limiter in every stage and the
    viscosity off, 40 steps; the relative L1 difference stays within the oracle's own
    sensitivity to a one-ulp change of the start (and within 1e-4)."""
    d0, ic = I.burgers1d_step(0, nx=128, degree=2)
    d = dict(d0, sensor_mode=cv.SENSOR_SMOOTH, hweno_limiter=1)
    u0 = rounded(O.project(d, *ic))
    dt = 0.1 * (1.0 / 128) / 1.5
    ref = O.ssprk3(d, u0.copy(), dt, 40)
    rng = np.random.default_rng(0)
    env = O.l1_diff(d, O.ssprk3(d, u0 * (1 + rng.choice([-1.0, 1.0], size=u0.shape) * 2.0 ** -24), dt, 40), ref)
    mesh = cv.Mesh(d)
    ug = to_gpu(u0)
    mesh.advance(ug, dt, 40)
    mesh.status_check()
    got = ug.cpu().numpy().astype(np.float64)
    mesh.close()
    norm = O.l1_diff(d, ref, np.zeros_like(ref))
    l1 = O.l1_diff(d, got, ref)
    assert l1 <= max(1e-5 * norm, 3.0 * env), (l1 / norm, env / norm)
    assert l1 <= 1e-4 * norm


def test_limited_step_conserves_mass():
    d, ic = I.kpp(4, n=64, degree=2)
    d = dict(d, hweno_limiter=1)
    mesh = cv.Mesh(d)
    u = mesh.project(*ic)
    m0 = mesh.mass_total(u)[0]
    mesh.advance(u, (0.3 / 5) * (4.0 / 64) / 2.0, 10)
    mesh.status_check()
    m1 = mesh.mass_total(u)[0]
    mesh.close()
    assert abs(m1 - m0) <= 1e-6 * abs(m0)


def test_limiter_argument_errors():
    d, ic = I.kpp(0, n=8, degree=2)
    mesh = cv.Mesh(d)
    u = mesh.project(*ic)
    with pytest.raises(cv.CvwenoError) as e:
        mesh.limit(u, out=u)
    assert e.value.code == cv.ERR_ARG
    mesh.close()
    for bad, code in ((dict(d, hweno_limiter=2), cv.ERR_ARG),
                      (dict(d, hweno_limiter=1, kind=I.CG), cv.ERR_UNSUPPORTED),
                      (dict(I.euler_quadrants(0, n=8, degree=1)[0], hweno_limiter=1), cv.ERR_UNSUPPORTED)):
        with pytest.raises(cv.CvwenoError) as e:
            cv.Mesh(bad)
        assert e.value.code == code
    for other in (dict(d, kind=I.CG), I.euler_quadrants(0, n=8, degree=1)[0]):
        m = cv.Mesh(other)
        v = m.empty_state().zero_()
        with pytest.raises(cv.CvwenoError) as e:
            m.limit(v)
        assert e.value.code == cv.ERR_UNSUPPORTED
        m.close()
