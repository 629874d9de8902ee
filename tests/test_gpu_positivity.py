"""GPU positivity limiter for the Euler equations (readings P1-P4) against the oracle:
the limited coefficients and theta on random states of every degree, admissible states
untouched, an inadmissible mean reported, and the limited SSP-RK3 step through a near
vacuum that the plain scheme does not survive."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2601_16911_gb300 import cvweno as cv
from paper_2601_16911_gb300 import inputs as I
from tests.gpu_common import rounded, to_gpu
from tests.test_oracle_positivity import random_state

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("amp", [0.05, 1.6])
def test_positivity_matches_oracle(p, amp):
    d = I.mesh(2, 19, 11, degree=p, system=I.EULER, bc=I.TRANSMISSIVE)
    u = rounded(random_state(d, np.random.default_rng(10 * p), amp))
    ref, th_ref, code = O.positivity(d, u)
    assert code == 0
    mesh = cv.Mesh(d)
    out, th = mesh.positivity(to_gpu(u))
    torch.cuda.synchronize()
    mesh.status_check()
    out, th = out.cpu().numpy().astype(np.float64), th.cpu().numpy().astype(np.float64)
    mesh.close()
    # theta: FP32 bisection (40 halvings) on FP32 pressures against the FP64 root (P3);
    # the 1e-5 bar of the other stages, measured at most 2.7e-7 on a GB300
    assert np.abs(th - th_ref).max() <= 1e-5
    if amp < 0.1:
        assert np.array_equal(out, u) and np.all(th == 1.0)
    else:
        assert (th_ref < 1).sum() > 10
    assert np.array_equal(out[:, :, 0], u[:, :, 0])
    err = np.abs(out - ref).max(axis=2) / np.abs(u).max(axis=2)
    assert err.max() <= 1e-5, err.max()  # limited modes, per cell relative: measured at most 2.7e-7


def test_in_place_and_inadmissible_mean():
    d = I.mesh(2, 6, 5, degree=2, system=I.EULER, bc=I.TRANSMISSIVE)
    u = rounded(random_state(d, np.random.default_rng(3), 1.6))
    u[0, 7, 0] = -0.5
    mesh = cv.Mesh(d)
    ug = to_gpu(u)
    ref = ug.clone()
    mesh.positivity(ug, out=ug)  # in place
    with pytest.raises(cv.CvwenoError) as e:
        mesh.status_check()
    assert e.value.code == cv.ERR_POSITIVITY
    got = ug.cpu().numpy()
    assert np.array_equal(got[:, 7], ref.cpu().numpy()[:, 7])  # the bad cell is copied
    mesh.close()


def test_limited_step_through_a_near_vacuum():
    d = I.mesh(2, 12, 4, degree=2, system=I.EULER, bc=I.TRANSMISSIVE, domain=(-1, 1, 0, 0.5))
    prm = [0.0, 0.25, 1.0, -3.0, 0.0, 0.01, 1.0, 3.0, 0.0, 0.01, 1.0, -3.0, 0.0, 0.01, 1.0, 3.0, 0.0, 0.01]
    u0 = rounded(O.project(d, I.IC_QUADRANTS, prm))
    dt = 0.05 * (2.0 / 12) / (3.0 + np.sqrt(1.4 * 0.01)) / 5
    plain = cv.Mesh(d)
    ug = to_gpu(u0)
    plain.advance(ug, dt, 10)
    with pytest.raises(cv.CvwenoError) as e:
        plain.status_check()
    assert e.value.code in (cv.ERR_POSITIVITY, cv.ERR_NONFINITE)
    plain.close()
    dp = dict(d, positivity=1)
    ref = O.ssprk3(dp, u0.copy(), dt, 40)
    mesh = cv.Mesh(dp)
    ug = to_gpu(u0)
    mesh.advance(ug, dt, 40)
    mesh.status_check()
    got = ug.cpu().numpy().astype(np.float64)
    mesh.close()
    norm = O.l1_diff(dp, ref, np.zeros_like(ref))
    # 40 limited steps through a near vacuum: every stage's theta (a root of a concave
    # pressure along a segment) is re-decided on FP32 data, so the run follows the oracle
    # to the sensitivity of those roots rather than to the per-stage 1e-5
    assert O.l1_diff(dp, got, ref) <= 1e-4 * norm


def test_positivity_argument_errors():
    d, _ = I.kpp(0, n=8, degree=2)
    m = cv.Mesh(d)
    with pytest.raises(cv.CvwenoError) as e:
        m.positivity(m.empty_state().zero_())
    assert e.value.code == cv.ERR_UNSUPPORTED
    m.close()
    for bad, code in ((dict(d, positivity=1), cv.ERR_UNSUPPORTED),
                      (dict(I.euler_quadrants(0, n=8, degree=1)[0], positivity=3), cv.ERR_ARG)):
        with pytest.raises(cv.CvwenoError) as e:
            cv.Mesh(bad)
        assert e.value.code == code
