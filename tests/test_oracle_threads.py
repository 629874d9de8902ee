"""The oracle's OpenMP loops (used only by the timed CPU baseline) change no result:
every cell, vertex and face row is computed and accumulated as with one thread, so the
states after two SSP-RK3 steps are bitwise equal for every thread count."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2601_16911_gb300 import inputs as I


def _cases():
    for kind in (I.DG, I.CG):
        for p in (1, 3):
            yield I.kpp(1, n=12, degree=p, kind=kind) + (2e-3,)
    yield I.euler_quadrants(1, n=10, degree=2) + (2e-4,)
    d = I.mesh(2, 9, 7, degree=2, system=I.BURGERS, bc=I.TRANSMISSIVE)
    yield d, (I.IC_FOURIER, I.fourier_modes(I.SplitMix64(2))), 1e-3
    yield I.burgers1d_step(3, nx=40, degree=3) + (1e-3,)


@pytest.mark.parametrize("threads", [2, 5])
def test_results_independent_of_thread_count(threads):
    try:
        ref = []
        O.set_threads(1)
        for d, ic, dt in _cases():
            u = O.project(d, *ic)
            ref.append((O.ssprk3(d, u, dt, 2), O.residual(d, u)))
        if O.set_threads(threads) == 1:
            pytest.skip("oracle built without OpenMP")
        for (d, ic, dt), (s_ref, r_ref) in zip(_cases(), ref):
            u = O.project(d, *ic)
            assert np.array_equal(O.ssprk3(d, u, dt, 2), s_ref)
            r = O.residual(d, u)
            for k in ("dudt", "gamma", "nu", "alpha", "troubled"):
                assert np.array_equal(r[k], r_ref[k]), k
    finally:
        O.set_threads(1)
