"""Batched persistent stages (many independent 2D Burgers DG meshes of uneven size and
degree, one launch per RK stage): parity with the oracle per instance, agreement with
the single-mesh path, every launch shape, graph replay, autotuning, status and
argument handling, and the full 64-instance workload on sampled windows."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2601_16911_gb300 import cvweno as cv
from paper_2601_16911_gb300 import inputs as I
from tests.gpu_common import RES_TOL, rel_err, rounded
from tests.test_gpu_e2e import window

pytestmark = pytest.mark.gpu

PLANS = [dict(schedule=s, tile=t, dynamic=dy, ctas_per_sm=c)
         for s in (cv.BATCH_FUSED, cv.BATCH_GROUPED) for t in (0, 1) for dy in (0, 1) for c in (0, 1)]


def small_batch(seed=3, count=9):
    """Ragged meshes (N not a multiple of either tile edge) covering every degree."""
    g = I.SplitMix64(seed)
    out = []
    for k in range(count):
        n = g.randint(5, 17)
        p = 1 + k % 4
        out.append((I.mesh(2, n, n, degree=p, system=I.BURGERS), (I.IC_FOURIER, I.fourier_modes(g))))
    return out


def project_batch(b, probs):
    u = b.empty_state()
    for k, (d, ic) in enumerate(probs):
        m = cv.Mesh(d)
        m.project(*ic, out=b.view(u, k).view(m.state_shape))
        m.close()
    torch.cuda.synchronize()
    return u


def state_of(b, u, k, d):
    nd = (d["degree"] + 1) ** 2
    return b.view(u, k).cpu().numpy().astype(np.float64).reshape(1, d["nx"] * d["ny"], nd)


def stable_dt(d):
    """Inside both the hyperbolic limit h / (lambda (2p+1)) and the explicit limit of
    the artificial viscosity nu_e = lambda h / (2p), which for p = 4 is the stricter
    (about h / (lambda p^3)); |u| < 4, lambda <= 2 |u|."""
    p = d["degree"]
    return 0.1 * (1.0 / d["nx"]) / (8.0 * (2 * p + 1) * p)


def decided_by_rounding(d, ref, width=1e-4):
    """Cells whose oracle sensor sits within `width` of the SC cutoff."""
    return np.abs(ref["gamma"] - d["c_gamma"]) < width


def test_batch_residual_matches_oracle_every_plan():
    probs = small_batch()
    b = cv.Batch([d for d, _ in probs])
    u = project_batch(b, probs)
    refs = []
    for k, (d, _) in enumerate(probs):
        uk = state_of(b, u, k, d)
        refs.append((O.residual(d, rounded(uk)), uk))
    for plan in PLANS:
        b.set_plan(**plan)
        r = b.residual(u)
        assert b.status_check() == -1
        for k, (d, _) in enumerate(probs):
            ref, uk = refs[k]
            got = state_of(b, r, k, d)
            keep = ~decided_by_rounding(d, ref)
            assert keep.sum() >= 0.9 * keep.size
            err = rel_err(got[:, keep, :], ref["dudt"][:, keep, :])
            assert err <= RES_TOL, (plan, k, d["nx"], d["degree"], err)
    b.close()


def test_batch_equals_single_mesh_path():
    """The batch runs the single-mesh stage body per tile: same results as
    cvweno_residual on each mesh (to the last bit, as the arithmetic is the same)."""
    probs = small_batch(seed=11, count=8)
    b = cv.Batch([d for d, _ in probs])
    u = project_batch(b, probs)
    for plan in PLANS[::3]:
        b.set_plan(**plan)
        r = b.residual(u)
        for k, (d, _) in enumerate(probs):
            m = cv.Mesh(d)
            single = m.residual(b.view(u, k).view(m.state_shape).clone())
            torch.cuda.synchronize()
            diff = (b.view(r, k) - single.reshape(-1)).abs().max().item()
            scale = single.abs().max().item()
            # the batch runs the single-mesh tile code on every tile: bit for bit
            assert diff == 0.0, (plan, k, diff, scale)
            m.close()
    b.close()


@pytest.mark.parametrize("use_graph", [0, 1])
def test_batch_advance_matches_oracle_steps(use_graph):
    """Three SSP-RK3 steps of every instance, each with its own dt, against the
    oracle's steps on the same FP32 start; relative L1 of the difference <= 1e-5."""
    probs = small_batch(seed=5, count=8)
    b = cv.Batch([d for d, _ in probs])
    b.set_plan(use_graph=use_graph)
    u = project_batch(b, probs)
    u0 = [rounded(state_of(b, u, k, d)) for k, (d, _) in enumerate(probs)]
    dts = [stable_dt(d) for d, _ in probs]
    b.advance(u, dts, 3)
    assert b.status_check() == -1
    for k, (d, _) in enumerate(probs):
        ref = O.ssprk3(d, u0[k], dts[k], 3)
        got = state_of(b, u, k, d)
        err = O.l1_diff(d, got, ref) / O.l1_diff(d, ref, np.zeros_like(ref))
        assert err <= 1e-5, (k, d["nx"], d["degree"], err)
    b.close()


def test_batch_advance_equals_per_mesh_advance_and_replays():
    """Graph replay over two calls (6 steps) equals the per-mesh path, and changing a
    step size between calls takes effect (the graph reads its arguments from memory)."""
    probs = small_batch(seed=7, count=6)
    b = cv.Batch([d for d, _ in probs])
    u = project_batch(b, probs)
    ref = u.clone()
    dts = [stable_dt(d) for d, _ in probs]
    b.advance(u, dts, 2)
    dts2 = [x * 0.5 for x in dts]
    b.advance(u, dts2, 4)
    for k, (d, _) in enumerate(probs):
        m = cv.Mesh(d)
        uk = b.view(ref, k).view(m.state_shape)
        m.advance(uk, dts[k], 2)
        m.advance(uk, dts2[k], 4)
        m.close()
    torch.cuda.synchronize()
    assert b.status_check() == -1
    diff = (u - ref).abs().max().item()
    assert diff == 0.0, diff  # the same tile code and RK epilogue: bit for bit
    b.close()


def test_batch_autotune_picks_a_valid_plan_and_keeps_results():
    probs = small_batch(seed=13, count=12)
    b = cv.Batch([d for d, _ in probs])
    u = project_batch(b, probs)
    before = b.residual(u).clone()
    u_copy = u.clone()
    best = b.autotune(u)
    assert torch.equal(u, u_copy)  # autotuning reads u only
    assert best["ms"] > 0.0 and best["schedule"] in (0, 1) and best["tile"] in (0, 1)
    assert b.plan()["schedule"] == best["schedule"] and b.plan()["tile"] == best["tile"]
    after = b.residual(u)
    diff = (after - before).abs().max().item()
    assert diff == 0.0  # every plan runs the same per-tile arithmetic
    b.close()


def test_batch_status_names_the_bad_instance():
    probs = small_batch(seed=17, count=5)
    b = cv.Batch([d for d, _ in probs])
    u = project_batch(b, probs)
    b.view(u, 3)[7] = float("nan")
    b.residual(u)
    with pytest.raises(cv.CvwenoError) as e:
        b.status_check()
    assert e.value.code == cv.ERR_NONFINITE
    # the words are cleared by the check; a clean state passes again
    u2 = project_batch(b, probs)
    b.residual(u2)
    assert b.status_check() == -1
    b.close()


def test_batch_first_bad_index():
    probs = small_batch(seed=19, count=5)
    b = cv.Batch([d for d, _ in probs])
    u = project_batch(b, probs)
    b.view(u, 2)[0] = float("inf")
    b.residual(u)
    import ctypes
    bad = ctypes.c_int(-7)
    code = cv.load().cvweno_batch_status_check(b.handle, ctypes.byref(bad), cv._stream(None))
    assert code == cv.ERR_NONFINITE and bad.value == 2
    b.close()


def test_batch_argument_errors():
    d = I.mesh(2, 8, 8, degree=2, system=I.BURGERS)
    with pytest.raises(cv.CvwenoError) as e:
        cv.Batch([d, dict(d, ny=9)])  # non-square cells
    assert e.value.code == cv.ERR_ARG
    with pytest.raises(cv.CvwenoError) as e:
        cv.Batch([d, dict(d, system=I.KPP)])
    assert e.value.code == cv.ERR_UNSUPPORTED
    with pytest.raises(cv.CvwenoError) as e:
        cv.Batch([dict(d, kind=I.CG)])
    assert e.value.code == cv.ERR_UNSUPPORTED
    with pytest.raises(cv.CvwenoError) as e:
        cv.Batch([dict(d, degree=5)])
    assert e.value.code == cv.ERR_UNSUPPORTED
    b = cv.Batch([d, dict(d, nx=12, ny=12, degree=4)])
    u = b.empty_state().zero_()
    with pytest.raises(cv.CvwenoError) as e:
        b.advance(u, [1e-3, 0.0], 1)
    assert e.value.code == cv.ERR_ARG
    for bad in (dict(schedule=2), dict(tile=2), dict(dynamic=3), dict(ctas_per_sm=-1), dict(use_graph=2)):
        with pytest.raises(cv.CvwenoError) as e:
            b.set_plan(**bad)
        assert e.value.code == cv.ERR_ARG
    with pytest.raises(cv.CvwenoError) as e:
        b.residual(u, out=u)
    assert e.value.code == cv.ERR_ARG
    b.close()


def test_batch_zero_state_is_steady():
    """u = 0 is a steady state of Burgers: every instance stays exactly zero."""
    probs = small_batch(seed=23, count=6)
    b = cv.Batch([d for d, _ in probs])
    u = b.empty_state().zero_()
    b.advance(u, [1e-3] * len(probs), 3)
    assert b.status_check() == -1
    assert float(u.abs().max()) == 0.0
    b.close()


def test_batch_full_workload_sampled_windows():
    """The 64-instance workload (N in 64..512, p in 1..4, Fourier data), one residual
    pass of the autotuned batch: equal to the single-mesh path on every instance, and
    equal to the oracle on sampled 6x6 windows of several instances."""
    probs = I.burgers2d_batch(0)
    b = cv.Batch([d for d, _ in probs])
    u = project_batch(b, probs)
    b.autotune(u)
    r = b.residual(u)
    assert b.status_check() == -1
    for k, (d, _) in enumerate(probs):
        m = cv.Mesh(d)
        single = m.residual(b.view(u, k).view(m.state_shape).clone())
        torch.cuda.synchronize()
        diff = (b.view(r, k) - single.reshape(-1)).abs().max().item()
        assert diff == 0.0, (k, diff)
        m.close()
    seen = set()
    for k, (d, _) in enumerate(probs):
        if d["degree"] in seen:
            continue
        seen.add(d["degree"])
        n = d["nx"]
        uk = state_of(b, u, k, d)
        rk = state_of(b, r, k, d)
        scale = np.abs(rk).max()
        for (i0, j0) in [(0, 0), (n - 6, n - 6), (n // 2, n // 3)]:
            sub, us, inner, sub_inner = window(d, uk, i0, j0, 6, 6)
            ref = O.residual(sub, us)
            keep = ~decided_by_rounding(d, ref)[sub_inner]
            err = np.abs(rk[:, inner, :][:, keep] - ref["dudt"][:, sub_inner, :][:, keep]).max() / scale
            assert err < RES_TOL, (k, n, d["degree"], i0, j0, err)
    assert seen == {1, 2, 3, 4}
    b.close()
