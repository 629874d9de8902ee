"""End-to-end pins of the oracle: design order of accuracy on smooth data.

Sec. 5.2 states that all schemes (CG and, in the remark on linear advection, DG)
converge at the optimal rate p+1 on smooth solutions.  The 1D Burgers solution with
u0 = sin(2 pi x) is smooth up to t = 1/(2 pi); its exact value at t = 0.1 follows
from the characteristics u = sin(2 pi (x - u t)).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2601_16911_gb300 import inputs as I


def burgers_exact(x, t):
    u = np.sin(2 * np.pi * x)
    for _ in range(100):
        g = u - np.sin(2 * np.pi * (x - u * t))
        dg = 1 + 2 * np.pi * t * np.cos(2 * np.pi * (x - u * t))
        u = u - g / dg
    return u


def burgers_l1_error(nx, p, t_end=0.1, cfl=0.1):
    d, ic = I.burgers1d_sine(nx, p)
    u = O.project(d, *ic)
    dx = 1.0 / nx
    nsteps = int(math.ceil(t_end / (cfl * dx)))
    dt = t_end / nsteps
    u = O.ssprk3(d, u, dt, nsteps)
    vals, xs, _, ws = O.eval_points(d, u, 0, 8)
    return float(np.sum(np.abs(vals - burgers_exact(xs, t_end)) * ws))


@pytest.mark.parametrize("p,lo,hi", [(1, 1.7, 2.5), (2, 2.6, 3.5), (3, 3.4, 4.6)])
def test_burgers_dg_design_order(p, lo, hi):
    e1 = burgers_l1_error(24, p)
    e2 = burgers_l1_error(48, p)
    eoc = math.log(e1 / e2) / math.log(2.0)
    assert lo <= eoc <= hi, (e1, e2, eoc)


def test_linear_advection_2d_design_order():
    """DG Q2, smooth periodic data sin(2 pi (x + y)), a = (1, 0.5), t = 0.05."""
    errs = []
    for n in (6, 12):
        d = I.mesh(2, n, n, degree=2, system=I.LINADV, adv_vx=1.0, adv_vy=0.5)
        ic = (I.IC_FOURIER, [1, 1.0, 1.0, 1.0, 0.0])
        u = O.project(d, *ic)
        t_end, dx = 0.05, 1.0 / n
        nsteps = int(math.ceil(t_end / (0.05 * dx)))
        u = O.ssprk3(d, u, t_end / nsteps, nsteps)
        vals, xs, ys, ws = O.eval_points(d, u, 0, 5)
        ex = np.sin(2 * np.pi * ((xs - 1.0 * t_end) + (ys - 0.5 * t_end)))
        errs.append(np.sum(np.abs(vals - ex) * ws))
    eoc = math.log(errs[0] / errs[1]) / math.log(2.0)
    assert 2.5 <= eoc <= 3.6, (errs, eoc)
