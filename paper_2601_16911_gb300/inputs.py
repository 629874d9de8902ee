"""Seeded synthetic inputs shared by the CUDA path, the tests and the oracle.

This module holds problem data only: the SplitMix64 generator, the seeded draws of
the initial-data parameters and the mesh/problem descriptions of the workloads the
paper runs (Sec. 5).  It contains none of the method's arithmetic and imports neither
the CUDA binding nor the oracle.

Initial data are described as ``(ic_type, params)``; both the oracle and the CUDA
library evaluate and project them independently.  Parameter layouts:

  IC_CONST        params[0:4] = conserved state
  IC_SINE_STEP    A sin(2 pi k (x - x0)/Lx) + B H(x - s): params = (A, k, B, s)
  IC_CIRCLE       center (cx, cy), radius R, inside value, outside value
  IC_QUADRANTS    split (xs, ys), then primitives (rho, vx, vy, p) for quadrants
                  qx + 2 qy (qx = 1 right of xs, qy = 1 above ys)
  IC_FOURIER      M, then per mode (a, kx, ky, phase):
                  sum a sin(2 pi (kx (x-x0)/Lx + ky (y-y0)/Ly) + phase)
  IC_POLY         sum_{i,j<=4} params[i + 5 j] x^i y^j
  IC_DENSITY_WAVE rho = 1 + A sin(2 pi (kx (x-x0)/Lx + ky (y-y0)/Ly)), v = (vx, vy),
                  p = p0: params = (A, kx, ky, vx, vy, p0)
"""
from __future__ import annotations

import math

IC_CONST, IC_SINE_STEP, IC_CIRCLE, IC_QUADRANTS, IC_FOURIER, IC_POLY, IC_DENSITY_WAVE = range(7)

DG, CG = 0, 1
PERIODIC, TRANSMISSIVE = 0, 1
BURGERS, KPP, LINADV, EULER = 0, 1, 2, 3

_MASK = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 (Steele, Lea, Flood 2014): 64-bit counter-based generator."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self, a: float = 0.0, b: float = 1.0) -> float:
        return a + (b - a) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] inclusive."""
        return lo + self.next_u64() % (hi - lo + 1)


def mesh(dim, nx, ny=1, degree=2, system=BURGERS, domain=(0.0, 1.0, 0.0, 1.0), bc=PERIODIC, kind=DG,
         **params) -> dict:
    """Problem description with the paper's parameter defaults (Sec. 3.2, Sec. 5)."""
    bcs = tuple(bc) if isinstance(bc, (tuple, list)) else (bc,) * 4
    d = dict(dim=dim, nx=nx, ny=ny if dim == 2 else 1, degree=degree, kind=kind, system=system, bc=bcs,
             x0=domain[0], x1=domain[1], y0=domain[2], y1=domain[3], eps=1e-6, r=2.0, q=1.0,
             gamma_vertex=1e-3, c_gamma=0.9, sc_quadrature=1, sensor_mode=0, lambda_const=0.0,
             gas_gamma=1.4, adv_vx=1.0, adv_vy=0.0, hweno_limiter=0, positivity=0)
    d.update(params)
    return d


# ---- the five workloads (shapes and value ranges of Sec. 5's experiments) -------------

def burgers1d_step(seed: int, nx: int = 128, degree: int = 2):
    """1D Burgers, periodic [0,1]: u0 = sin(2 pi x) + 0.5 H(x - x0), x0 ~ U(0.3, 0.7)."""
    g = SplitMix64(seed)
    x0 = g.uniform(0.3, 0.7)
    return mesh(1, nx, degree=degree, system=BURGERS), (IC_SINE_STEP, [1.0, 1.0, 0.5, x0])


def burgers1d_sine(nx: int, degree: int):
    """1D Burgers, periodic [0,1]: u0 = sin(2 pi x) (Sec. 5.2, smooth until t = 1/(2 pi))."""
    return mesh(1, nx, degree=degree, system=BURGERS), (IC_SINE_STEP, [1.0, 1.0, 0.0, 2.0])


def kpp(seed: int, n: int = 256, degree: int = 3, kind: int = DG):
    """KPP f = (sin u, cos u) on [-2,2]^2 periodic: 3.5 pi inside a circle of radius
    U(0.5, 1.0) centred at the origin, 0.25 pi outside; lambda_e = 1 (Sec. 5.3)."""
    g = SplitMix64(seed)
    R = g.uniform(0.5, 1.0)
    d = mesh(2, n, n, degree=degree, system=KPP, domain=(-2.0, 2.0, -2.0, 2.0), kind=kind, lambda_const=1.0)
    return d, (IC_CIRCLE, [0.0, 0.0, R, 3.5 * math.pi, 0.25 * math.pi])


def euler_quadrants(seed: int, n: int = 512, degree: int = 3):
    """2D Euler, gamma = 1.4, [0,1]^2 transmissive: four constant quadrants split at
    (0.5, 0.5) with rho, p ~ U(0.1, 1.5) and vx, vy ~ U(-1, 1)."""
    g = SplitMix64(seed)
    prm = [0.5, 0.5]
    for _q in range(4):
        rho = g.uniform(0.1, 1.5)
        vx = g.uniform(-1.0, 1.0)
        vy = g.uniform(-1.0, 1.0)
        p = g.uniform(0.1, 1.5)
        prm += [rho, vx, vy, p]
    return mesh(2, n, n, degree=degree, system=EULER, bc=TRANSMISSIVE), (IC_QUADRANTS, prm)


def fourier_modes(g: SplitMix64, nmodes: int = 4):
    prm = [float(nmodes)]
    for _ in range(nmodes):
        a = g.uniform(0.0, 1.0)
        while True:
            kx, ky = g.randint(0, 3), g.randint(0, 3)
            if kx or ky:
                break
        phase = g.uniform(0.0, 2.0 * math.pi)
        prm += [a, float(kx), float(ky), phase]
    return prm


def burgers2d_batch(seed: int, count: int = 64, nmin: int = 64, nmax: int = 512):
    """Independent 2D Burgers f = (u^2/2, u^2/2) instances on periodic [0,1]^2 with
    N ~ U{nmin..nmax}, p ~ U{1..4} and a seeded sum of 4 Fourier modes."""
    g = SplitMix64(seed)
    out = []
    for _ in range(count):
        n = g.randint(nmin, nmax)
        p = g.randint(1, 4)
        out.append((mesh(2, n, n, degree=p, system=BURGERS), (IC_FOURIER, fourier_modes(g))))
    return out


def mlp_init(seed: int) -> "list[float]":
    """Initial parameters of the 12 -> 64 -> 64 -> 2 surrogate network in its flat layout
    (W1 (64,12), b1, W2 (64,64), b2, W3 (2,64), b3): weights uniform in +-sqrt(6/(fan_in +
    fan_out)), biases zero.  Both the oracle and the GPU training start from these."""
    g = SplitMix64(seed)
    out = []
    for rows, cols in ((64, 12), (64, 64), (2, 64)):
        a = math.sqrt(6.0 / (rows + cols))
        out += [g.uniform(-a, a) for _ in range(rows * cols)]
        out += [0.0] * rows
    return out
