"""Python wrapper of the FP64 CPU oracle (``cvweno_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's ``cpu_baseline`` / ``--impl reference`` legs may import this module.  It
never imports the CUDA package, and the CUDA package never imports it.

Every function takes a plain ``dict`` mesh description (keys of ``or_desc`` in the C
file) and numpy float64 arrays laid out ``u[var][cell][k]`` with ``k = kx + n*ky``
(tensor Legendre modes, reading A11), ``cell = i + nx*j``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cvweno_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libcvweno_oracle.so")
_lock = threading.Lock()
_lib = None

# status codes, systems, boundary kinds and initial-data kinds (oracle numbering)
OK, ERR_ARG, ERR_NONFINITE, ERR_POSITIVITY, ERR_UNSUPPORTED = 0, 1, 3, 4, 6
DG, CG = 0, 1
PERIODIC, TRANSMISSIVE = 0, 1
BURGERS, KPP, LINADV, EULER = 0, 1, 2, 3


class OracleError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"oracle {where} failed with status {code}")
        self.code = code


class _Desc(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("degree", ctypes.c_int), ("kind", ctypes.c_int), ("system", ctypes.c_int),
        ("bc", ctypes.c_int * 4),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double),
        ("y0", ctypes.c_double), ("y1", ctypes.c_double),
        ("eps", ctypes.c_double), ("r", ctypes.c_double), ("q", ctypes.c_double),
        ("gamma_vertex", ctypes.c_double), ("c_gamma", ctypes.c_double),
        ("sc_quadrature", ctypes.c_int), ("sensor_mode", ctypes.c_int),
        ("lambda_const", ctypes.c_double), ("gas_gamma", ctypes.c_double),
        ("adv_vx", ctypes.c_double), ("adv_vy", ctypes.c_double),
        ("hweno_limiter", ctypes.c_int), ("positivity", ctypes.c_int),
    ]


# paper parameters (Sec. 3.2: eps = 1e-6, r = 2; Sec. 5: q = 1, C_gamma = 0.9;
# vertex linear weight 1e-3; Sec. 5.4: gamma = 1.4)
DEFAULTS = dict(
    dim=2, nx=8, ny=8, degree=2, kind=DG, system=BURGERS, bc=(PERIODIC,) * 4,
    x0=0.0, x1=1.0, y0=0.0, y1=1.0, eps=1e-6, r=2.0, q=1.0, gamma_vertex=1e-3,
    c_gamma=0.9, sc_quadrature=1, sensor_mode=0, lambda_const=0.0, gas_gamma=1.4,
    adv_vx=1.0, adv_vy=0.0, hweno_limiter=0, positivity=0,
)


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library (plain gcc, -O2, no fast-math), with
    OpenMP where gcc supports it (the results do not depend on the thread count)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        if subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True).returncode != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            d = P(_Desc)
            dp = P(ctypes.c_double)
            ip = P(ctypes.c_int)
            sig = {
                "or_mesh_counts": [d, ip, ip, ip, ip, ip],
                "or_state_size": [d, ip],
                "or_vertex_patches": [d, ip, ip, ip, ip],
                "or_gauss_rule": [ctypes.c_int, dp, dp],
                "or_hermite": [d, dp, dp, dp],
                "or_vertex_average": [d, dp, dp],
                "or_residual": [d, dp, ip, dp, dp, dp, dp, ip],
                "or_residual_given": [d, dp, dp, dp, dp, dp],
                "or_sc_weights": [d, dp, dp, dp, ip],
                "or_limit": [d, dp, ctypes.c_int, dp, ip],
                "or_features": [d, dp, dp, dp, dp],
                "or_positivity": [d, dp, dp, dp],
                "or_max_wavespeed": [d, dp, dp],
                "or_ssprk3": [d, dp, ctypes.c_double, ctypes.c_int],
                "or_mass_total": [d, dp, dp],
                "or_ic_point": [d, ctypes.c_int, dp, ctypes.c_double, ctypes.c_double, dp],
                "or_project": [d, ctypes.c_int, dp, dp],
                "or_eval_points": [d, dp, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp],
            }
            for name, args in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            lib.or_legendre_dk.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double]
            lib.or_legendre_dk.restype = ctypes.c_double
            lib.or_set_threads.argtypes = [ctypes.c_int]
            lib.or_set_threads.restype = ctypes.c_int
            lib.or_set_threads(1)  # one thread unless a caller asks for more
            _lib = lib
    return _lib


def set_threads(n: int) -> int:
    """Threads of the oracle's cell loops (1 by default); returns the count in effect (1
    when it was built without OpenMP).  Results are bitwise the same for any count."""
    return int(_load().or_set_threads(int(n)))


def desc(**kw) -> dict:
    d = dict(DEFAULTS)
    for k, v in kw.items():
        if k not in d:
            raise KeyError(k)
        d[k] = v
    return d


def _cdesc(d: dict) -> _Desc:
    c = _Desc()
    for k, v in d.items():
        if k == "bc":
            for i in range(4):
                c.bc[i] = int(v[i])
        else:
            setattr(c, k, v)
    return c


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) if a is not None else None


def _check(code, where):
    if code != OK:
        raise OracleError(code, where)


def counts(d: dict) -> dict:
    lib = _load()
    v = [ctypes.c_int() for _ in range(5)]
    _check(lib.or_mesh_counts(ctypes.byref(_cdesc(d)), *[ctypes.byref(x) for x in v]), "mesh_counts")
    return dict(ncell=v[0].value, nd=v[1].value, nvar=v[2].value, nvert=v[3].value, nq=v[4].value)


def state_shape(d: dict):
    """(nvar, ncell, (p+1)^dim) for DG; (nvar, nnode) nodal GLL values for CG."""
    c = counts(d)
    if d.get("kind", DG) == CG:
        n = ctypes.c_int()
        _check(_load().or_state_size(ctypes.byref(_cdesc(d)), ctypes.byref(n)), "state_size")
        return (c["nvar"], n.value // c["nvar"])
    return (c["nvar"], c["ncell"], c["nd"])


def gauss_rule(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    _check(_load().or_gauss_rule(n, _dp(x), _dp(w)), "gauss_rule")
    return x, w


def legendre_dk(m: int, k: int, x: float) -> float:
    return _load().or_legendre_dk(m, k, x)


def vertex_patches(d: dict):
    """Geometric patches: (count[V], cell[V,4], corner[V,4], cvert[E,ncorner])."""
    c = counts(d)
    nv, ne = c["nvert"], c["ncell"]
    ncorner = 4 if d["dim"] == 2 else 2
    cnt = np.zeros(nv, np.int32)
    cell = np.zeros((nv, 4), np.int32)
    cor = np.zeros((nv, 4), np.int32)
    cv = np.zeros((ne, ncorner), np.int32)
    _check(_load().or_vertex_patches(ctypes.byref(_cdesc(d)), _ip(cnt), _ip(cell), _ip(cor), _ip(cv)), "patches")
    return cnt, cell, cor, cv


def _u(u):
    return np.ascontiguousarray(u, dtype=np.float64)


def hermite(d: dict, u):
    """Stage (a): T[e, corner, k] (physical derivatives) and beta[e, corner]."""
    c = counts(d)
    ncorner = 4 if d["dim"] == 2 else 2
    T = np.zeros((c["ncell"], ncorner, c["nd"]))
    beta = np.zeros((c["ncell"], ncorner))
    _check(_load().or_hermite(ctypes.byref(_cdesc(d)), _dp(_u(u)), _dp(T), _dp(beta)), "hermite")
    return T, beta


def vertex_average(d: dict, u):
    """Stage (b): T*[v, k] (physical derivatives of the vertex candidate at x_v)."""
    c = counts(d)
    Ts = np.zeros((c["nvert"], c["nd"]))
    _check(_load().or_vertex_average(ctypes.byref(_cdesc(d)), _dp(_u(u)), _dp(Ts)), "vertex_average")
    return Ts


def residual(d: dict, u, override_troubled=None):
    """Stages (a)-(e): returns dict(dudt, gamma, nu, alpha, troubled)."""
    c = counts(d)
    u = _u(u)
    out = dict(
        dudt=np.zeros(state_shape(d)),
        gamma=np.zeros(c["ncell"]),
        nu=np.zeros(c["ncell"]),
        alpha=np.zeros((c["ncell"], c["nvar"], c["nq"])),
        troubled=np.zeros(c["ncell"], np.int32),
    )
    ov = None if override_troubled is None else np.ascontiguousarray(override_troubled, dtype=np.int32)
    _check(_load().or_residual(ctypes.byref(_cdesc(d)), _dp(u), _ip(ov), _dp(out["dudt"]), _dp(out["gamma"]),
                               _dp(out["nu"]), _dp(out["alpha"]), _ip(out["troubled"])), "residual")
    return out


def residual_given(d: dict, u, gamma, nu, alpha):
    c = counts(d)
    r = np.zeros((c["nvar"], c["ncell"], c["nd"]))
    _check(_load().or_residual_given(ctypes.byref(_cdesc(d)), _dp(_u(u)), _dp(_u(gamma)), _dp(_u(nu)),
                                     _dp(_u(alpha)), _dp(r)), "residual_given")
    return r


def sc_weights(d: dict, u, gamma):
    c = counts(d)
    alpha = np.zeros((c["ncell"], c["nvar"], c["nq"]))
    tr = np.zeros(c["ncell"], np.int32)
    _check(_load().or_sc_weights(ctypes.byref(_cdesc(d)), _dp(_u(u)), _dp(_u(gamma)), _dp(alpha), _ip(tr)),
           "sc_weights")
    return alpha, tr


def limit(d: dict, u, all_cells: bool = False):
    """HWENO limiter (Sec. 3, readings A27/A28): (limited state, limited-cell flags)."""
    c = counts(d)
    uu = _u(u)
    out = np.zeros_like(uu)
    tr = np.zeros(c["ncell"], np.int32)
    _check(_load().or_limit(ctypes.byref(_cdesc(d)), _dp(uu), 1 if all_cells else 0, _dp(out), _ip(tr)), "limit")
    return out.reshape(np.shape(u)), tr


def positivity(d: dict, u):
    """Positivity limiter (readings P1-P4): (limited state, theta per cell, status code:
    0, or 4 when some cell mean is not admissible)."""
    c = counts(d)
    uu = _u(u)
    out = np.zeros_like(uu)
    th = np.zeros(c["ncell"])
    code = _load().or_positivity(ctypes.byref(_cdesc(d)), _dp(uu), _dp(out), _dp(th))
    if code not in (0, 4):
        _check(code, "positivity")
    return out.reshape(np.shape(u)), th, code


def features(d: dict, u):
    """Surrogate-sensor inputs (ncell, 12), the computed sensor gamma (ncell) and the
    element semi-norms ||u^e||_e (ncell); see or_features."""
    c = counts(d)
    f = np.zeros((c["ncell"], 12))
    g = np.zeros(c["ncell"])
    nrm = np.zeros(c["ncell"])
    _check(_load().or_features(ctypes.byref(_cdesc(d)), _dp(_u(u)), _dp(f), _dp(g), _dp(nrm)), "features")
    return f, g, nrm


def max_wavespeed(d: dict, u) -> float:
    lam = ctypes.c_double()
    _check(_load().or_max_wavespeed(ctypes.byref(_cdesc(d)), _dp(_u(u)), ctypes.byref(lam)), "max_wavespeed")
    return lam.value


def ssprk3(d: dict, u, dt: float, nsteps: int = 1):
    """nsteps SSP-RK3 steps; returns the new state (input untouched)."""
    w = _u(u).copy()
    _check(_load().or_ssprk3(ctypes.byref(_cdesc(d)), _dp(w), float(dt), int(nsteps)), "ssprk3")
    return w


def mass_total(d: dict, u):
    c = counts(d)
    t = np.zeros(c["nvar"])
    _check(_load().or_mass_total(ctypes.byref(_cdesc(d)), _dp(_u(u)), _dp(t)), "mass_total")
    return t


def _params(params):
    p = np.zeros(64)
    p[: len(params)] = params
    return p


def ic_point(d: dict, ic_type: int, params, x: float, y: float = 0.0):
    U = np.zeros(4)
    _check(_load().or_ic_point(ctypes.byref(_cdesc(d)), int(ic_type), _dp(_params(params)), x, y, _dp(U)), "ic")
    return U


def project(d: dict, ic_type: int, params):
    """L2 projection of an analytic initial datum (12-point Gauss rule, reading A17)."""
    u = np.zeros(state_shape(d))
    _check(_load().or_project(ctypes.byref(_cdesc(d)), int(ic_type), _dp(_params(params)), _dp(u)), "project")
    return u


def eval_points(d: dict, u, var: int = 0, nq1d: int = 6):
    """Values at nq1d^dim Gauss points per cell with coordinates and weights."""
    c = counts(d)
    npts = c["ncell"] * nq1d ** d["dim"]
    vals, xs, ys, ws = (np.zeros(npts) for _ in range(4))
    _check(_load().or_eval_points(ctypes.byref(_cdesc(d)), _dp(_u(u)), int(var), int(nq1d), _dp(vals), _dp(xs),
                                  _dp(ys), _dp(ws)), "eval_points")
    return vals, xs, ys, ws


def l1_diff(d: dict, u, v, var: int = 0, nq1d: int = 6) -> float:
    """L1(Omega) norm of the difference of two discrete states of the same mesh."""
    a, _, _, w = eval_points(d, u, var, nq1d)
    b, _, _, _ = eval_points(d, v, var, nq1d)
    return float(np.sum(np.abs(a - b) * w))
