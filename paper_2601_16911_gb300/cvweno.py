"""Thin ctypes binding of the CUDA library (``include/cvweno.h``).

Argument marshalling only: every function below calls the C entry point of the same
name; all arithmetic runs in the library's sm_103a kernels.  Device arrays are torch
CUDA tensors (their data pointers are passed), streams are torch CUDA streams (the
current stream by default).  There is no CPU fallback: ``load()`` raises when the
library is missing or cannot be loaded.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_CUDA, ERR_NONFINITE, ERR_POSITIVITY, ERR_TIMEOUT, ERR_UNSUPPORTED, ERR_NOMEM, ERR_CHECK = range(9)
DG, CG = 0, 1
PERIODIC, TRANSMISSIVE = 0, 1
BURGERS, KPP, LINADV, EULER = 0, 1, 2, 3
SENSOR_COMPUTED, SENSOR_SMOOTH, SENSOR_TROUBLED = 0, 1, 2


class CvwenoError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = load().cvweno_status_string(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {msg} (status {code})")
        self.code = code


class cvweno_params(ctypes.Structure):
    _fields_ = [
        ("eps", ctypes.c_double), ("r", ctypes.c_double), ("q", ctypes.c_double),
        ("gamma_vertex", ctypes.c_double), ("c_gamma", ctypes.c_double),
        ("sc_quadrature", ctypes.c_int), ("sensor_mode", ctypes.c_int),
        ("lambda_const", ctypes.c_double), ("gas_gamma", ctypes.c_double),
        ("adv_vx", ctypes.c_double), ("adv_vy", ctypes.c_double),
        ("hweno_limiter", ctypes.c_int), ("positivity", ctypes.c_int),
    ]


class cvweno_mesh_desc(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("degree", ctypes.c_int),
        ("kind", ctypes.c_int), ("system", ctypes.c_int), ("bc", ctypes.c_int * 4),
        ("x0", ctypes.c_double), ("x1", ctypes.c_double), ("y0", ctypes.c_double), ("y1", ctypes.c_double),
        ("params", cvweno_params),
    ]


class cvweno_batch_plan(ctypes.Structure):
    _fields_ = [
        ("schedule", ctypes.c_int), ("tile", ctypes.c_int), ("dynamic", ctypes.c_int),
        ("ctas_per_sm", ctypes.c_int), ("use_graph", ctypes.c_int), ("ms", ctypes.c_float),
    ]


BATCH_FUSED, BATCH_GROUPED = 0, 1

_VP = ctypes.c_void_p
_I64P = ctypes.POINTER(ctypes.c_int64)
_IP = ctypes.POINTER(ctypes.c_int)
_I32P = ctypes.POINTER(ctypes.c_int32)
_DP = ctypes.POINTER(ctypes.c_double)

_SIGNATURES = {
    "cvweno_default_params": (None, [ctypes.POINTER(cvweno_params)]),
    "cvweno_mesh_create": (ctypes.c_int, [ctypes.POINTER(cvweno_mesh_desc), ctypes.POINTER(_VP)]),
    "cvweno_mesh_destroy": (ctypes.c_int, [_VP]),
    "cvweno_mesh_info": (ctypes.c_int, [_VP, _I64P, _I64P, _IP, _I64P, _IP]),
    "cvweno_mesh_tables": (ctypes.c_int, [_VP, _I32P, _I32P, _I32P]),
    "cvweno_state_size": (ctypes.c_int, [_VP, _I64P]),
    "cvweno_project": (ctypes.c_int, [_VP, ctypes.c_int, _DP, _VP, _VP]),
    "cvweno_vertex_data": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "cvweno_sensor": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "cvweno_residual_ex": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "cvweno_residual": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "cvweno_step": (ctypes.c_int, [_VP, _VP, ctypes.c_double, ctypes.c_double, _DP, _VP]),
    "cvweno_advance": (ctypes.c_int, [_VP, _VP, ctypes.c_double, ctypes.c_int, _VP]),
    "cvweno_mass_total": (ctypes.c_int, [_VP, _VP, _DP, _VP]),
    "cvweno_max_wavespeed": (ctypes.c_int, [_VP, _VP, _DP, _VP]),
    "cvweno_status_check": (ctypes.c_int, [_VP, _VP]),
    "cvweno_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "cvweno_step_static": (ctypes.c_int, [ctypes.POINTER(cvweno_mesh_desc), _VP, ctypes.c_double,
                                          ctypes.POINTER(ctypes.c_int32), _VP]),
    "cvweno_limit": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP, _VP]),
    "cvweno_positivity": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP]),
    "cvweno_mesh_set_kernel_timing": (ctypes.c_int, [_VP, ctypes.c_int]),
    "cvweno_kernel_times": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float), ctypes.c_int, _IP]),
    "cvweno_mesh_set_tensor_cores": (ctypes.c_int, [_VP, ctypes.c_int]),
    "cvweno_mesh_set_check_extents": (ctypes.c_int, [_VP, ctypes.c_int64, ctypes.c_int64]),
    "cvweno_kpp_sincos": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP]),
    "cvweno_mlp_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_VP)]),
    "cvweno_mlp_destroy": (ctypes.c_int, [_VP]),
    "cvweno_mlp_get_params": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_float)]),
    "cvweno_mlp_loss_grad": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, ctypes.POINTER(ctypes.c_float),
                                            ctypes.POINTER(ctypes.c_float), _VP]),
    "cvweno_mlp_adam_step": (ctypes.c_int, [_VP, ctypes.c_float, _VP]),
    "cvweno_mlp_train": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, ctypes.c_float,
                                        ctypes.POINTER(ctypes.c_float), _VP]),
    "cvweno_mlp_infer": (ctypes.c_int, [_VP, _VP, ctypes.c_int64, _VP, _VP]),
    "cvweno_features": (ctypes.c_int, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "cvweno_mesh_set_surrogate": (ctypes.c_int, [_VP, _VP, ctypes.c_float]),
    "cvweno_mlp_fallbacks": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_uint64), ctypes.c_int, _VP]),
    "cvweno_batch_create": (ctypes.c_int, [ctypes.POINTER(cvweno_mesh_desc), ctypes.c_int, ctypes.POINTER(_VP)]),
    "cvweno_batch_destroy": (ctypes.c_int, [_VP]),
    "cvweno_batch_offsets": (ctypes.c_int, [_VP, _I64P]),
    "cvweno_batch_set_plan": (ctypes.c_int, [_VP, ctypes.POINTER(cvweno_batch_plan)]),
    "cvweno_batch_get_plan": (ctypes.c_int, [_VP, ctypes.POINTER(cvweno_batch_plan)]),
    "cvweno_batch_autotune": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(cvweno_batch_plan), _VP]),
    "cvweno_batch_residual": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "cvweno_batch_advance": (ctypes.c_int, [_VP, _VP, _DP, ctypes.c_int, _VP]),
    "cvweno_batch_status_check": (ctypes.c_int, [_VP, _IP, _VP]),
}


def checked() -> bool:
    """True when CVWENO_CHECKED=1 selects the bounds-checked library (libcvweno_check.so)."""
    return os.environ.get("CVWENO_CHECKED", "0") == "1"


def library_path() -> str:
    return _build.lib_path(checked())


def load(build_if_missing: bool = False):
    """Load libcvweno.so, or libcvweno_check.so under CVWENO_CHECKED=1 (optionally building
    it first).  Raises if unavailable."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if build_if_missing and _build.is_stale(checked()):
                _build.build(checked=checked())
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library {path} is not built; run paper_2601_16911_gb300.build.build()")
            lib = ctypes.CDLL(path)
            for name, (res, args) in _SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGNATURES)


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check(code, where):
    if code != OK:
        raise CvwenoError(code, where)


def default_params() -> cvweno_params:
    p = cvweno_params()
    load().cvweno_default_params(ctypes.byref(p))
    return p


def make_desc(d: dict) -> cvweno_mesh_desc:
    """Build the C mesh description from a problem dict (see inputs.mesh)."""
    c = cvweno_mesh_desc()
    c.dim, c.nx, c.ny, c.degree = int(d["dim"]), int(d["nx"]), int(d.get("ny", 1)), int(d["degree"])
    c.kind, c.system = int(d.get("kind", DG)), int(d["system"])
    for i in range(4):
        c.bc[i] = int(d["bc"][i])
    c.x0, c.x1, c.y0, c.y1 = float(d["x0"]), float(d["x1"]), float(d.get("y0", 0.0)), float(d.get("y1", 1.0))
    p = default_params()
    for f, _ in cvweno_params._fields_:
        if f in d:
            setattr(p, f, type(getattr(p, f))(d[f]))
    c.params = p
    return c


class Mesh:
    """Owning handle of a cvweno_mesh; methods mirror the C entry points."""

    def __init__(self, d: dict):
        lib = load()
        self.desc = dict(d)
        self._h = _VP()
        _check(lib.cvweno_mesh_create(ctypes.byref(make_desc(d)), ctypes.byref(self._h)), "cvweno_mesh_create")
        nc, nd, nverts = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        nv, nq = ctypes.c_int(), ctypes.c_int()
        _check(lib.cvweno_mesh_info(self._h, ctypes.byref(nc), ctypes.byref(nd), ctypes.byref(nv),
                                    ctypes.byref(nverts), ctypes.byref(nq)), "cvweno_mesh_info")
        self.ncells, self.ndof, self.nvars, self.nverts, self.nquad = nc.value, nd.value, nv.value, nverts.value, nq.value
        ns = ctypes.c_int64()
        _check(lib.cvweno_state_size(self._h, ctypes.byref(ns)), "cvweno_state_size")
        self.nstate = ns.value
        if int(d.get("kind", DG)) == CG:
            self.state_shape = (self.nvars, self.nstate // self.nvars)
        else:
            self.state_shape = (self.nvars, self.ncells, self.ndof)

    def close(self):
        if self._h:
            load().cvweno_mesh_destroy(self._h)
            self._h = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def empty_state(self, device="cuda"):
        return torch.empty(self.state_shape, dtype=torch.float32, device=device)

    def tables(self):
        import numpy as np
        ncorner = 4 if self.desc["dim"] == 2 else 2
        cv = np.zeros((self.ncells, ncorner), np.int32)
        vc = np.zeros((self.nverts, ncorner), np.int32)
        col = np.zeros(self.ncells, np.int32)
        _check(load().cvweno_mesh_tables(self._h, cv.ctypes.data_as(_I32P), vc.ctypes.data_as(_I32P),
                                         col.ctypes.data_as(_I32P)), "cvweno_mesh_tables")
        return cv, vc, col

    def project(self, ic_type: int, params, out=None, stream=None):
        prm = (ctypes.c_double * 64)()
        for i, v in enumerate(params):
            prm[i] = float(v)
        u = out if out is not None else self.empty_state()
        _check(load().cvweno_project(self._h, int(ic_type), prm, _ptr(u), _stream(stream)), "cvweno_project")
        return u

    def vertex_data(self, u, stream=None):
        ts = torch.empty((self.nverts, self.ndof), dtype=torch.float32, device=u.device)
        _check(load().cvweno_vertex_data(self._h, _ptr(u), _ptr(ts), _stream(stream)), "cvweno_vertex_data")
        return ts

    def sensor(self, u, stream=None):
        g = torch.empty(self.ncells, dtype=torch.float32, device=u.device)
        nu = torch.empty_like(g)
        _check(load().cvweno_sensor(self._h, _ptr(u), _ptr(g), _ptr(nu), _stream(stream)), "cvweno_sensor")
        return g, nu

    def residual(self, u, out=None, stream=None):
        r = out if out is not None else torch.empty_like(u)
        _check(load().cvweno_residual(self._h, _ptr(u), _ptr(r), _stream(stream)), "cvweno_residual")
        return r

    def residual_ex(self, u, troubled_override=None, stream=None):
        dev = u.device
        out = dict(
            dudt=torch.empty_like(u),
            gamma=torch.empty(self.ncells, dtype=torch.float32, device=dev),
            nu=torch.empty(self.ncells, dtype=torch.float32, device=dev),
            alpha=torch.empty((self.ncells, self.nvars, self.nquad), dtype=torch.float32, device=dev),
            troubled=torch.empty(self.ncells, dtype=torch.int32, device=dev),
        )
        _check(load().cvweno_residual_ex(self._h, _ptr(u), _ptr(troubled_override), _ptr(out["dudt"]),
                                         _ptr(out["gamma"]), _ptr(out["nu"]), _ptr(out["alpha"]),
                                         _ptr(out["troubled"]), _stream(stream)), "cvweno_residual_ex")
        return out

    def step(self, u, dt: float = 0.0, cfl: float = 0.0, stream=None) -> float:
        used = ctypes.c_double()
        _check(load().cvweno_step(self._h, _ptr(u), float(dt), float(cfl), ctypes.byref(used), _stream(stream)),
               "cvweno_step")
        return used.value

    def advance(self, u, dt: float, nsteps: int, stream=None):
        _check(load().cvweno_advance(self._h, _ptr(u), float(dt), int(nsteps), _stream(stream)), "cvweno_advance")

    def mass_total(self, u, stream=None):
        t = (ctypes.c_double * self.nvars)()
        _check(load().cvweno_mass_total(self._h, _ptr(u), t, _stream(stream)), "cvweno_mass_total")
        return [t[i] for i in range(self.nvars)]

    def max_wavespeed(self, u, stream=None) -> float:
        lam = ctypes.c_double()
        _check(load().cvweno_max_wavespeed(self._h, _ptr(u), ctypes.byref(lam), _stream(stream)),
               "cvweno_max_wavespeed")
        return lam.value

    def positivity(self, u, out=None, stream=None):
        """Positivity limiter (Euler): (limited state, theta per cell)."""
        out = torch.empty_like(u) if out is None else out
        th = torch.empty(self.ncells, dtype=torch.float32, device=u.device)
        _check(load().cvweno_positivity(self._h, _ptr(u), _ptr(out), _ptr(th), _stream(stream)), "cvweno_positivity")
        return out, th

    def limit(self, u, all_cells: bool = False, out=None, stream=None):
        """HWENO limiter (Sec. 3): (limited state, int32 flags of the limited cells)."""
        out = torch.empty_like(u) if out is None else out
        tr = torch.empty(self.ncells, dtype=torch.int32, device=u.device)
        _check(load().cvweno_limit(self._h, _ptr(u), _ptr(out), 1 if all_cells else 0, _ptr(tr), _stream(stream)),
               "cvweno_limit")
        return out, tr

    def features(self, u, with_norm: bool = False, stream=None):
        """Surrogate inputs (ncells, 12), the computed sensor gamma (ncells) and, with
        with_norm, the semi-norms ||u^e||_e (ncells)."""
        f = torch.empty((self.ncells, 12), dtype=torch.float32, device=u.device)
        g = torch.empty(self.ncells, dtype=torch.float32, device=u.device)
        n = torch.empty(self.ncells, dtype=torch.float32, device=u.device) if with_norm else None
        _check(load().cvweno_features(self._h, _ptr(u), _ptr(f), _ptr(g), _ptr(n), _stream(stream)),
               "cvweno_features")
        return (f, g, n) if with_norm else (f, g)

    def set_surrogate(self, net, conf_min: float = 0.5):
        """Attach a trained Mlp (None detaches); keep `net` alive while attached."""
        self._surrogate = net
        _check(load().cvweno_mesh_set_surrogate(self._h, net.handle if net is not None else None, float(conf_min)),
               "cvweno_mesh_set_surrogate")

    def set_kernel_timing(self, enable: bool = True):
        _check(load().cvweno_mesh_set_kernel_timing(self._h, 1 if enable else 0), "cvweno_mesh_set_kernel_timing")

    def set_tensor_cores(self, enable: bool = True):
        """Stage (c)'s corner products on the tensor cores (split TF32) or as FP32 FMAs."""
        _check(load().cvweno_mesh_set_tensor_cores(self._h, 1 if enable else 0), "cvweno_mesh_set_tensor_cores")

    def set_check_extents(self, state_floats: int = -1, cells: int = -1):
        """Narrow the extents the checked library's bounds checks use (-1, -1: the mesh's
        own).  Raises CvwenoError(ERR_UNSUPPORTED) on the normal library."""
        _check(load().cvweno_mesh_set_check_extents(self._h, int(state_floats), int(cells)),
               "cvweno_mesh_set_check_extents")

    def kernel_times(self):
        """Durations (ms) of the kernels of the most recent step, in launch order."""
        buf = (ctypes.c_float * 64)()
        n = ctypes.c_int(0)
        _check(load().cvweno_kernel_times(self._h, buf, 64, ctypes.byref(n)), "cvweno_kernel_times")
        return [buf[i] for i in range(n.value)]

    def status_check(self, stream=None):
        _check(load().cvweno_status_check(self._h, _stream(stream)), "cvweno_status_check")


# ---- the C entry points under their own names (argument marshalling only) ----------------

def _h(mesh):
    return mesh.handle if isinstance(mesh, Mesh) else mesh


def cvweno_mesh_create(desc: dict) -> Mesh:
    return Mesh(desc)


def cvweno_mesh_destroy(mesh: Mesh):
    mesh.close()


def cvweno_mesh_info(mesh: Mesh) -> dict:
    return dict(ncells=mesh.ncells, ndof_per_var=mesh.ndof, nvars=mesh.nvars, nverts=mesh.nverts, nquad=mesh.nquad)


def cvweno_mesh_tables(mesh: Mesh):
    return mesh.tables()


def cvweno_state_size(mesh: Mesh) -> int:
    return mesh.nstate


def cvweno_project(mesh: Mesh, ic_type: int, params, u, stream=None):
    return mesh.project(ic_type, params, out=u, stream=stream)


def cvweno_vertex_data(mesh: Mesh, u, tstar, stream=None):
    _check(load().cvweno_vertex_data(_h(mesh), _ptr(u), _ptr(tstar), _stream(stream)), "cvweno_vertex_data")


def cvweno_sensor(mesh: Mesh, u, gamma, nu, stream=None):
    _check(load().cvweno_sensor(_h(mesh), _ptr(u), _ptr(gamma), _ptr(nu), _stream(stream)), "cvweno_sensor")


def cvweno_residual_ex(mesh: Mesh, u, troubled_override, dudt, gamma=None, nu=None, alpha=None, troubled=None,
                       stream=None):
    _check(load().cvweno_residual_ex(_h(mesh), _ptr(u), _ptr(troubled_override), _ptr(dudt), _ptr(gamma), _ptr(nu),
                                     _ptr(alpha), _ptr(troubled), _stream(stream)), "cvweno_residual_ex")


def cvweno_residual(mesh: Mesh, u, dudt, stream=None):
    _check(load().cvweno_residual(_h(mesh), _ptr(u), _ptr(dudt), _stream(stream)), "cvweno_residual")


def cvweno_step(mesh: Mesh, u, dt: float = 0.0, cfl: float = 0.0, stream=None) -> float:
    return mesh.step(u, dt, cfl, stream)


def cvweno_advance(mesh: Mesh, u, dt: float, nsteps: int, stream=None):
    mesh.advance(u, dt, nsteps, stream)


def cvweno_mass_total(mesh: Mesh, u, stream=None):
    return mesh.mass_total(u, stream)


def cvweno_max_wavespeed(mesh: Mesh, u, stream=None) -> float:
    return mesh.max_wavespeed(u, stream)


def cvweno_status_check(mesh: Mesh, stream=None):
    mesh.status_check(stream)


def cvweno_status_string(code: int) -> str:
    return load().cvweno_status_string(int(code)).decode()


def cvweno_default_params() -> cvweno_params:
    return default_params()


def cvweno_step_static(desc: dict, u, dt: float, check_status: bool = False, stream=None) -> int:
    """One SSP-RK3 step that allocates nothing (see include/cvweno.h); returns the
    device status bits when check_status is set (the call then synchronises)."""
    st = ctypes.c_int32(0)
    _check(load().cvweno_step_static(ctypes.byref(make_desc(desc)), _ptr(u), float(dt),
                                     ctypes.byref(st) if check_status else None, _stream(stream)),
           "cvweno_step_static")
    return st.value


def _plan_dict(p: cvweno_batch_plan) -> dict:
    return {f: getattr(p, f) for f, _ in cvweno_batch_plan._fields_}


class Batch:
    """Owning handle of a cvweno_batch: independent 2D DG meshes advanced together.
    The batch state is one flat float32 CUDA tensor; instance k occupies
    ``u[offsets[k]:offsets[k+1]]`` in that mesh's state layout."""

    def __init__(self, descs):
        lib = load()
        self.descs = [dict(d) for d in descs]
        arr = (cvweno_mesh_desc * len(descs))(*[make_desc(d) for d in descs])
        self._h = _VP()
        _check(lib.cvweno_batch_create(arr, len(descs), ctypes.byref(self._h)), "cvweno_batch_create")
        off = (ctypes.c_int64 * (len(descs) + 1))()
        _check(lib.cvweno_batch_offsets(self._h, off), "cvweno_batch_offsets")
        self.offsets = [int(v) for v in off]
        self.count = len(descs)

    def close(self):
        if self._h:
            load().cvweno_batch_destroy(self._h)
            self._h = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    @property
    def nstate(self) -> int:
        return self.offsets[-1]

    def empty_state(self, device="cuda"):
        return torch.empty(self.nstate, dtype=torch.float32, device=device)

    def view(self, u, k: int):
        """Instance k's slice of the batch state (a view, flat)."""
        return u[self.offsets[k]:self.offsets[k + 1]]

    def set_plan(self, **kw):
        p = cvweno_batch_plan()
        _check(load().cvweno_batch_get_plan(self._h, ctypes.byref(p)), "cvweno_batch_get_plan")
        for k, v in kw.items():
            setattr(p, k, type(getattr(p, k))(v))
        _check(load().cvweno_batch_set_plan(self._h, ctypes.byref(p)), "cvweno_batch_set_plan")

    def plan(self) -> dict:
        p = cvweno_batch_plan()
        _check(load().cvweno_batch_get_plan(self._h, ctypes.byref(p)), "cvweno_batch_get_plan")
        return _plan_dict(p)

    def autotune(self, u, stream=None) -> dict:
        p = cvweno_batch_plan()
        _check(load().cvweno_batch_autotune(self._h, _ptr(u), ctypes.byref(p), _stream(stream)),
               "cvweno_batch_autotune")
        return _plan_dict(p)

    def residual(self, u, out=None, stream=None):
        out = torch.empty_like(u) if out is None else out
        _check(load().cvweno_batch_residual(self._h, _ptr(u), _ptr(out), _stream(stream)), "cvweno_batch_residual")
        return out

    def advance(self, u, dt, nsteps: int, stream=None):
        dts = (ctypes.c_double * self.count)(*[float(x) for x in dt])
        _check(load().cvweno_batch_advance(self._h, _ptr(u), dts, int(nsteps), _stream(stream)),
               "cvweno_batch_advance")

    def status_check(self, stream=None) -> int:
        bad = ctypes.c_int(-1)
        _check(load().cvweno_batch_status_check(self._h, ctypes.byref(bad), _stream(stream)),
               "cvweno_batch_status_check")
        return bad.value


def cvweno_batch_create(descs) -> Batch:
    return Batch(descs)


def cvweno_batch_destroy(batch: Batch):
    batch.close()


def cvweno_batch_offsets(batch: Batch):
    return list(batch.offsets)


def cvweno_batch_set_plan(batch: Batch, **plan):
    batch.set_plan(**plan)


def cvweno_batch_get_plan(batch: Batch) -> dict:
    return batch.plan()


def cvweno_batch_autotune(batch: Batch, u, stream=None) -> dict:
    return batch.autotune(u, stream)


def cvweno_batch_residual(batch: Batch, u, dudt, stream=None):
    batch.residual(u, dudt, stream)


def cvweno_batch_advance(batch: Batch, u, dt, nsteps: int, stream=None):
    batch.advance(u, dt, nsteps, stream)


def cvweno_batch_status_check(batch: Batch, stream=None) -> int:
    return batch.status_check(stream)


def cvweno_mesh_set_kernel_timing(mesh: Mesh, enable: bool = True):
    mesh.set_kernel_timing(enable)


def cvweno_kernel_times(mesh: Mesh):
    return mesh.kernel_times()


def cvweno_mesh_set_tensor_cores(mesh: Mesh, enable: bool = True):
    mesh.set_tensor_cores(enable)


def cvweno_mesh_set_check_extents(mesh: Mesh, state_floats: int = -1, cells: int = -1):
    mesh.set_check_extents(state_floats, cells)


def cvweno_kpp_sincos(d, stream=None):
    """(sin d, cos d - 1) of a float32 CUDA tensor, in the KPP flux's FP32 forms."""
    d = d.contiguous()
    out = torch.empty(2 * d.numel(), dtype=torch.float32, device=d.device)
    _check(load().cvweno_kpp_sincos(_ptr(d), _ptr(out), int(d.numel()), _stream(stream)), "cvweno_kpp_sincos")
    return out[:d.numel()].view(d.shape), out[d.numel():].view(d.shape)


def cvweno_limit(mesh: Mesh, u, out, all_cells: bool = False, troubled=None, stream=None):
    _check(load().cvweno_limit(mesh.handle, _ptr(u), _ptr(out), 1 if all_cells else 0, _ptr(troubled),
                               _stream(stream)), "cvweno_limit")


NPARAM_MLP = 5122


class Mlp:
    """Owning handle of the surrogate network (cvweno_mlp)."""

    def __init__(self, params=None):
        self._h = _VP()
        buf = None
        if params is not None:
            buf = (ctypes.c_float * NPARAM_MLP)(*[float(v) for v in params])
        _check(load().cvweno_mlp_create(buf, ctypes.byref(self._h)), "cvweno_mlp_create")

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            load().cvweno_mlp_destroy(self._h)
            self._h = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        buf = (ctypes.c_float * NPARAM_MLP)()
        _check(load().cvweno_mlp_get_params(self._h, buf), "cvweno_mlp_get_params")
        return [buf[i] for i in range(NPARAM_MLP)]

    def loss_grad(self, X, y, stream=None):
        loss = ctypes.c_float()
        grad = (ctypes.c_float * NPARAM_MLP)()
        _check(load().cvweno_mlp_loss_grad(self._h, _ptr(X), _ptr(y), int(X.shape[0]), ctypes.byref(loss), grad,
                                           _stream(stream)), "cvweno_mlp_loss_grad")
        return loss.value, [grad[i] for i in range(NPARAM_MLP)]

    def adam_step(self, lr: float, stream=None):
        _check(load().cvweno_mlp_adam_step(self._h, float(lr), _stream(stream)), "cvweno_mlp_adam_step")

    def train(self, X, y, batch: int, epochs: int, lr: float, stream=None) -> float:
        loss = ctypes.c_float()
        _check(load().cvweno_mlp_train(self._h, _ptr(X), _ptr(y), int(X.shape[0]), int(batch), int(epochs),
                                       float(lr), ctypes.byref(loss), _stream(stream)), "cvweno_mlp_train")
        return loss.value

    def infer(self, X, stream=None):
        out = torch.empty((X.shape[0], 2), dtype=torch.float32, device=X.device)
        _check(load().cvweno_mlp_infer(self._h, _ptr(X), int(X.shape[0]), _ptr(out), _stream(stream)),
               "cvweno_mlp_infer")
        return out

    def fallbacks(self, reset: bool = False, stream=None) -> int:
        c = ctypes.c_uint64()
        _check(load().cvweno_mlp_fallbacks(self._h, ctypes.byref(c), 1 if reset else 0, _stream(stream)),
               "cvweno_mlp_fallbacks")
        return c.value


def cvweno_mlp_create(params=None) -> Mlp:
    return Mlp(params)


def cvweno_mlp_destroy(net: Mlp):
    net.close()


def cvweno_mlp_get_params(net: Mlp):
    return net.params()


def cvweno_mlp_loss_grad(net: Mlp, X, y, stream=None):
    return net.loss_grad(X, y, stream)


def cvweno_mlp_adam_step(net: Mlp, lr: float, stream=None):
    net.adam_step(lr, stream)


def cvweno_mlp_train(net: Mlp, X, y, batch: int, epochs: int, lr: float, stream=None) -> float:
    return net.train(X, y, batch, epochs, lr, stream)


def cvweno_mlp_infer(net: Mlp, X, stream=None):
    return net.infer(X, stream)


def cvweno_features(mesh: Mesh, u, with_norm: bool = False, stream=None):
    return mesh.features(u, with_norm, stream)


def cvweno_mesh_set_surrogate(mesh: Mesh, net, conf_min: float = 0.5):
    mesh.set_surrogate(net, conf_min)


def cvweno_mlp_fallbacks(net: Mlp, reset: bool = False, stream=None) -> int:
    return net.fallbacks(reset, stream)


def cvweno_positivity(mesh: Mesh, u, out, theta=None, stream=None):
    _check(load().cvweno_positivity(mesh.handle, _ptr(u), _ptr(out), _ptr(theta), _stream(stream)),
           "cvweno_positivity")
