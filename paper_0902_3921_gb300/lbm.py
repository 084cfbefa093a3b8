"""Thin Python binding of the C ABI in include/hybrid_lbm.h (ctypes).

Argument marshalling only: every step of the method runs in the CUDA library
paper_0902_3921_gb300/_build/liblbm.so.  There is no CPU fallback: if the
library is missing or no GPU is present the calls raise.

Functions keep the C names (lbm_create, lbm_init_fields, lbm_step,
lbm_moments, lbm_populations, lbm_diagnostics, lbm_free, ...); `Lattice` is a
small convenience class over them.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblbm.so")

LBM_OK, LBM_EINVAL, LBM_ECUDA, LBM_ENOMEM, LBM_ENONFINITE, LBM_ETIMEOUT, LBM_ESTATE = (
    0, -1, -2, -3, -4, -5, -6)
LBM_F64, LBM_F32DEV, LBM_F16DEV = 0, 1, 2
LBM_ADV_PAPER, LBM_ADV_FLUX = 0, 1
PRECISIONS = {"f64": LBM_F64, "f32dev": LBM_F32DEV, "f16dev": LBM_F16DEV}

# the exported symbols of include/hybrid_lbm.h
EXPORTS = ("lbm_create", "lbm_buffer_bytes", "lbm_create_with_buffers", "lbm_init_fields", "lbm_step", "lbm_moments", "lbm_populations",
           "lbm_lattice", "lbm_diagnostics", "lbm_synchronize", "lbm_time", "lbm_fd_substeps",
           "lbm_set_graphs", "lbm_set_kernel_timing", "lbm_kernel_times", "lbm_save",
           "lbm_load", "lbm_free", "lbm_last_error", "lbm_tuning", "lbm_diagnostics_noalloc",
           "lbm_noalloc_last_error", "lbm_batch_create", "lbm_batch_init_fields",
           "lbm_batch_step", "lbm_batch_moments", "lbm_batch_set_graphs", "lbm_batch_shape",
           "lbm_batch_synchronize", "lbm_batch_free", "lbm_batch_last_error", "lbm_net_create",
           "lbm_net_param_count", "lbm_net_params", "lbm_net_grads", "lbm_net_set_normalisation",
           "lbm_net_normalisation", "lbm_net_forward", "lbm_net_layer_times", "lbm_net_train_step",
           "lbm_surrogate_state",
           "lbm_surrogate_advance", "lbm_surrogate_advance_relaxed", "lbm_net_free",
           "lbm_net_last_error")


class c_lbm_buffers(ctypes.Structure):
    _fields_ = [("populations", ctypes.c_void_p * 2), ("phi", ctypes.c_void_p * 3),
                ("u", ctypes.c_void_p)]


class c_lbm_params(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int), ("Lx", ctypes.c_int), ("Ly", ctypes.c_int),
                ("Lz", ctypes.c_int), ("a", ctypes.c_double), ("b", ctypes.c_double),
                ("kappa", ctypes.c_double), ("T", ctypes.c_double), ("tau", ctypes.c_double),
                ("Gamma", ctypes.c_double), ("N", ctypes.c_double), ("Q", ctypes.c_double),
                ("fd_substeps", ctypes.c_int), ("adv_variant", ctypes.c_int),
                ("cubic_at_half", ctypes.c_int), ("g", ctypes.c_double * 3),
                ("force_steps", ctypes.c_longlong), ("precision", ctypes.c_int),
                ("f16_scale_log2", ctypes.c_int), ("stencil_fd", ctypes.c_int)]


class c_lbm_diag(ctypes.Structure):
    _fields_ = [("t", ctypes.c_longlong), ("sum_n", ctypes.c_double),
                ("sum_phi", ctypes.c_double), ("momentum", ctypes.c_double * 3),
                ("u_max", ctypes.c_double), ("dp", ctypes.c_double),
                ("r_cm", ctypes.c_double * 3), ("v_f", ctypes.c_double * 3),
                ("area", ctypes.c_double), ("R_eff", ctypes.c_double),
                ("nonfinite", ctypes.c_int)]


class c_lbm_instance(ctypes.Structure):
    _fields_ = [("Lx", ctypes.c_int), ("Ly", ctypes.c_int), ("g", ctypes.c_double * 2),
                ("force_steps", ctypes.c_longlong)]


class LbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"liblbm error {code}: {msg}")
        self.code = code


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads liblbm.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "or python paper_0902_3921_gb300/build.py")
    lib = ctypes.CDLL(path)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
    H = ctypes.c_void_p
    lib.lbm_create.argtypes = [ctypes.POINTER(c_lbm_params), vp, ctypes.POINTER(H)]
    lib.lbm_buffer_bytes.argtypes = [ctypes.POINTER(c_lbm_params), ctypes.POINTER(ctypes.c_ulonglong)]
    lib.lbm_create_with_buffers.argtypes = [ctypes.POINTER(c_lbm_params), vp,
                                            ctypes.POINTER(c_lbm_buffers), ctypes.POINTER(H)]
    lib.lbm_init_fields.argtypes = [H, dp, dp, dp, dp, dp]
    lib.lbm_step.argtypes = [H, ctypes.c_longlong]
    lib.lbm_moments.argtypes = [H, dp, dp, dp, dp, dp]
    lib.lbm_populations.argtypes = [H, dp]
    lib.lbm_lattice.argtypes = [ip, ctypes.POINTER(ctypes.c_int), dp]
    lib.lbm_diagnostics.argtypes = [H, ctypes.POINTER(c_lbm_diag)]
    lib.lbm_synchronize.argtypes = [H]
    lib.lbm_time.argtypes = [H]
    lib.lbm_time.restype = ctypes.c_longlong
    lib.lbm_fd_substeps.argtypes = [H]
    lib.lbm_tuning.argtypes = [H, ctypes.POINTER(ctypes.c_int), ip]
    lib.lbm_tuning.restype = ctypes.c_int
    lib.lbm_set_graphs.argtypes = [H, ip]
    lib.lbm_set_kernel_timing.argtypes = [H, ip]
    lib.lbm_kernel_times.argtypes = [H, dp, ctypes.POINTER(ctypes.c_longlong), ip]
    lib.lbm_save.argtypes = [H, ctypes.c_char_p]
    lib.lbm_load.argtypes = [H, ctypes.c_char_p]
    lib.lbm_free.argtypes = [H]
    lib.lbm_free.restype = None
    lib.lbm_last_error.argtypes = [H]
    lib.lbm_last_error.restype = ctypes.c_char_p
    lib.lbm_diagnostics_noalloc.argtypes = [ctypes.POINTER(c_lbm_params), vp, dp, vp,
                                            ctypes.POINTER(c_lbm_diag)]
    lib.lbm_diagnostics_noalloc.restype = ctypes.c_int
    lib.lbm_noalloc_last_error.argtypes = []
    lib.lbm_noalloc_last_error.restype = ctypes.c_char_p
    B = ctypes.c_void_p
    lib.lbm_batch_create.argtypes = [ctypes.POINTER(c_lbm_params), ctypes.POINTER(c_lbm_instance),
                                     ip, vp, ctypes.POINTER(B)]
    lib.lbm_batch_init_fields.argtypes = [B, ip, dp, dp, dp, dp]
    lib.lbm_batch_step.argtypes = [B, ctypes.c_longlong]
    lib.lbm_batch_moments.argtypes = [B, ip, dp, dp, dp, dp]
    lib.lbm_batch_set_graphs.argtypes = [B, ip]
    lib.lbm_batch_shape.argtypes = [B, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_longlong)]
    lib.lbm_batch_synchronize.argtypes = [B]
    lib.lbm_batch_free.argtypes = [B]
    lib.lbm_batch_free.restype = None
    lib.lbm_batch_last_error.argtypes = [B]
    lib.lbm_batch_last_error.restype = ctypes.c_char_p
    Nt = ctypes.c_void_p
    fp = ctypes.POINTER(ctypes.c_float)
    lib.lbm_net_create.argtypes = [ip, ip, ctypes.c_ulonglong, ctypes.POINTER(Nt)]
    lib.lbm_net_param_count.argtypes = [Nt]
    lib.lbm_net_param_count.restype = ctypes.c_longlong
    lib.lbm_net_params.argtypes = [Nt, fp, ctypes.c_longlong, ip]
    lib.lbm_net_grads.argtypes = [Nt, fp, ctypes.c_longlong]
    lib.lbm_net_set_normalisation.argtypes = [Nt, fp, fp, fp]
    lib.lbm_net_normalisation.argtypes = [Nt, fp]
    lib.lbm_net_forward.argtypes = [Nt, vp, ip, ip, ip, vp, vp]
    lib.lbm_net_layer_times.argtypes = [Nt, vp, ip, ip, ip, ip, ctypes.POINTER(ctypes.c_float), vp]
    lib.lbm_net_train_step.argtypes = [Nt, vp, vp, ip, ip, ip, ctypes.c_float, ip,
                                       ctypes.POINTER(ctypes.c_double), vp]
    lib.lbm_surrogate_state.argtypes = [H, vp]
    lib.lbm_surrogate_advance.argtypes = [H, Nt, ip, ip, ctypes.c_double, ip, ctypes.c_double,
                                          ctypes.POINTER(ctypes.c_int)]
    lib.lbm_surrogate_advance_relaxed.argtypes = [H, Nt, ip, ip, ip, ctypes.c_double, ip, ctypes.c_double,
                                                  ctypes.POINTER(ctypes.c_int)]
    lib.lbm_net_free.argtypes = [Nt]
    lib.lbm_net_free.restype = None
    lib.lbm_net_last_error.argtypes = [Nt]
    lib.lbm_net_last_error.restype = ctypes.c_char_p
    for name in ("lbm_net_create", "lbm_net_params", "lbm_net_grads", "lbm_net_set_normalisation",
                 "lbm_net_normalisation", "lbm_net_forward", "lbm_net_layer_times", "lbm_net_train_step",
                 "lbm_surrogate_state", "lbm_surrogate_advance", "lbm_surrogate_advance_relaxed"):
        getattr(lib, name).restype = ctypes.c_int
    for name in ("lbm_batch_create", "lbm_batch_init_fields", "lbm_batch_step", "lbm_batch_moments",
                 "lbm_batch_set_graphs", "lbm_batch_shape", "lbm_batch_synchronize"):
        getattr(lib, name).restype = ctypes.c_int
    for name in ("lbm_create", "lbm_init_fields", "lbm_step", "lbm_moments", "lbm_populations",
                 "lbm_lattice", "lbm_diagnostics", "lbm_synchronize", "lbm_fd_substeps",
                 "lbm_set_graphs", "lbm_set_kernel_timing", "lbm_kernel_times", "lbm_save",
                 "lbm_load"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _dptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, S):
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    if a.size != S:
        raise ValueError(f"expected {S} values, got {a.size}")
    return a


@dataclass
class LbmParams:
    """Mirror of lbm_params (names as in the paper: Eqs. 1, 10, 11, 30-31)."""
    dims: int = 2
    Lx: int = 64
    Ly: int = 64
    Lz: int = 1
    a: float = -0.1
    b: float = 0.1
    kappa: float = 0.14
    T: float = 1.0 / 3.0
    tau: float = 1.0
    Gamma: float = 0.5
    N: float = 0.3
    Q: float = 2.5
    fd_substeps: int = 0
    adv_variant: int = LBM_ADV_PAPER
    cubic_at_half: int = 0
    g: tuple = (0.0, 0.0, 0.0)
    force_steps: int = 0
    precision: int = LBM_F32DEV
    f16_scale_log2: int = 0
    stencil_fd: int = 0

    def to_c(self) -> c_lbm_params:
        c = c_lbm_params()
        for k, _ in c_lbm_params._fields_:
            if k == "g":
                c.g = (ctypes.c_double * 3)(*[float(x) for x in self.g])
            else:
                setattr(c, k, getattr(self, k))
        return c

    @property
    def shape(self):
        return (self.Lz, self.Ly, self.Lx) if self.dims == 3 else (self.Ly, self.Lx)

    @property
    def S(self):
        return int(np.prod(self.shape))

    @property
    def q(self):
        return 19 if self.dims == 3 else 9


def _check(h, rc, what=""):
    if rc != LBM_OK:
        msg = load_library().lbm_last_error(h)
        raise LbmError(rc, (what + ": " if what else "") + (msg.decode() if msg else ""))


def lbm_create(params: LbmParams, cuda_stream: int | None = None):
    lib = load_library()
    h = ctypes.c_void_p()
    cp = params.to_c()
    rc = lib.lbm_create(ctypes.byref(cp), ctypes.c_void_p(cuda_stream or 0), ctypes.byref(h))
    if rc != LBM_OK:
        raise LbmError(rc, lib.lbm_last_error(None).decode())
    return h


def lbm_buffer_bytes(params: LbmParams):
    """(population lattice, phi plane, u* planes) byte counts for lbm_create_with_buffers."""
    lib = load_library()
    b = (ctypes.c_ulonglong * 3)()
    cp = params.to_c()
    rc = lib.lbm_buffer_bytes(ctypes.byref(cp), b)
    if rc != LBM_OK:
        raise LbmError(rc, lib.lbm_last_error(None).decode())
    return int(b[0]), int(b[1]), int(b[2])


def lbm_create_with_buffers(params: LbmParams, populations, phi, u, cuda_stream: int | None = None):
    """lbm_create on caller-owned device buffers, given as integer pointers:
    populations (2), phi (3), u.  The caller keeps them alive."""
    lib = load_library()
    h = ctypes.c_void_p()
    cp = params.to_c()
    buf = c_lbm_buffers()
    for k in range(2):
        buf.populations[k] = populations[k]
    for k in range(3):
        buf.phi[k] = phi[k]
    buf.u = u
    rc = lib.lbm_create_with_buffers(ctypes.byref(cp), ctypes.c_void_p(cuda_stream or 0),
                                     ctypes.byref(buf), ctypes.byref(h))
    if rc != LBM_OK:
        raise LbmError(rc, lib.lbm_last_error(None).decode())
    return h


def lbm_init_fields(h, params: LbmParams, n, phi, u):
    S = params.S
    n, phi = _f64(n, S), _f64(phi, S)
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(params.dims, S)
    uz = u[2] if params.dims == 3 else None
    _check(h, load_library().lbm_init_fields(h, _dptr(n), _dptr(phi), _dptr(u[0]), _dptr(u[1]),
                                             _dptr(uz)), "lbm_init_fields")


def lbm_step(h, nsteps: int):
    _check(h, load_library().lbm_step(h, int(nsteps)), "lbm_step")


def lbm_moments(h, params: LbmParams):
    S, d = params.S, params.dims
    n = np.empty(S)
    phi = np.empty(S)
    u = np.empty((d, S))
    _check(h, load_library().lbm_moments(h, _dptr(n), _dptr(phi), _dptr(u[0]), _dptr(u[1]),
                                         _dptr(u[2]) if d == 3 else None), "lbm_moments")
    shp = params.shape
    return n.reshape(shp), phi.reshape(shp), u.reshape((d,) + shp)


def lbm_populations(h, params: LbmParams):
    f = np.empty(params.q * params.S)
    _check(h, load_library().lbm_populations(h, _dptr(f)), "lbm_populations")
    return f.reshape((params.q,) + params.shape)


def lbm_lattice(dims: int):
    q = 19 if dims == 3 else 9
    e = (ctypes.c_int * (3 * q))()
    w = np.empty(q)
    rc = load_library().lbm_lattice(dims, e, _dptr(w))
    if rc < 0:
        raise LbmError(rc, "lbm_lattice")
    return np.array(e[:], dtype=np.int32).reshape(q, 3), w


def lbm_diagnostics(h, dims: int = 2):
    d = c_lbm_diag()
    rc = load_library().lbm_diagnostics(h, ctypes.byref(d))
    if rc not in (LBM_OK, LBM_ENONFINITE):
        _check(h, rc, "lbm_diagnostics")
    return {"t": d.t, "sum_n": d.sum_n, "sum_phi": d.sum_phi,
            "momentum": list(d.momentum)[:dims], "u_max": d.u_max, "dp": d.dp,
            "r_cm": list(d.r_cm)[:dims], "v_f": list(d.v_f)[:dims], "area": d.area,
            "R_eff": d.R_eff, "nonfinite": d.nonfinite, "rc": rc}


def lbm_diagnostics_noalloc(params: LbmParams, fields_device_ptr: int, r_ref=None,
                            cuda_stream: int | None = None):
    """Allocation-free diagnostics of caller-owned device fields
    [n | phi | u*_x | u*_y (| u*_z)] (FP64); see include/hybrid_lbm.h.
    Returns (rc, dict)."""
    lib = load_library()
    d = c_lbm_diag()
    cp = params.to_c()
    rr = None
    if r_ref is not None:
        rr_arr = (ctypes.c_double * 3)(*[float(x) for x in (list(r_ref) + [0.0] * 3)[:3]])
        rr = ctypes.cast(rr_arr, ctypes.POINTER(ctypes.c_double))
    rc = lib.lbm_diagnostics_noalloc(ctypes.byref(cp), ctypes.c_void_p(fields_device_ptr), rr,
                                     ctypes.c_void_p(cuda_stream or 0), ctypes.byref(d))
    if rc not in (LBM_OK, LBM_ENONFINITE):
        raise LbmError(rc, lib.lbm_noalloc_last_error().decode())
    dims = params.dims
    return rc, {"sum_n": d.sum_n, "sum_phi": d.sum_phi, "momentum": list(d.momentum)[:dims],
                "u_max": d.u_max, "dp": d.dp, "r_cm": list(d.r_cm)[:dims],
                "v_f": list(d.v_f)[:dims], "area": d.area, "R_eff": d.R_eff,
                "nonfinite": d.nonfinite}


def lbm_synchronize(h):
    _check(h, load_library().lbm_synchronize(h), "lbm_synchronize")


def lbm_time(h) -> int:
    return load_library().lbm_time(h)


def lbm_fd_substeps(h) -> int:
    return load_library().lbm_fd_substeps(h)


def lbm_tuning(h) -> dict:
    v = (ctypes.c_int * 6)()
    load_library().lbm_tuning(h, v, 6)
    return {"fd_substeps_per_launch": v[0], "fd_rows_per_warp": v[1], "fd_cols_per_lane": v[2],
            "collide_sites_per_thread": v[3], "m": v[4], "fd_tile_width": v[5]}


def lbm_set_graphs(h, enable: bool):
    _check(h, load_library().lbm_set_graphs(h, int(enable)))


def lbm_set_kernel_timing(h, enable: bool):
    _check(h, load_library().lbm_set_kernel_timing(h, int(enable)))


def lbm_kernel_times(h, reset: bool = False):
    ms = (ctypes.c_double * 3)()
    n = (ctypes.c_longlong * 3)()
    _check(h, load_library().lbm_kernel_times(h, ms, n, int(reset)), "lbm_kernel_times")
    names = ("collide", "fd", "density")
    return {k: (ms[i], n[i]) for i, k in enumerate(names)}


def lbm_save(h, path: str):
    _check(h, load_library().lbm_save(h, path.encode()), "lbm_save")


def lbm_load(h, path: str) -> int:
    return load_library().lbm_load(h, path.encode())


def lbm_free(h):
    if h:
        load_library().lbm_free(h)


def lbm_last_error(h=None) -> str:
    m = load_library().lbm_last_error(h)
    return m.decode() if m else ""


@dataclass
class Lattice:
    """Owning wrapper around one lbm_handle.  buffers (optional): caller-owned
    device tensors {"populations": (a, b), "phi": (a, b, c), "u": a} with
    .data_ptr() (e.g. torch tensors of the sizes lbm_buffer_bytes gives); the
    lattice keeps references to them so that they outlive the handle."""
    params: LbmParams
    stream: int | None = None
    buffers: dict | None = None
    handle: object = field(default=None, init=False)

    def __post_init__(self):
        if self.buffers is None:
            self.handle = lbm_create(self.params, self.stream)
        else:
            b = self.buffers
            self.handle = lbm_create_with_buffers(
                self.params, [t.data_ptr() for t in b["populations"]], [t.data_ptr() for t in b["phi"]],
                b["u"].data_ptr(), self.stream)

    def init_fields(self, n, phi, u):
        lbm_init_fields(self.handle, self.params, n, phi, u)
        return self

    def step(self, nsteps: int):
        lbm_step(self.handle, nsteps)
        return self

    def moments(self):
        return lbm_moments(self.handle, self.params)

    def populations(self):
        return lbm_populations(self.handle, self.params)

    def diagnostics(self):
        return lbm_diagnostics(self.handle, self.params.dims)

    def synchronize(self):
        lbm_synchronize(self.handle)

    @property
    def t(self):
        return lbm_time(self.handle)

    @property
    def m(self):
        return lbm_fd_substeps(self.handle)

    def close(self):
        if self.handle:
            lbm_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owning wrapper around one lbm_batch: independent 2D lattices advanced
    together (one persistent launch per call, or the tiled path's launches per
    LB step; the library picks the faster at creation).  `instances` is a list
    of (Lx, Ly, (gx, gy), force_steps)."""

    def __init__(self, common: LbmParams, instances, stream: int | None = None):
        lib = load_library()
        self.common = common
        self.instances = [tuple(i) for i in instances]
        arr = (c_lbm_instance * len(instances))()
        for k, (Lx, Ly, g, fs) in enumerate(self.instances):
            arr[k].Lx, arr[k].Ly = int(Lx), int(Ly)
            arr[k].g = (ctypes.c_double * 2)(float(g[0]), float(g[1]))
            arr[k].force_steps = int(fs)
        self.handle = ctypes.c_void_p()
        cp = common.to_c()
        rc = lib.lbm_batch_create(ctypes.byref(cp), arr, len(instances),
                                  ctypes.c_void_p(stream or 0), ctypes.byref(self.handle))
        if rc != LBM_OK:
            self.handle = None
            raise LbmError(rc, lib.lbm_batch_last_error(None).decode())

    def _check(self, rc, what):
        if rc != LBM_OK:
            raise LbmError(rc, what + ": " + load_library().lbm_batch_last_error(self.handle).decode())

    def init_fields(self, k, n, phi, u):
        Lx, Ly = self.instances[k][:2]
        S = Lx * Ly
        n, phi = _f64(n, S), _f64(phi, S)
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(2, S)
        self._check(load_library().lbm_batch_init_fields(self.handle, k, _dptr(n), _dptr(phi),
                                                         _dptr(u[0]), _dptr(u[1])),
                    "lbm_batch_init_fields")

    def step(self, nsteps):
        self._check(load_library().lbm_batch_step(self.handle, int(nsteps)), "lbm_batch_step")
        return self

    def moments(self, k):
        Lx, Ly = self.instances[k][:2]
        S = Lx * Ly
        n, phi, u = np.empty(S), np.empty(S), np.empty((2, S))
        self._check(load_library().lbm_batch_moments(self.handle, k, _dptr(n), _dptr(phi),
                                                     _dptr(u[0]), _dptr(u[1])), "lbm_batch_moments")
        return n.reshape(Ly, Lx), phi.reshape(Ly, Lx), u.reshape(2, Ly, Lx)

    def set_graphs(self, enable):
        load_library().lbm_batch_set_graphs(self.handle, int(enable))

    def shape(self):
        t, c, st = ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
        load_library().lbm_batch_shape(self.handle, ctypes.byref(t), ctypes.byref(c), ctypes.byref(st))
        return {"threads": t.value, "ctas": c.value, "sites": st.value}

    def synchronize(self):
        self._check(load_library().lbm_batch_synchronize(self.handle), "lbm_batch_synchronize")

    def close(self):
        if self.handle:
            load_library().lbm_batch_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Net:
    """Owning wrapper around one lbm_net (the learned surrogate).  Device
    arrays are passed as integer pointers (e.g. torch.Tensor.data_ptr())."""

    def __init__(self, channels=32, layers=6, seed=0):
        lib = load_library()
        self.handle = ctypes.c_void_p()
        rc = lib.lbm_net_create(int(channels), int(layers), int(seed), ctypes.byref(self.handle))
        if rc != LBM_OK:
            self.handle = None
            raise LbmError(rc, lib.lbm_net_last_error(None).decode())
        self.channels, self.layers = channels, layers

    def _check(self, rc, what):
        if rc != LBM_OK:
            raise LbmError(rc, what + ": " + load_library().lbm_net_last_error(self.handle).decode())

    @property
    def nparams(self):
        return load_library().lbm_net_param_count(self.handle)

    def get_params(self):
        a = np.empty(self.nparams, dtype=np.float32)
        self._check(load_library().lbm_net_params(self.handle, a.ctypes.data_as(
            ctypes.POINTER(ctypes.c_float)), a.size, 0), "lbm_net_params")
        return a

    def set_params(self, a):
        a = np.ascontiguousarray(a, dtype=np.float32)
        self._check(load_library().lbm_net_params(self.handle, a.ctypes.data_as(
            ctypes.POINTER(ctypes.c_float)), a.size, 1), "lbm_net_params")

    def get_grads(self):
        a = np.empty(self.nparams, dtype=np.float32)
        self._check(load_library().lbm_net_grads(self.handle, a.ctypes.data_as(
            ctypes.POINTER(ctypes.c_float)), a.size), "lbm_net_grads")
        return a

    def set_normalisation(self, in_mean, in_std, out_std):
        arrs = [np.ascontiguousarray(v, dtype=np.float32) for v in (in_mean, in_std, out_std)]
        ptrs = [a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)) for a in arrs]
        self._check(load_library().lbm_net_set_normalisation(self.handle, *ptrs),
                    "lbm_net_set_normalisation")

    def normalisation(self):
        a = np.empty(12, dtype=np.float32)
        self._check(load_library().lbm_net_normalisation(self.handle, a.ctypes.data_as(
            ctypes.POINTER(ctypes.c_float))), "lbm_net_normalisation")
        return a[:4], a[4:8], a[8:]

    def forward(self, x0_ptr, N, H, W, x1_ptr, stream=None):
        self._check(load_library().lbm_net_forward(self.handle, ctypes.c_void_p(x0_ptr), N, H, W,
                                                   ctypes.c_void_p(x1_ptr),
                                                   ctypes.c_void_p(stream or 0)), "lbm_net_forward")

    def layer_times(self, x0_ptr, N, H, W, reps=10, stream=None):
        """Mean milliseconds of each convolution layer's launch (CUDA events)."""
        ms = (ctypes.c_float * self.layers)()
        self._check(load_library().lbm_net_layer_times(self.handle, ctypes.c_void_p(x0_ptr), N, H, W,
                                                       int(reps), ms, ctypes.c_void_p(stream or 0)),
                    "lbm_net_layer_times")
        return [float(v) for v in ms]

    def train_step(self, x0_ptr, x1_ptr, N, H, W, lr, update=True, stream=None):
        loss = ctypes.c_double()
        self._check(load_library().lbm_net_train_step(
            self.handle, ctypes.c_void_p(x0_ptr), ctypes.c_void_p(x1_ptr), N, H, W, float(lr),
            int(update), ctypes.byref(loss), ctypes.c_void_p(stream or 0)), "lbm_net_train_step")
        return loss.value

    def close(self):
        if self.handle:
            load_library().lbm_net_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lbm_surrogate_state(h, out_ptr):
    _check(h, load_library().lbm_surrogate_state(h, ctypes.c_void_p(out_ptr)), "lbm_surrogate_state")


def lbm_surrogate_advance(h, net: Net, windows, window_steps, mass_tol=2e-3, conserve_mass=True,
                          phi_clamp=0.0, relax_steps=0):
    fb = ctypes.c_int()
    rc = load_library().lbm_surrogate_advance_relaxed(h, net.handle, int(windows), int(window_steps),
                                                      int(relax_steps), float(mass_tol), int(conserve_mass),
                                                      float(phi_clamp), ctypes.byref(fb))
    if rc != LBM_OK:
        msg = load_library().lbm_net_last_error(net.handle).decode() or lbm_last_error(h)
        raise LbmError(rc, "lbm_surrogate_advance: " + msg)
    return fb.value
