"""Plain FP64 CPU oracle of the hybrid lattice Boltzmann scheme (arXiv:0902.3921).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The product path (the
CUDA library and its binding) never imports this package, and this package
never imports the product: the two share no code.

The arithmetic lives in ``hybrid_lbm_oracle.c`` (plain loops, FP64, built
with ``-ffp-contract=off``); this module builds it with gcc, loads it with
ctypes and adds the FP64 diagnostics of Sec. III (sums, maximum spurious
speed, Laplace pressure jump, centre of mass) in plain numpy.

The 3D (D3Q19) stencil weights generalise Eqs. 30-31, which the paper states
for 2D only: no printed 3D value exists, and the 3D operators are pinned by
closed forms (polynomial exactness, Fourier symbols, the flat interface of
Eq. 2 in 3D) instead.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hybrid_lbm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

CS2 = 1.0 / 3.0


def build(force: bool = False) -> str:
    """Compiles the oracle into oracle/_build/liboracle.so (plain gcc, FP64)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                           "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int), ("Lx", ctypes.c_int), ("Ly", ctypes.c_int),
                ("Lz", ctypes.c_int), ("a", ctypes.c_double), ("b", ctypes.c_double),
                ("kappa", ctypes.c_double), ("T", ctypes.c_double), ("tau", ctypes.c_double),
                ("Gamma", ctypes.c_double), ("N", ctypes.c_double), ("Q", ctypes.c_double),
                ("m", ctypes.c_int), ("adv_variant", ctypes.c_int),
                ("cubic_at_half", ctypes.c_int), ("g", ctypes.c_double * 3),
                ("force_steps", ctypes.c_long), ("stencil_fd", ctypes.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        pp = ctypes.POINTER(_Params)
        L = ctypes.c_long
        sig = {
            "orc_stencil_weights": [ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp],
            "orc_grad_D": [pp, dp, dp],
            "orc_lap_D": [pp, dp, dp],
            "orc_lap_std": [pp, dp, dp],
            "orc_mu": [pp, dp, dp],
            "orc_force": [pp, dp, dp, L, dp],
            "orc_feq": [ctypes.c_int, ctypes.c_double, dp, dp],
            "orc_forcing_term": [ctypes.c_int, ctypes.c_double, dp, dp, dp],
            "orc_density": [pp, dp, dp],
            "orc_moments": [pp, dp, dp, dp, dp],
            "orc_init": [pp, dp, dp, dp, dp],
            "orc_lb_step": [pp, dp, dp, L, dp, dp],
            "orc_advect": [pp, dp, dp, ctypes.c_double, dp],
            "orc_diffuse": [pp, dp, dp, ctypes.c_double, dp],
            "orc_fd_step": [pp, dp, dp],
            "orc_run": [pp, dp, dp, L, L, ctypes.c_void_p, ctypes.c_void_p],
            "orc_observe": [pp, dp, dp, L, dp, dp, dp],
        }
        for name, args in sig.items():
            fn = getattr(_lib, name)
            fn.argtypes = args
            fn.restype = None
        _lib.orc_nq.argtypes = [ctypes.c_int]
        _lib.orc_nq.restype = ctypes.c_int
        _lib.orc_set_threads.argtypes = [ctypes.c_int]
        _lib.orc_set_threads.restype = ctypes.c_int
        _lib.orc_lattice.argtypes = [ctypes.c_int, np.ctypeslib.ndpointer(dtype=np.int32),
                                     dp]
        _lib.orc_lattice.restype = None
    return _lib


def set_threads(n: int = 0) -> int:
    """Threads of the oracle's site loops (0: all cores); returns the count.
    Any count gives the same bits (no reduction crosses sites)."""
    return int(lib().orc_set_threads(int(n)))


@dataclass
class Params:
    """Parameters of the scheme, named as in the paper (Eqs. 1, 10, 11, 30-31)."""
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
    m: int = 4
    adv_variant: int = 0
    cubic_at_half: int = 0
    g: tuple = (0.0, 0.0, 0.0)
    force_steps: int = 0
    stencil_fd: int = 0

    @property
    def shape(self):
        return (self.Lz, self.Ly, self.Lx) if self.dims == 3 else (self.Ly, self.Lx)

    @property
    def S(self):
        return self.Lx * self.Ly * (self.Lz if self.dims == 3 else 1)

    @property
    def q(self):
        return 19 if self.dims == 3 else 9

    def c(self):
        p = _Params()
        p.dims, p.Lx, p.Ly = self.dims, self.Lx, self.Ly
        p.Lz = self.Lz if self.dims == 3 else 1
        p.a, p.b, p.kappa, p.T, p.tau, p.Gamma = (self.a, self.b, self.kappa, self.T,
                                                   self.tau, self.Gamma)
        p.N, p.Q, p.m = self.N, self.Q, self.m
        p.adv_variant, p.cubic_at_half = self.adv_variant, self.cubic_at_half
        p.g = (ctypes.c_double * 3)(*[float(x) for x in self.g])
        p.force_steps = int(self.force_steps)
        p.stencil_fd = int(self.stencil_fd)
        return ctypes.byref(p), p


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def lattice(dims):
    q = lib().orc_nq(dims)
    e = np.zeros((q, 3), dtype=np.int32)
    w = np.zeros(q)
    lib().orc_lattice(dims, e, w)
    return e, w


def stencil_weights(dims, N, Q):
    """(grad[3,3,3,3], lap[3,3,3]) weight cubes indexed [alpha][dz+1][dy+1][dx+1]."""
    g = np.zeros(81)
    l = np.zeros(27)
    lib().orc_stencil_weights(dims, float(N), float(Q), g, l)
    return g.reshape(3, 3, 3, 3), l.reshape(3, 3, 3)


def _field_op(name, p: Params, field, ncomp_out=1):
    ref, keep = p.c()
    field = _f64(field).reshape(-1)
    out = np.zeros(p.S * ncomp_out)
    getattr(lib(), name)(ref, field, out)
    shp = p.shape if ncomp_out == 1 else (ncomp_out,) + p.shape
    return out.reshape(shp)


def grad_D(p, field):
    return _field_op("orc_grad_D", p, field, p.dims)


def lap_D(p, field):
    return _field_op("orc_lap_D", p, field)


def lap_std(p, field):
    return _field_op("orc_lap_std", p, field)


def mu(p, phi):
    return _field_op("orc_mu", p, phi)


def force(p: Params, phi, n, t=0):
    ref, keep = p.c()
    out = np.zeros(p.S * p.dims)
    lib().orc_force(ref, _f64(phi).reshape(-1), _f64(n).reshape(-1), int(t), out)
    return out.reshape((p.dims,) + p.shape)


def feq(dims, n, u):
    q = lib().orc_nq(dims)
    out = np.zeros(q)
    uu = np.zeros(3)
    uu[:len(u)] = u
    lib().orc_feq(dims, float(n), uu, out)
    return out


def forcing_term(dims, tau, u, F):
    q = lib().orc_nq(dims)
    out = np.zeros(q)
    uu = np.zeros(3)
    ff = np.zeros(3)
    uu[:len(u)] = u
    ff[:len(F)] = F
    lib().orc_forcing_term(dims, float(tau), uu, ff, out)
    return out


def init(p: Params, n, phi, u):
    """Initial populations [q][...] with u*(0) = u (Eqs. 15, 18)."""
    ref, keep = p.c()
    f = np.zeros(p.q * p.S)
    lib().orc_init(ref, _f64(n).reshape(-1), _f64(phi).reshape(-1), _f64(u).reshape(-1), f)
    return f.reshape((p.q,) + p.shape)


def lb_step(p: Params, f, phi, t):
    """One LB step in place on f; returns (n(t), u*(t))."""
    ref, keep = p.c()
    assert f.dtype == np.float64 and f.flags.c_contiguous
    n = np.zeros(p.S)
    u = np.zeros(p.S * p.dims)
    lib().orc_lb_step(ref, f.reshape(-1), _f64(phi).reshape(-1), int(t), n, u)
    return n.reshape(p.shape), u.reshape((p.dims,) + p.shape)


def advect(p, phi, u, dt):
    ref, keep = p.c()
    out = np.zeros(p.S)
    lib().orc_advect(ref, _f64(phi).reshape(-1), _f64(u).reshape(-1), float(dt), out)
    return out.reshape(p.shape)


def diffuse(p, phi_half, phi_old, dt):
    ref, keep = p.c()
    out = np.zeros(p.S)
    lib().orc_diffuse(ref, _f64(phi_half).reshape(-1), _f64(phi_old).reshape(-1),
                      float(dt), out)
    return out.reshape(p.shape)


def fd_step(p, phi, u):
    """m FD substeps in place on phi (float64, contiguous)."""
    ref, keep = p.c()
    assert phi.dtype == np.float64 and phi.flags.c_contiguous
    lib().orc_fd_step(ref, phi.reshape(-1), _f64(u).reshape(-1))


def observe(p: Params, f, phi, t):
    """(n, u*, p0) at time t (Eqs. 6, 12, 18)."""
    ref, keep = p.c()
    n = np.zeros(p.S)
    u = np.zeros(p.S * p.dims)
    p0 = np.zeros(p.S)
    lib().orc_observe(ref, _f64(f).reshape(-1), _f64(phi).reshape(-1), int(t), n, u, p0)
    return n.reshape(p.shape), u.reshape((p.dims,) + p.shape), p0.reshape(p.shape)


@dataclass
class State:
    """Oracle simulation state: pre-collision populations and phi at time t."""
    p: Params
    f: np.ndarray
    phi: np.ndarray
    t: int = 0
    r_ref: np.ndarray = field(default=None)

    @classmethod
    def create(cls, p: Params, n, phi, u):
        f = init(p, n, phi, u)
        st = cls(p, f, _f64(phi).reshape(p.shape).copy(), 0)
        st.r_ref = np.array([p.Lx / 2.0, p.Ly / 2.0, (p.Lz / 2.0 if p.dims == 3 else 0.0)])
        return st

    def run(self, nsteps):
        ref, keep = self.p.c()
        lib().orc_run(ref, self.f.reshape(-1), self.phi.reshape(-1), int(self.t),
                      int(nsteps), None, None)
        self.t += int(nsteps)

    def moments(self):
        n, u, _ = observe(self.p, self.f, self.phi, self.t)
        return n, u

    def diagnostics(self):
        return diagnostics(self.p, self.f, self.phi, self.t, self.r_ref, update=self)


def phi0_of(p: Params):
    """Bulk equilibrium value phi_eq = sqrt(-a/b) (Sec. II)."""
    return float(np.sqrt(-p.a / p.b))


def sigma_of(p: Params):
    """Surface tension sqrt(-8 kappa a^3 / (9 b^2)); equal to Eq. 4 when -a = b."""
    return float(np.sqrt(-8.0 * p.kappa * p.a ** 3 / (9.0 * p.b ** 2)))


def xi_of(p: Params):
    """Width of phi0 tanh(x/xi): xi = sqrt(-2 kappa / a), half the xi of Eq. 3."""
    return float(np.sqrt(-2.0 * p.kappa / p.a))


def diagnostics(p: Params, f, phi, t, r_ref, update=None):
    """FP64 observables of Sec. III at time t.

    sum_n, sum_phi, momentum sum n u*, u_max = max |u*| (Table I divides it by
    c_s), dp = p0(centre) - p0(corner site (0,0,0)) (the Laplace jump of a
    centred drop, p0 of Eq. 6), r_cm = sum phi r / sum phi over sites with
    phi > 0 (Eq. 40; periodic images taken nearest to r_ref), v_f = u* at r_cm
    (bi/trilinear, periodic), area = sum (1 + phi/phi0)/2 and R_eff.
    """
    n, u, p0 = observe(p, f, phi, t)
    d = p.dims
    phi = np.asarray(phi).reshape(p.shape)
    umag = np.sqrt(np.sum(u * u, axis=0))
    L = np.array([p.Lx, p.Ly, p.Lz if d == 3 else 1], dtype=np.float64)
    centre = tuple(int(x) for x in (L[::-1][3 - d:] // 2))
    out = {
        "t": t,
        "sum_n": float(np.sum(n)),
        "sum_phi": float(np.sum(phi)),
        "momentum": [float(np.sum(n * u[a])) for a in range(d)],
        "u_max": float(np.max(umag)),
        "dp": float(p0[centre] - p0[(0,) * d]),
        "nonfinite": int(not (np.all(np.isfinite(phi)) and np.all(np.isfinite(f)))),
    }
    # centre of mass over phi > 0 (Eq. 40) with minimum-image unwrap around r_ref
    grids = np.meshgrid(*[np.arange(int(L[a])) for a in range(d)][::-1], indexing="ij")
    coords = grids[::-1]  # x, y(, z) arrays shaped like the field
    mask = phi > 0
    w = phi[mask]
    r_cm = np.zeros(3)
    for a in range(d):
        rel = coords[a][mask] - r_ref[a]
        rel = rel - L[a] * np.floor(rel / L[a] + 0.5)
        r_cm[a] = r_ref[a] + np.sum(w * rel) / np.sum(w)
    out["r_cm"] = [float(x) for x in r_cm[:d]]
    # fluid velocity at r_cm by multilinear interpolation (periodic)
    base = np.floor(r_cm[:d]).astype(int)
    frac = r_cm[:d] - base
    vf = np.zeros(d)
    for corner in range(1 << d):
        idx = []
        wt = 1.0
        for a in range(d):
            bit = (corner >> a) & 1
            idx.append(int((base[a] + bit) % int(L[a])))
            wt *= frac[a] if bit else 1.0 - frac[a]
        for c in range(d):
            vf[c] += wt * u[(c,) + tuple(idx[::-1])]
    out["v_f"] = [float(x) for x in vf]
    phi0 = phi0_of(p)
    area = float(np.sum((1.0 + phi / phi0) / 2.0))
    out["area"] = area
    out["R_eff"] = float(np.sqrt(area / np.pi) if d == 2 else (3.0 * area / (4.0 * np.pi)) ** (1 / 3))
    if update is not None:
        update.r_ref = r_cm.copy()
    return out
