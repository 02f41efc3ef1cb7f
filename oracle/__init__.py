"""FP64 CPU oracle of the MLS-MPM substep (ctypes wrapper over ``mpm_oracle.c``).

TEST INFRASTRUCTURE ONLY. The tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers. The product path (the
CUDA library and its binding) never imports this package, and this package
imports nothing from the product.

Each wrapper names the step it runs; the equations and their sources are in
``mpm_oracle.h`` / ``mpm_oracle.c`` (Sec. 3 and Algorithm 1 of the paper, with
the published MLS-MPM, APIC, fixed-corotated and von Mises methods the paper
points to). Inputs arrive as arrays (usually FP32 states from the seeded
generators) and are widened to FP64 here; the oracle never draws random numbers.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpm_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "splat_oracle.c")]
_HDRS = [os.path.join(_HERE, "mpm_oracle.h"), os.path.join(_HERE, "splat_oracle.h")]
_LIB_PATH = os.path.join(_HERE, "libmpm_oracle.so")
_lib = None

PLASTICINE = 0
FLUID = 1
BOX = 0
CAPSULE = 1
SDF_VOLUME = 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction, no fast-math)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
        os.path.getmtime(f) for f in _SRCS + _HDRS
    ):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(
        ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
         "-Wall", "-o", tmp, *_SRCS, "-lm"],
        check=True,
    )
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int),
        ("dt", ctypes.c_double),
        ("gravity", ctypes.c_double * 3),
        ("bound", ctypes.c_int),
        ("kind", ctypes.c_int),
        ("mu", ctypes.c_double),
        ("lam", ctypes.c_double),
        ("yield_stress", ctypes.c_double),
        ("p_vol", ctypes.c_double),
        ("p_mass", ctypes.c_double),
    ]


class _Collider(ctypes.Structure):
    _fields_ = [
        ("type", ctypes.c_int),
        ("half", ctypes.c_double * 3),
        ("friction", ctypes.c_double),
        ("pos", ctypes.c_double * 3),
        ("quat", ctypes.c_double * 4),
        ("lin_vel", ctypes.c_double * 3),
        ("ang_vel", ctypes.c_double * 3),
        ("com", ctypes.c_double * 3),
        ("sdf", ctypes.POINTER(ctypes.c_double)),
        ("res", ctypes.c_int * 3),
        ("sdf_origin", ctypes.c_double * 3),
        ("sdf_h", ctypes.c_double),
    ]


class _Camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int), ("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double), ("eye", ctypes.c_double * 3),
                ("rot", ctypes.c_double * 9), ("near_z", ctypes.c_double)]


class _Render(ctypes.Structure):
    _fields_ = [("radius", ctypes.c_double), ("smooth", ctypes.c_double), ("sigma_depth", ctypes.c_double),
                ("window", ctypes.c_int), ("light", ctypes.c_double * 3), ("albedo", ctypes.c_double * 3),
                ("ambient", ctypes.c_double), ("background", ctypes.c_double * 3)]


class _Penalty(ctypes.Structure):
    _fields_ = [("stiffness", ctypes.c_double), ("damping", ctypes.c_double)]


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_u8p = ctypes.POINTER(ctypes.c_ubyte)


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        L.orc_lame.argtypes = [ctypes.c_double, ctypes.c_double, _dp, _dp]
        L.orc_bspline.argtypes = [ctypes.c_double]
        L.orc_bspline.restype = ctypes.c_double
        L.orc_stencil.argtypes = [ctypes.c_int, _dp, _ip, _ip, _dp, _dp]
        L.orc_svd3.argtypes = [_dp, _dp, _dp, _dp]
        L.orc_svd3.restype = ctypes.c_int
        L.orc_stress_fixed_corotated.argtypes = [ctypes.c_double, ctypes.c_double, _dp, _dp]
        L.orc_return_map.argtypes = [ctypes.c_double, ctypes.c_double, _dp, _dp, _ip]
        L.orc_return_map.restype = ctypes.c_int
        L.orc_collider_pose.argtypes = [ctypes.POINTER(_Collider), ctypes.c_double, _dp, _dp, _dp]
        L.orc_collider_sdf.argtypes = [ctypes.POINTER(_Collider), ctypes.c_double, _dp, _dp, _ip]
        L.orc_collider_sdf.restype = ctypes.c_double
        L.orc_p2g.argtypes = [ctypes.POINTER(_Params), ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp]
        L.orc_grid_update.argtypes = [ctypes.POINTER(_Params), _dp, ctypes.c_int, ctypes.POINTER(_Collider),
                                      ctypes.c_double, _dp, _u8p]
        L.orc_g2p.argtypes = [ctypes.POINTER(_Params), ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _ip]
        L.orc_g2p.restype = ctypes.c_int
        L.orc_substep.argtypes = [ctypes.POINTER(_Params), ctypes.c_int, _dp, _dp, _dp, _dp, _dp,
                                  ctypes.c_int, ctypes.POINTER(_Collider), ctypes.c_double, _dp, _dp, _u8p]
        L.orc_substep.restype = ctypes.c_int
        L.orc_p2g_forces.argtypes = [ctypes.POINTER(_Params), ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
        L.orc_sdf_volume.argtypes = [ctypes.POINTER(_Collider), _dp, _dp, _dp, _ip]
        L.orc_sdf_volume.restype = ctypes.c_int
        L.orc_penalty_accel.argtypes = [ctypes.POINTER(_Params), ctypes.POINTER(_Penalty), ctypes.c_int, _dp, _dp,
                                        ctypes.c_int, ctypes.POINTER(_Collider), ctypes.c_double, _dp, _dp, _u8p]
        L.orc_penalty_accel.restype = ctypes.c_int
        L.orc_substep_penalty.argtypes = [ctypes.POINTER(_Params), ctypes.POINTER(_Penalty), ctypes.c_int, _dp, _dp,
                                          _dp, _dp, _dp, ctypes.c_int, ctypes.POINTER(_Collider), ctypes.c_double,
                                          _dp, _dp, _dp, _u8p]
        L.orc_substep_penalty.restype = ctypes.c_int
        L.orc_splat_depth.argtypes = [ctypes.POINTER(_Camera), ctypes.POINTER(_Render), ctypes.c_int, _dp, _dp, _u8p]
        L.orc_splat_depth.restype = ctypes.c_int
        L.orc_bilateral.argtypes = [ctypes.POINTER(_Camera), ctypes.POINTER(_Render), _dp, _dp]
        L.orc_shade.argtypes = [ctypes.POINTER(_Camera), ctypes.POINTER(_Render), _dp, _dp, _dp, _u8p]
        _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def lame(E: float, nu: float):
    """Lame parameters (mu, lambda) of Young's modulus E and Poisson ratio nu (Table 4 parameters)."""
    mu = ctypes.c_double()
    la = ctypes.c_double()
    lib().orc_lame(E, nu, ctypes.byref(mu), ctypes.byref(la))
    return mu.value, la.value


@dataclass
class Params:
    """Scene constants of one substep (see ``orc_params`` in ``mpm_oracle.h``)."""

    n: int
    dt: float
    gravity: tuple = (0.0, -9.8, 0.0)
    bound: int = 3
    kind: int = PLASTICINE
    E: float = 5e3
    nu: float = 0.3
    yield_stress: float = 50.0
    bulk_modulus: float = 1e4
    rho: float = 1e3
    p_vol: float = 1.0

    def c(self) -> _Params:
        if self.kind == PLASTICINE:
            mu, la = lame(self.E, self.nu)
        else:
            mu, la = 0.0, self.bulk_modulus
        return _Params(self.n, self.dt, (ctypes.c_double * 3)(*self.gravity), self.bound, self.kind, mu, la,
                       self.yield_stress, self.p_vol, self.rho * self.p_vol)


@dataclass
class Collider:
    """One kinematic collider (see ``orc_collider``); pose and velocities as set at t = 0.

    An SDF volume (type SDF_VOLUME) carries ``sdf`` of shape (nx, ny, nz), sample [i, j, k] at the
    shape-frame point ``sdf_origin + sdf_h * (i, j, k)``."""

    type: int
    half: tuple
    friction: float
    pos: tuple
    quat: tuple = (1.0, 0.0, 0.0, 0.0)
    lin_vel: tuple = (0.0, 0.0, 0.0)
    ang_vel: tuple = (0.0, 0.0, 0.0)
    com: tuple | None = None
    sdf: np.ndarray | None = None
    sdf_origin: tuple = (0.0, 0.0, 0.0)
    sdf_h: float = 1.0

    def c(self) -> _Collider:
        com = self.pos if self.com is None else self.com
        d3 = ctypes.c_double * 3
        col = _Collider(self.type, d3(*self.half), self.friction, d3(*self.pos),
                        (ctypes.c_double * 4)(*self.quat), d3(*self.lin_vel), d3(*self.ang_vel), d3(*com))
        if self.sdf is not None:
            # i fastest: element (i, j, k) at i + nx * (j + ny * k); kept alive on the object
            self._flat = np.ascontiguousarray(np.asarray(self.sdf, np.float64).transpose(2, 1, 0))
            col.sdf = self._flat.ctypes.data_as(_dp)
            col.res = (ctypes.c_int * 3)(*self.sdf.shape)
            col.sdf_origin = d3(*self.sdf_origin)
            col.sdf_h = self.sdf_h
        return col


@dataclass
class Penalty:
    """Constants of the particle contact (see ``orc_penalty``): stiffness 1/s^2, damping 1/s."""

    stiffness: float
    damping: float

    def c(self) -> _Penalty:
        return _Penalty(self.stiffness, self.damping)


def _cols(colliders):
    arr = (_Collider * max(1, len(colliders)))()
    for i, c in enumerate(colliders):
        arr[i] = c.c()
    return arr


@dataclass
class State:
    """FP64 particle state, structure of arrays: x (3,N), v (3,N), C (9,N), F (9,N) or J (N,)."""

    x: np.ndarray
    v: np.ndarray
    C: np.ndarray
    F: np.ndarray | None = None
    J: np.ndarray | None = None
    extra: dict = field(default_factory=dict)

    @staticmethod
    def from_arrays(x, v, C, F=None, J=None) -> "State":
        return State(_f64(x).copy(), _f64(v).copy(), _f64(C).copy(),
                     None if F is None else _f64(F).copy(), None if J is None else _f64(J).copy())

    @property
    def n(self) -> int:
        return self.x.shape[1]

    def copy(self) -> "State":
        return State.from_arrays(self.x, self.v, self.C, self.F, self.J)


# ------------------------------------------------------------------ single-step wrappers

def bspline(u: float) -> float:
    return lib().orc_bspline(float(u))


def stencil(n: int, x):
    """27-node stencil of one particle: (base[3], node index[27], weight[27], dpos[27,3])."""
    x = _f64(x)
    base = (ctypes.c_int * 3)()
    idx = (ctypes.c_int * 27)()
    w = np.zeros(27)
    d = np.zeros(81)
    lib().orc_stencil(n, _ptr(x), base, idx, _ptr(w), _ptr(d))
    return np.array(base[:]), np.array(idx[:]), w, d.reshape(27, 3)


def svd3(F):
    F = _f64(F).reshape(9)
    U = np.zeros(9); S = np.zeros(3); V = np.zeros(9)
    sweeps = lib().orc_svd3(_ptr(F), _ptr(U), _ptr(S), _ptr(V))
    return U.reshape(3, 3), S, V.reshape(3, 3), sweeps


def stress(mu: float, lam: float, F):
    """Fixed-corotated Kirchhoff stress of one deformation gradient."""
    F = _f64(F).reshape(9)
    tau = np.zeros(9)
    lib().orc_stress_fixed_corotated(mu, lam, _ptr(F), _ptr(tau))
    return tau.reshape(3, 3)


def return_map(mu: float, yield_stress: float, Ftr):
    """Von Mises return map in Hencky strain: (F_new, projected, clamped)."""
    Ftr = _f64(Ftr).reshape(9)
    out = np.zeros(9)
    cl = ctypes.c_int(0)
    proj = lib().orc_return_map(mu, yield_stress, _ptr(Ftr), _ptr(out), ctypes.byref(cl))
    return out.reshape(3, 3), bool(proj), bool(cl.value)


def collider_pose(col: Collider, t: float):
    c = col.c()
    R = np.zeros(9); p = np.zeros(3); com = np.zeros(3)
    lib().orc_collider_pose(ctypes.byref(c), t, _ptr(R), _ptr(p), _ptr(com))
    return R.reshape(3, 3), p, com


def collider_sdf(col: Collider, t: float, x):
    c = col.c()
    x = _f64(x)
    nrm = np.zeros(3)
    amb = ctypes.c_int(0)
    phi = lib().orc_collider_sdf(ctypes.byref(c), t, _ptr(x), _ptr(nrm), ctypes.byref(amb))
    return phi, nrm, bool(amb.value)


def p2g(params: Params, s: State) -> np.ndarray:
    """Step A1+A2: returns the dense grid (n,n,n,4): mass and momentum."""
    n = params.n
    grid = np.zeros(n * n * n * 4)
    P = params.c()
    lib().orc_p2g(ctypes.byref(P), s.n, _ptr(s.x), _ptr(s.v), _ptr(s.C), _ptr(s.F), _ptr(s.J), _ptr(grid))
    return grid.reshape(n, n, n, 4)


def grid_update(params: Params, grid, colliders=(), t: float = 0.0, wrench=None, want_ambiguous=False):
    """Step A3 on a copy of ``grid`` (n,n,n,4); returns (grid with velocities, wrench (k,6), ambiguous)."""
    n = params.n
    g = _f64(grid).reshape(-1).copy()
    k = len(colliders)
    w = np.zeros(6 * max(k, 1)) if wrench is None else _f64(wrench).reshape(-1).copy()
    amb = np.zeros(n ** 3, dtype=np.uint8) if want_ambiguous else None
    P = params.c()
    cols = _cols(colliders)
    lib().orc_grid_update(ctypes.byref(P), _ptr(g), k, cols, t, _ptr(w),
                          None if amb is None else amb.ctypes.data_as(_u8p))
    return g.reshape(n, n, n, 4), w[: 6 * k].reshape(k, 6), (None if amb is None else amb.reshape(n, n, n))


def g2p(params: Params, grid, s: State):
    """Steps A4+A5 in place on ``s``; returns (clamped coordinates, clamped singular values)."""
    g = _f64(grid).reshape(-1)
    P = params.c()
    svc = ctypes.c_int(0)
    ncl = lib().orc_g2p(ctypes.byref(P), s.n, _ptr(g), _ptr(s.x), _ptr(s.v), _ptr(s.C), _ptr(s.F), _ptr(s.J),
                        ctypes.byref(svc))
    return ncl, svc.value


def substep(params: Params, s: State, colliders=(), t: float = 0.0, wrench=None, want_ambiguous=False):
    """One full substep in place on ``s`` at collider time t.

    Returns (clamped coordinate count, wrench (k,6) accumulated onto ``wrench`` if given, ambiguous
    node mask or None)."""
    n = params.n
    grid = np.zeros(n ** 3 * 4)
    k = len(colliders)
    w = np.zeros(6 * max(k, 1)) if wrench is None else wrench.reshape(-1)
    amb = np.zeros(n ** 3, dtype=np.uint8) if want_ambiguous else None
    P = params.c()
    cols = _cols(colliders)
    ncl = lib().orc_substep(ctypes.byref(P), s.n, _ptr(s.x), _ptr(s.v), _ptr(s.C), _ptr(s.F), _ptr(s.J), k, cols,
                            t, _ptr(w), _ptr(grid), None if amb is None else amb.ctypes.data_as(_u8p))
    return ncl, w[: 6 * k].reshape(k, 6), (None if amb is None else amb.reshape(n, n, n))


def rollout(params: Params, s: State, nsub: int, colliders=(), t0: float = 0.0, wrench=None):
    """``nsub`` substeps in place; collider time advances by dt per substep from t0."""
    total = 0
    for k in range(nsub):
        ncl, wrench, _ = substep(params, s, colliders, t0 + k * params.dt, wrench)
        total += ncl
    return total, wrench


def surrogate_window(params: Params, s: State, dv, box, unit: float, k: int, colliders=(), t: float = 0.0):
    """One learned-surrogate window written out with the steps above (the surrogate is this project's
    extension; the paper has no learned component): the transfer of the state (step A1+A2), one grid
    update with the substep's dt (A3), the correction v += dv * unit at nodes with mass inside ``box``
    (zero in the sticky wall band), then grid-to-particle (A4+A5) with time step k*dt, in place on ``s``.

    dv: (D, H, W, 3) over box = (i0, j0, k0, D, H, W) in node indices. Returns a dict of the grid sums the
    fallback gate compares: M, P0 (before the grid update), P1 (after), P_hat (after the correction)."""
    n = params.n
    g0 = p2g(params, s)                       # (m, m v)
    g1, _, _ = grid_update(params, g0, colliders, t)  # (m, v)
    g2 = g1.copy()
    i0, j0, k0, D, H, W = box
    band = params.bound
    for i in range(max(i0, 0), min(i0 + D, n)):
        for j in range(max(j0, 0), min(j0 + H, n)):
            for kk in range(max(k0, 0), min(k0 + W, n)):
                if not g1[i, j, kk, 0] > 0.0:
                    continue
                v = g1[i, j, kk, 1:] + unit * np.asarray(dv[i - i0, j - j0, kk - k0], np.float64)
                if min(i, j, kk) < band or max(i, j, kk) >= n - band:
                    v = np.zeros(3)
                g2[i, j, kk, 1:] = v
    big = Params(**{**params.__dict__, "dt": params.dt * k})
    g2p(big, g2, s)
    return {"M": g0[..., 0].sum(), "P0": g0[..., 1:].reshape(-1, 3).sum(axis=0),
            "P1": (g1[..., :1] * g1[..., 1:]).reshape(-1, 3).sum(axis=0),
            "P_hat": (g2[..., :1] * g2[..., 1:]).reshape(-1, 3).sum(axis=0)}


# ------------------------------------------------------------------ particle contact (Sec. 3's default form)

def sdf_volume(col: Collider, l):
    """Trilinear value and gradient of ``col``'s SDF volume at the shape-frame point l, or None outside
    the lattice: (phi, grad (3,), ambiguous)."""
    c = col.c()
    l = _f64(l)
    phi = ctypes.c_double(0.0)
    g = np.zeros(3)
    amb = ctypes.c_int(0)
    inside = lib().orc_sdf_volume(ctypes.byref(c), _ptr(l), ctypes.byref(phi), _ptr(g), ctypes.byref(amb))
    return (phi.value, g, bool(amb.value)) if inside else None


def penalty_accel(params: Params, pen: Penalty, s: State, colliders=(), t: float = 0.0):
    """Penalty accelerations (3, N), the wrench (k, 6) they put on the bodies, the ambiguous-particle mask
    and the number of contacts."""
    k = len(colliders)
    acc = np.zeros((3, s.n))
    w = np.zeros(6 * max(k, 1))
    amb = np.zeros(s.n, dtype=np.uint8)
    P, Pe = params.c(), pen.c()
    cols = _cols(colliders)
    nc = lib().orc_penalty_accel(ctypes.byref(P), ctypes.byref(Pe), s.n, _ptr(s.x), _ptr(s.v), k, cols, t,
                                 _ptr(acc), _ptr(w), amb.ctypes.data_as(_u8p))
    return acc, w[: 6 * k].reshape(k, 6), amb.astype(bool), nc


def p2g_forces(params: Params, s: State, accel) -> np.ndarray:
    """P2G with external particle accelerations (3, N): the dense grid (n,n,n,4)."""
    n = params.n
    grid = np.zeros(n * n * n * 4)
    a = _f64(accel)
    P = params.c()
    lib().orc_p2g_forces(ctypes.byref(P), s.n, _ptr(s.x), _ptr(s.v), _ptr(s.C), _ptr(s.F), _ptr(s.J), _ptr(a),
                         _ptr(grid))
    return grid.reshape(n, n, n, 4)


def substep_penalty(params: Params, pen: Penalty, s: State, colliders=(), t: float = 0.0, wrench=None):
    """One substep with the particle contact, in place on ``s`` at collider time t.

    Returns (clamped coordinate count, wrench (k,6) accumulated onto ``wrench`` if given, ambiguous
    particle mask)."""
    n = params.n
    grid = np.zeros(n ** 3 * 4)
    acc = np.zeros(3 * s.n)
    k = len(colliders)
    w = np.zeros(6 * max(k, 1)) if wrench is None else wrench.reshape(-1)
    amb = np.zeros(s.n, dtype=np.uint8)
    P, Pe = params.c(), pen.c()
    cols = _cols(colliders)
    ncl = lib().orc_substep_penalty(ctypes.byref(P), ctypes.byref(Pe), s.n, _ptr(s.x), _ptr(s.v), _ptr(s.C),
                                    _ptr(s.F), _ptr(s.J), k, cols, t, _ptr(w), _ptr(grid), _ptr(acc),
                                    amb.ctypes.data_as(_u8p))
    return ncl, w[: 6 * k].reshape(k, 6), amb.astype(bool)


def rollout_penalty(params: Params, pen: Penalty, s: State, nsub: int, colliders=(), t0: float = 0.0,
                    wrench=None):
    """``nsub`` particle-contact substeps in place; collider time advances by dt per substep from t0.
    Returns (clamped count, wrench, mask of particles that were ambiguous in any substep)."""
    total = 0
    amb_any = np.zeros(s.n, dtype=bool)
    for k in range(nsub):
        ncl, wrench, amb = substep_penalty(params, pen, s, colliders, t0 + k * params.dt, wrench)
        total += ncl
        amb_any |= amb
    return total, wrench, amb_any


# ------------------------------------------------------------------ particle renderer (App. D.2)

@dataclass
class Camera:
    """Pinhole camera (see ``orc_camera``): rot is world -> camera (x right, y down, z forward)."""

    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    eye: tuple
    rot: np.ndarray
    near_z: float = 1e-3

    def c(self) -> _Camera:
        return _Camera(self.width, self.height, self.fx, self.fy, self.cx, self.cy, (ctypes.c_double * 3)(*self.eye),
                       (ctypes.c_double * 9)(*np.asarray(self.rot, np.float64).reshape(9)), self.near_z)


@dataclass
class RenderParams:
    """Splatting, filter and shading constants (see ``orc_render``)."""

    radius: float
    smooth: float
    sigma_depth: float
    window: int
    light: tuple = (0.3, -0.6, -0.75)
    albedo: tuple = (0.85, 0.6, 0.4)
    ambient: float = 0.25
    background: tuple = (0.0, 0.0, 0.0)

    def c(self) -> _Render:
        d3 = ctypes.c_double * 3
        return _Render(self.radius, self.smooth, self.sigma_depth, self.window, d3(*self.light), d3(*self.albedo),
                       self.ambient, d3(*self.background))


def splat_depth(cam: Camera, rp: RenderParams, x):
    """Step 1: (depth (H, W), ambiguous mask (H, W), particles drawn)."""
    x = _f64(x)
    n = x.shape[1]
    depth = np.zeros(cam.width * cam.height)
    amb = np.zeros(cam.width * cam.height, np.uint8)
    C, Rr = cam.c(), rp.c()
    drawn = lib().orc_splat_depth(ctypes.byref(C), ctypes.byref(Rr), n, _ptr(x), _ptr(depth), amb.ctypes.data_as(_u8p))
    return depth.reshape(cam.height, cam.width), amb.reshape(cam.height, cam.width).astype(bool), drawn


def bilateral(cam: Camera, rp: RenderParams, depth):
    """Step 2: the smoothed depth (H, W)."""
    d = _f64(depth).reshape(-1)
    out = np.zeros_like(d)
    C, Rr = cam.c(), rp.c()
    lib().orc_bilateral(ctypes.byref(C), ctypes.byref(Rr), _ptr(d), _ptr(out))
    return out.reshape(cam.height, cam.width)


def shade(cam: Camera, rp: RenderParams, smoothed):
    """Steps 3 and 4: (normals (H, W, 3), rgb (H, W, 3), ambiguous mask (H, W))."""
    z = _f64(smoothed).reshape(-1)
    nrm = np.zeros(3 * z.size)
    rgb = np.zeros(3 * z.size)
    amb = np.zeros(z.size, np.uint8)
    C, Rr = cam.c(), rp.c()
    lib().orc_shade(ctypes.byref(C), ctypes.byref(Rr), _ptr(z), _ptr(nrm), _ptr(rgb), amb.ctypes.data_as(_u8p))
    H, W = cam.height, cam.width
    return nrm.reshape(H, W, 3), rgb.reshape(H, W, 3), amb.reshape(H, W).astype(bool)
