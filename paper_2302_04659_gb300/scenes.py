"""Seeded synthetic inputs for the MPM substep: particle clouds, states and collider scripts.

This module only generates inputs. It holds none of the method's arithmetic
(no weights, stress, transfer or contact), so both the FP64 oracle and the CUDA
path can be fed from it without sharing any of the computation.

Random numbers come from splitmix64 (Steele, Lea & Flood 2014) used as a
counter-based generator: the i-th 64-bit word of stream ``seed`` is
``mix(seed + (i + 1) * 0x9E3779B97F4A7C15)``; a double in [0, 1) takes its top
53 bits. Every state is generated in FP64 and rounded to FP32, and those FP32
values are what both sides consume.

Workloads (the paper's soft-body tasks and assets are not available, so these
synthetic scenes stand in for the Pinch and Pour scenes of Sec. 2 / App. C;
parameters follow the ranges of Table 4 where the workload does not fix them):
  * ``cube_scene``   -- 32^3 grid, 8,192 particles stratified-jittered in a
    0.25-side plasticine cube, rho 1e3, E 5e3, nu 0.3, yield 50, dt 2e-4.
  * ``pinch_scene``  -- 64^3 grid, 200,000 particles uniform in a seeded
    ellipsoid of plasticine, two kinematic capsule fingers (radius 0.02) closing
    on seeded sinusoidal paths, friction 0.5, 25 substeps per env step.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

PLASTICINE = 0
FLUID = 1
BOX = 0
CAPSULE = 1
SDF_VOLUME = 2


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Words ``offset .. offset+count-1`` of the splitmix64 stream ``seed`` (uint64)."""
    i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of each word."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Standard normal variates by the Box-Muller transform of pairs of uniforms."""
    u = uniform(seed, 2 * count, 2 * offset)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


@dataclass
class Material:
    kind: int = PLASTICINE
    rho: float = 1e3
    E: float = 5e3
    nu: float = 0.3
    yield_stress: float = 50.0
    bulk_modulus: float = 1e4
    p_vol: float = 1.0


@dataclass
class Shape:
    """Collider shape: box half extents, or capsule (radius, half length along local z, 0), or an SDF
    volume: ``sdf`` (nx, ny, nz) FP32 samples, [i, j, k] at ``sdf_origin + sdf_h * (i, j, k)`` in the
    shape frame."""

    type: int
    half: tuple
    friction: float
    sdf: np.ndarray | None = None
    sdf_origin: tuple = (0.0, 0.0, 0.0)
    sdf_h: float = 1.0


@dataclass
class Scene:
    n: int
    dt: float
    material: Material
    x: np.ndarray                      # (3, N) float32
    v: np.ndarray                      # (3, N) float32
    C: np.ndarray                      # (9, N) float32
    F: np.ndarray                      # (9, N) float32 (identity for a fresh body)
    gravity: tuple = (0.0, -9.8, 0.0)
    bound: int = 3
    shapes: list = field(default_factory=list)
    substeps_per_env_step: int = 25
    script: dict = field(default_factory=dict)   # collider path parameters

    @property
    def N(self) -> int:
        return self.x.shape[1]


def _identity_F(N: int) -> np.ndarray:
    F = np.zeros((9, N), dtype=np.float32)
    F[0] = F[4] = F[8] = 1.0
    return F


def cube_particles(lower, side: float, lattice=(16, 16, 32), seed: int = 1) -> np.ndarray:
    """One jittered sample per sub-cell of a ``lattice`` over an axis-aligned cube (FP32, (3, N))."""
    nx, ny, nz = lattice
    N = nx * ny * nz
    u = uniform(seed, 3 * N).reshape(N, 3)
    ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    cell = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1).astype(np.float64)
    size = np.array([side / nx, side / ny, side / nz])
    x = np.asarray(lower, dtype=np.float64)[None, :] + (cell + u) * size[None, :]
    return np.ascontiguousarray(x.T.astype(np.float32))


def cube_scene(variant: str = "floor", seed: int = 1) -> Scene:
    """The 32^3 / 8,192-particle plasticine cube.

    ``floor``: lower face at y = 3.25 dx so the first layer rests against the sticky floor band.
    ``ff``:    centred (lower face at y = 0.375), free fall for the whole 50-substep rollout.
    ``rand``:  the ``floor`` positions with random v ~ N(0, 0.5^2), C ~ N(0, 5^2),
               F = I + N(0, 0.05^2) (seed 2), to exercise every branch in one substep.
    """
    n = 32
    dx = 1.0 / n
    side = 0.25
    ylow = 0.375 if variant == "ff" else 3.25 * dx
    x = cube_particles((0.375, ylow, 0.375), side, seed=seed)
    N = x.shape[1]
    mat = Material(PLASTICINE, rho=1e3, E=5e3, nu=0.3, yield_stress=50.0, p_vol=side ** 3 / N)
    v = np.zeros((3, N), np.float32)
    C = np.zeros((9, N), np.float32)
    F = _identity_F(N)
    if variant == "rand":
        v, C, F = random_state(N, seed=2)
    return Scene(n=n, dt=2e-4, material=mat, x=x, v=v, C=C, F=F, substeps_per_env_step=50)


def random_state(N: int, seed: int, v_std: float = 0.5, C_std: float = 5.0, F_std: float = 0.05):
    """Random v, C and F = I + noise (det F > 0 is checked), rounded to FP32."""
    z = normal(seed, 21 * N).reshape(21, N)
    v = (v_std * z[0:3]).astype(np.float32)
    C = (C_std * z[3:12]).astype(np.float32)
    F = (np.eye(3).reshape(9, 1) + F_std * z[12:21]).astype(np.float32)
    det = np.linalg.det(F.T.reshape(N, 3, 3).astype(np.float64))
    if not np.all(det > 0):
        raise ValueError("random deformation gradient with det <= 0; lower F_std")
    return v, C, F


def ellipsoid_particles(N: int, center, semi, seed: int) -> np.ndarray:
    """N points uniform in an axis-aligned ellipsoid by rejection from its bounding box (FP32, (3, N))."""
    center = np.asarray(center, np.float64)
    semi = np.asarray(semi, np.float64)
    if N == 0:
        return np.zeros((3, 0), np.float32)
    out = []
    have = 0
    offset = 0
    while have < N:
        m = 2 * (N - have) + 1024
        u = uniform(seed, 3 * m, offset).reshape(m, 3)
        offset += 3 * m
        p = 2.0 * u - 1.0
        keep = p[(p * p).sum(axis=1) < 1.0]
        out.append(keep)
        have += len(keep)
    p = np.concatenate(out)[:N]
    x = center[None, :] + p * semi[None, :]
    return np.ascontiguousarray(x.T.astype(np.float32))


def pinch_scene(seed: int = 1000, N: int = 200_000, n: int = 64) -> Scene:
    """Plasticine pinch: a seeded ellipsoid on the floor band and two capsule fingers closing along x.

    Semi-axes ~ U[0.18, 0.26]^3, centre (0.5, 3 dx + b, 0.5). Each finger is a capsule of radius 0.02
    and half length 0.05 with its axis along world x (tips facing each other), starting 0.01 outside
    the ellipsoid at its mid height. Finger c moves as c0 +- x A (1 - cos 2 pi f t) / 2 with
    A ~ U[0.05, 0.12], f ~ U[1, 3] Hz, friction 0.5.
    """
    dx = 1.0 / n
    u = uniform(seed, 8, offset=0)
    semi = 0.18 + 0.08 * u[0:3]
    center = (0.5, 3 * dx + semi[1], 0.5)
    x = ellipsoid_particles(N, center, semi, seed=seed + 1)
    vol = 4.0 / 3.0 * math.pi * semi[0] * semi[1] * semi[2]
    mat = Material(PLASTICINE, rho=1e3, E=5e3, nu=0.3, yield_stress=50.0, p_vol=vol / N)
    r, h = 0.02, 0.05
    amp = 0.05 + 0.07 * u[3:5]
    freq = 1.0 + 2.0 * u[5:7]
    shapes = [Shape(CAPSULE, (r, h, 0.0), 0.5), Shape(CAPSULE, (r, h, 0.0), 0.5)]
    c0 = [
        (0.5 - (semi[0] + 0.01 + h + r), center[1], 0.5),
        (0.5 + (semi[0] + 0.01 + h + r), center[1], 0.5),
    ]
    s = math.sqrt(0.5)
    script = {
        "c0": np.array(c0),
        "dir": np.array([1.0, -1.0]),
        "amp": amp,
        "freq": freq,
        "quat": np.array([[s, 0.0, s, 0.0], [s, 0.0, s, 0.0]]),  # local z -> world x
    }
    return Scene(n=n, dt=2e-4, material=mat, x=x, v=np.zeros((3, N), np.float32),
                 C=np.zeros((9, N), np.float32), F=_identity_F(N), shapes=shapes, script=script,
                 substeps_per_env_step=25)


def finger_state(scene: Scene, t: float):
    """Collider inputs at time t of a scripted scene.

    Returns float32 arrays pose (k,7: position, quaternion w x y z), lin_vel (k,3), ang_vel (k,3),
    com (k,3)."""
    sc = scene.script
    k = len(sc["c0"])
    pose = np.zeros((k, 7))
    lin = np.zeros((k, 3))
    ang = np.zeros((k, 3)) if "ang" not in sc else np.asarray(sc["ang"], np.float64)
    for i in range(k):
        A, f = sc["amp"][i], sc["freq"][i]
        axis = np.asarray(sc["axis"][i], np.float64) if "axis" in sc else np.array([sc["dir"][i], 0.0, 0.0])
        pose[i, :3] = sc["c0"][i] + axis * A * (1.0 - math.cos(2 * math.pi * f * t)) / 2.0
        pose[i, 3:] = _quat_mul(_quat_of_rotvec(ang[i] * t), np.asarray(sc["quat"][i], np.float64))
        lin[i] = axis * A * math.pi * f * math.sin(2 * math.pi * f * t)
    return (pose.astype(np.float32), lin.astype(np.float32), ang.astype(np.float32),
            pose[:, :3].astype(np.float32))


def _quat_of_rotvec(r) -> np.ndarray:
    """Unit quaternion (w, x, y, z) of the rotation by |r| about r."""
    a = float(np.linalg.norm(r))
    if a == 0.0:
        return np.array([1.0, 0.0, 0.0, 0.0])
    return np.concatenate([[math.cos(a / 2)], math.sin(a / 2) * np.asarray(r) / a])


def _quat_mul(p, q) -> np.ndarray:
    """Hamilton product p q (apply q, then p)."""
    w1, v1 = p[0], np.asarray(p[1:])
    w2, v2 = q[0], np.asarray(q[1:])
    return np.concatenate([[w1 * w2 - v1 @ v2], w1 * v2 + w2 * v1 + np.cross(v1, v2)])


# ---------------------------------------------------------------------------- SDF volumes

def torus_volume(R: float, r: float, h: float, pad: int = 2):
    """Signed distances of a torus about local z (ring radius R, tube radius r) sampled on a lattice
    of spacing h covering it with ``pad`` samples to spare: (samples (nx, ny, nz) FP32, origin).
    A stand-in for a mesh's SDF volume (Sec. 3): a shape no primitive describes."""
    ext = np.array([R + r, R + r, r]) + pad * h
    res = tuple(int(math.ceil(2 * e / h)) + 1 for e in ext)
    origin = tuple(-(res[a] - 1) * h / 2 for a in range(3))
    ii = np.indices(res).astype(np.float64)
    x, y, z = (origin[a] + h * ii[a] for a in range(3))
    d = np.sqrt((np.sqrt(x * x + y * y) - R) ** 2 + z * z) - r
    return d.astype(np.float32), origin


def ring_press_scene(seed: int = 4000, N: int = 50_000, n: int = 64) -> Scene:
    """A plasticine ellipsoid (as the pinch scene's) pressed by a spinning ring tool held as an SDF
    volume: a torus with R ~ U[0.06, 0.09], r ~ U[0.02, 0.03], sampled at half the grid spacing, its axis
    tilted by up to 0.4 rad from vertical, starting 0.01 above the body and pressing down along -y as
    c0 - y A (1 - cos 2 pi f t) / 2 (A ~ U[0.05, 0.1], f ~ U[1, 3] Hz) while it spins about world y at
    w ~ U[-4, 4] rad/s; friction 0.5."""
    dx = 1.0 / n
    u = uniform(seed, 12, offset=0)
    semi = 0.16 + 0.06 * u[0:3]
    center = (0.5, 3 * dx + semi[1], 0.5)
    x = ellipsoid_particles(N, center, semi, seed=seed + 1)
    vol = 4.0 / 3.0 * math.pi * semi[0] * semi[1] * semi[2]
    mat = Material(PLASTICINE, rho=1e3, E=5e3, nu=0.3, yield_stress=50.0, p_vol=vol / N)
    R = 0.06 + 0.03 * u[3]
    r = 0.02 + 0.01 * u[4]
    samples, origin = torus_volume(R, r, 0.5 * dx)
    tilt = 0.4 * (u[5:7] - 0.5) * 2
    q0 = _quat_mul(_quat_of_rotvec([tilt[0], 0.0, tilt[1]]), _quat_of_rotvec([-math.pi / 2, 0.0, 0.0]))
    shapes = [Shape(SDF_VOLUME, (0.0, 0.0, 0.0), 0.5, sdf=samples, sdf_origin=origin, sdf_h=0.5 * dx)]
    c0 = [(0.5 + 0.02 * (u[7] - 0.5), center[1] + semi[1] + 0.01 + r, 0.5 + 0.02 * (u[8] - 0.5))]
    script = {"c0": np.array(c0), "axis": np.array([[0.0, -1.0, 0.0]]), "amp": np.array([0.05 + 0.05 * u[9]]),
              "freq": np.array([1.0 + 2.0 * u[10]]), "quat": np.array([q0]),
              "ang": np.array([[0.0, 8.0 * (u[11] - 0.5), 0.0]])}
    return Scene(n=n, dt=2e-4, material=mat, x=x, v=np.zeros((3, N), np.float32),
                 C=np.zeros((9, N), np.float32), F=_identity_F(N), shapes=shapes, script=script,
                 substeps_per_env_step=25)


# ---------------------------------------------------------------------------- batched workloads

def box_particles(N: int, lower, size, seed: int) -> np.ndarray:
    """N points uniform in an axis-aligned box (FP32, (3, N))."""
    u = uniform(seed, 3 * N).reshape(N, 3)
    x = np.asarray(lower, np.float64)[None, :] + u * np.asarray(size, np.float64)[None, :]
    return np.ascontiguousarray(x.T.astype(np.float32))


def tool_scene(seed: int, kind: int, N: int, n: int = 64, extra_capsule: bool = False) -> Scene:
    """One environment of the batched workloads: a body on the floor band and a moving box tool.

    The tool is a box with half extents ~ U[0.03, 0.08]^3 and friction 0.5, moving along a seeded
    direction (a main axis plus lateral components ~ U[-0.3, 0.3], normalised) as
    c0 + d A (1 - cos 2 pi f t) / 2, A ~ U[0.05, 0.12], f ~ U[1, 3] Hz.
    Plasticine: a seeded ellipsoid (semi-axes ~ U[0.12, 0.2]^3, centred in x and z, resting on the band
    at 3 dx); the tool starts 0.01 above it and presses down (main axis -y). Tool centres are offset by
    U[-0.02, 0.02] in x and z from the mid-plane (no node sits where the box's face normal flips sign).
    Fluid: a seeded block of water (half extents ~ U[0.1, 0.2]^3, centred in x and z, on the band); the
    tool starts 0.01 outside its -x face, its bottom 0.03 above the band, and sweeps along +x.
    With ``extra_capsule`` a capsule finger (radius 0.02, half length 0.05, along x) closes in from the +x
    side at mid height, as in the pinch scene.
    """
    dx = 1.0 / n
    u = uniform(seed, 16, offset=0)
    A = 0.05 + 0.07 * u[3]
    f = 1.0 + 2.0 * u[4]
    half = tuple(float(h) for h in 0.03 + 0.05 * u[7:10])
    lateral = -0.3 + 0.6 * u[10:12]
    off = 0.04 * (u[12:14] - 0.5)  # tool centre off the mid-plane nodes (no sign ties inside the box)
    q_id = [1.0, 0.0, 0.0, 0.0]
    floor = 3 * dx
    if kind == PLASTICINE:
        semi = 0.12 + 0.08 * u[0:3]
        center = (0.5, floor + semi[1], 0.5)
        x = ellipsoid_particles(N, center, semi, seed=seed + 1)
        vol = 4.0 / 3.0 * math.pi * semi[0] * semi[1] * semi[2]
        mat = Material(PLASTICINE, rho=1e3, E=5e3, nu=0.3, yield_stress=50.0, p_vol=vol / max(N, 1))
        c0 = [(0.5 + off[0], center[1] + semi[1] + 0.01 + half[1], 0.5 + off[1])]
        d = np.array([lateral[0], -1.0, lateral[1]])
        mid_y, side_x = center[1], 0.5 + semi[0]
    else:
        hw = 0.1 + 0.1 * u[0:3]
        lower = (0.5 - hw[0], floor, 0.5 - hw[2])
        size = 2.0 * hw
        x = box_particles(N, lower, size, seed=seed + 1)
        vol = float(np.prod(size))
        mat = Material(FLUID, rho=1e3, bulk_modulus=1e4, p_vol=vol / max(N, 1))
        c0 = [(lower[0] - half[0] - 0.01, floor + 0.03 + half[1], 0.5 + off[1])]
        d = np.array([1.0, lateral[0], lateral[1]])
        mid_y, side_x = floor + hw[1], lower[0] + size[0]
    axis = [tuple(d / np.linalg.norm(d))]
    shapes = [Shape(BOX, half, 0.5)]
    quat = [q_id]
    amp, freq = [A], [f]
    if extra_capsule:
        r, h = 0.02, 0.05
        s2 = math.sqrt(0.5)
        shapes.append(Shape(CAPSULE, (r, h, 0.0), 0.5))
        c0.append((side_x + 0.01 + h + r, mid_y, 0.5))
        axis.append((-1.0, 0.0, 0.0))
        quat.append([s2, 0.0, s2, 0.0])
        amp.append(0.05 + 0.07 * u[5])
        freq.append(1.0 + 2.0 * u[6])
    script = {"c0": np.array(c0), "axis": np.array(axis), "amp": np.array(amp), "freq": np.array(freq),
              "quat": np.array(quat)}
    return Scene(n=n, dt=2e-4, material=mat, x=x, v=np.zeros((3, N), np.float32),
                 C=np.zeros((9, N), np.float32), F=_identity_F(N), shapes=shapes, script=script,
                 substeps_per_env_step=25)


def batch_counts(nenv: int, seed: int, lo: int, hi: int, log_uniform: bool = False) -> np.ndarray:
    """Seeded particle counts per env: uniform in [lo, hi], or log-uniform over that range."""
    u = uniform(seed, nenv)
    if log_uniform:
        c = np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))
    else:
        c = lo + u * (hi - lo + 1)
    return np.clip(np.floor(c), lo, hi).astype(np.int64)


def batch_workload(nenv: int = 256, seed: int = 2000, n: int = 64, lo: int = 20_000, hi: int = 120_000,
                   counts=None) -> list:
    """Many independent envs with their own n^3 grids: counts uniform in [lo, hi] from the seed, the first
    half plasticine and the second half fluid, one moving box tool each (``tool_scene``)."""
    counts = batch_counts(nenv, seed, lo, hi) if counts is None else counts
    return [tool_scene(seed + 7919 * (e + 1), PLASTICINE if e < nenv // 2 else FLUID, int(counts[e]), n)
            for e in range(nenv)]


def serving_workload(nenv: int = 1024, seed: int = 3000, lo: int = 2_000, hi: int = 200_000,
                     grids=(48, 64, 80, 96)) -> list:
    """The serving mix: counts log-uniform in [lo, hi], grid sizes drawn from ``grids``, plasticine and
    fluid alternating, each env with a box tool and a capsule finger."""
    counts = batch_counts(nenv, seed, lo, hi, log_uniform=True)
    g = uniform(seed + 1, nenv)
    return [tool_scene(seed + 7919 * (e + 1), PLASTICINE if e % 2 == 0 else FLUID, int(counts[e]),
                       int(grids[min(int(g[e] * len(grids)), len(grids) - 1)]), extra_capsule=True)
            for e in range(nenv)]


def concat_states(envs: list):
    """Concatenated (x, v, C, F) SoA arrays of a list of scenes, in env order, and the counts."""
    counts = [sc.N for sc in envs]
    cat = [np.ascontiguousarray(np.concatenate([getattr(sc, k) for sc in envs], axis=1)) for k in "xvCF"]
    return counts, cat


def concat_tool_states(envs: list, t: float):
    """Concatenated collider inputs (pose, lin, ang, com) of all envs at time t."""
    parts = [finger_state(sc, t) for sc in envs if sc.shapes]
    if not parts:
        z = np.zeros((0, 3), np.float32)
        return np.zeros((0, 7), np.float32), z, z, z
    return tuple(np.ascontiguousarray(np.concatenate([p[i] for p in parts])) for i in range(4))


class ToolPaths:
    """The scripted collider paths of many envs stacked into arrays: ``at(t)`` gives the concatenated
    collider inputs of all envs (the same values as ``concat_tool_states``) in one vectorised pass."""

    def __init__(self, envs: list):
        c0, axis, amp, freq, quat = [], [], [], [], []
        for sc in envs:
            s = sc.script
            for i in range(len(sc.shapes)):
                c0.append(s["c0"][i])
                axis.append(s["axis"][i] if "axis" in s else (s["dir"][i], 0.0, 0.0))
                amp.append(s["amp"][i])
                freq.append(s["freq"][i])
                quat.append(s["quat"][i])
        self.k = len(c0)
        self.c0 = np.asarray(c0, np.float64).reshape(-1, 3)
        self.axis = np.asarray(axis, np.float64).reshape(-1, 3)
        self.amp = np.asarray(amp, np.float64)
        self.freq = np.asarray(freq, np.float64)
        self.quat = np.asarray(quat, np.float64).reshape(-1, 4)

    def at(self, t: float):
        ph = 2 * math.pi * self.freq * t
        pos = self.c0 + self.axis * (self.amp * (1.0 - np.cos(ph)) / 2.0)[:, None]
        lin = self.axis * (self.amp * math.pi * self.freq * np.sin(ph))[:, None]
        pose = np.concatenate([pos, self.quat], axis=1).astype(np.float32)
        return (np.ascontiguousarray(pose), np.ascontiguousarray(lin.astype(np.float32)),
                np.zeros((self.k, 3), np.float32), np.ascontiguousarray(pos.astype(np.float32)))
