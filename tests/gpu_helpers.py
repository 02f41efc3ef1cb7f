"""Shared helpers of the GPU parity tests: build the scene on both sides from the same FP32 arrays.

The CUDA side is driven through the C-ABI binding; the oracle side gets the same
FP32 values widened to FP64. Nothing here computes any part of the method.
"""
import numpy as np

import oracle
from paper_2302_04659_gb300 import scenes

# Tolerances of the parity tests (relative L2 error over all particles, e = |a - b| / |b|).
# Positions and velocities: the 1e-4 per-substep bound the method is held to. C and F: the same
# bound; F is also compared relative to |F|, where FP32 storage of F ~ I rounds at ~6e-8.
TOL_X = 1e-4
TOL_V = 1e-4
TOL_C = 1e-4
TOL_F = 1e-5


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def rel_C(C, C_ref, v_ref, dx):
    """Error of the affine velocity C relative to its natural scale, |C_ref| + |v_ref| / dx: C is a
    velocity gradient gathered from node velocities with weights summing to a cancellation, so its FP32
    rounding error scales with |v| / dx even where C itself is near zero (e.g. free fall)."""
    C = np.asarray(C, np.float64)
    C_ref = np.asarray(C_ref, np.float64)
    scale = np.linalg.norm(C_ref) + np.linalg.norm(np.asarray(v_ref, np.float64)) / dx
    return np.linalg.norm(C - C_ref) / (scale if scale > 0 else 1.0)


def oracle_params(sc: scenes.Scene) -> oracle.Params:
    m = sc.material
    return oracle.Params(n=sc.n, dt=sc.dt, gravity=tuple(sc.gravity), bound=sc.bound, kind=m.kind, E=m.E, nu=m.nu,
                         yield_stress=m.yield_stress, bulk_modulus=m.bulk_modulus, rho=m.rho, p_vol=m.p_vol)


def oracle_state(sc: scenes.Scene, x=None, v=None, C=None, F=None) -> oracle.State:
    x = sc.x if x is None else x
    v = sc.v if v is None else v
    C = sc.C if C is None else C
    F = sc.F if F is None else F
    if sc.material.kind == scenes.FLUID:
        J = np.linalg.det(np.asarray(F, np.float32).T.reshape(-1, 3, 3).astype(np.float64))
        return oracle.State.from_arrays(x, v, C, None, J)
    return oracle.State.from_arrays(x, v, C, F)


def oracle_colliders(sc: scenes.Scene, pose, lin, ang, com):
    cols = []
    for i, sh in enumerate(sc.shapes):
        vol = {}
        if getattr(sh, "sdf", None) is not None:  # the same FP32 samples, widened
            vol = dict(sdf=np.asarray(sh.sdf, np.float32).astype(np.float64),
                       sdf_origin=tuple(float(np.float32(a)) for a in sh.sdf_origin),
                       sdf_h=float(np.float32(sh.sdf_h)))
        cols.append(oracle.Collider(sh.type, tuple(float(h) for h in sh.half), float(sh.friction),
                                    tuple(float(a) for a in pose[i, :3]), tuple(float(a) for a in pose[i, 3:]),
                                    tuple(float(a) for a in lin[i]), tuple(float(a) for a in ang[i]),
                                    tuple(float(a) for a in com[i]), **vol))
    return cols


def stencil_neighbours(x, n, bad):
    """Particles whose 27-node stencil shares a node with the stencil of a particle in ``bad``."""
    base = np.floor(np.asarray(x, np.float64) * n - 0.5).astype(np.int64)  # (3, N)
    out = np.zeros(base.shape[1], bool)
    for q in np.flatnonzero(bad):
        out |= np.all(np.abs(base - base[:, q:q + 1]) <= 2, axis=0)
    return out


def make_sim(sc: scenes.Scene, max_particles=None):
    from paper_2302_04659_gb300.sim import Sim
    return Sim(sc.n, sc.dt, sc.material, max_particles or max(sc.N, 1), gravity=sc.gravity, bound=sc.bound,
               max_colliders=max(len(sc.shapes), 1))


def fluid_scene(seed=77, N=6000, n=32):
    """A box of water (J-only fluid) with random velocities and affine C, for parity of the fluid branch."""
    dx = 1.0 / n
    x = scenes.cube_particles((0.3, 3.5 * dx, 0.3), 0.3, lattice=(20, 15, 20), seed=seed)[:, :N]
    N = x.shape[1]
    v, C, F = scenes.random_state(N, seed + 1, v_std=0.3, C_std=2.0, F_std=0.03)
    mat = scenes.Material(scenes.FLUID, rho=1e3, bulk_modulus=1e4, p_vol=0.3 ** 3 / N)
    return scenes.Scene(n=n, dt=2e-4, material=mat, x=x, v=v, C=C, F=F)


def stats(x, v, m):
    """Aggregate rollout statistics: centre of mass, momentum, kinetic energy, bounding box."""
    x = np.asarray(x, np.float64)
    v = np.asarray(v, np.float64)
    return {
        "com": x.mean(1),
        "p": m * v.sum(1),
        "ke": 0.5 * m * (v ** 2).sum(),
        "lo": x.min(1),
        "hi": x.max(1),
    }


def chamfer(a, b, chunk=2048):
    """Symmetric Chamfer distance (mean nearest-neighbour distance both ways) of two point sets (3,N)."""
    from scipy.spatial import cKDTree
    a = np.asarray(a, np.float64).T
    b = np.asarray(b, np.float64).T
    da, _ = cKDTree(b).query(a)
    db, _ = cKDTree(a).query(b)
    return 0.5 * (da.mean() + db.mean())
