"""``Sim`` (one soft-body scene) and ``BatchSim`` (many independent scenes advanced by the same
launches) on the GPU, driven through the C-ABI with PyTorch memory and streams.

PyTorch only supplies the device workspace and the current CUDA stream; every
step of the substep runs in the CUDA library (``_native``). Host arrays may be
numpy or CPU tensors, device arrays CUDA tensors; all are FP32 SoA with the
particle index fastest (x (3,N), v (3,N), C (9,N), F (9,N)).
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native as mpm


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _dev_ptr(t):
    if t is None:
        return 0
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError("device arrays must be contiguous float32 CUDA tensors")
    return t.data_ptr()


def _material(m) -> "mpm.mpm_material":
    return mpm.mpm_material(m.kind, m.rho, m.E, m.nu, m.yield_stress, m.bulk_modulus, m.p_vol)


class _Handle:
    """Calls shared by the single-scene and the batched handle."""

    handle = 0

    def close(self):
        if getattr(self, "handle", 0):
            torch.cuda.synchronize(self.device)
            mpm.mpm_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def N(self) -> int:
        return mpm.mpm_num_particles(self.handle)

    # ------------------------------------------------------------------ state
    def read_state(self, on_device: bool = True, stream=None):
        N = self.N
        if on_device:
            out = {k: torch.empty((d, N), dtype=torch.float32, device=self.device)
                   for k, d in (("x", 3), ("v", 3), ("C", 9), ("F", 9))}
            mpm.mpm_read_state(self.handle, *(out[k].data_ptr() for k in ("x", "v", "C", "F")), 1, _stream(stream))
            return out
        out = {k: np.empty((d, N), dtype=np.float32) for k, d in (("x", 3), ("v", 3), ("C", 9), ("F", 9))}
        if N:
            mpm.mpm_read_state(self.handle, *(out[k].ctypes.data for k in ("x", "v", "C", "F")), 0, _stream(stream))
        return out

    # ------------------------------------------------------------------ colliders
    def set_colliders(self, pose, lin_vel, ang_vel=None, com=None, stream=None):
        arrs = [None if a is None else np.ascontiguousarray(np.asarray(a, dtype=np.float32))
                for a in (pose, lin_vel, ang_vel, com)]
        ptrs = [0 if a is None else a.ctypes.data for a in arrs]
        mpm.mpm_set_colliders(self.handle, self.k, *ptrs, _stream(stream))

    def read_wrench(self, stream=None):
        out = np.zeros((max(self.k, 1), 6), dtype=np.float64)
        n = mpm.mpm_read_wrench(self.handle, out.ctypes.data, _stream(stream))
        return out[: self.k], n

    # ------------------------------------------------------------------ stepping
    def substep(self, n: int = 1, stream=None):
        mpm.mpm_substep(self.handle, n, _stream(stream))

    def status(self, clear: bool = False, stream=None) -> int:
        return mpm.mpm_get_status(self.handle, int(clear), _stream(stream))

    def set_timing(self, kinds=True):
        """Time launches of the given kernel kinds (names of ``KERNEL_NAMES``), all (True) or none."""
        if kinds is True:
            mask = (1 << mpm.MPM_K_COUNT) - 1
        elif not kinds:
            mask = 0
        else:
            mask = 0
            for k in kinds:
                mask |= 1 << mpm.KERNEL_NAMES.index(k)
        mpm.mpm_set_timing(self.handle, mask)

    def set_graphs(self, on: bool):
        mpm.mpm_set_graphs(self.handle, int(on))

    def read_timing(self, reset: bool = False):
        ms, cnt = mpm.mpm_read_timing(self.handle, int(reset))
        return {name: (ms[i], cnt[i]) for i, name in enumerate(mpm.KERNEL_NAMES)}

    @property
    def launches(self) -> int:
        return mpm.mpm_launch_count(self.handle)

    def set_launch(self, chunk: int = 0, fused_ctas_per_sm: int = 0, grid_ctas_per_sm: int = 0):
        """Launch shape of the substep kernels (0 keeps a value); drops cached graphs."""
        mpm.mpm_set_launch(self.handle, chunk, fused_ctas_per_sm, grid_ctas_per_sm)

    def get_launch(self):
        """(chunk, fused CTAs per SM, grid-update CTAs per SM)."""
        return mpm.mpm_get_launch(self.handle)

    def set_contact(self, mode: str = "grid", stiffness: float = 0.0, damping: float = 0.0):
        """Contact form: "grid" (colliders act on grid nodes) or "particle" (penalty accelerations at
        the particles: stiffness in 1/s^2, damping in 1/s); drops cached graphs."""
        m = {"grid": mpm.MPM_CONTACT_GRID, "particle": mpm.MPM_CONTACT_PARTICLE}[mode]
        mpm.mpm_set_contact(self.handle, m, stiffness, damping)

    def _shape_structs(self, shapes):
        """ABI shape structs; SDF volumes are copied to device buffers that live with the handle."""
        arr = []
        bufs = []
        for sh in shapes:
            st = mpm.mpm_shape(sh.type, (ctypes.c_float * 3)(*sh.half), sh.friction)
            if getattr(sh, "sdf", None) is not None:
                vol = np.asarray(sh.sdf, np.float32)
                buf = torch.from_numpy(np.ascontiguousarray(vol.transpose(2, 1, 0))).to(self.device)
                bufs.append(buf)
                st.sdf = buf.data_ptr()
                st.res = (ctypes.c_int * 3)(*vol.shape)
                st.sdf_origin = (ctypes.c_float * 3)(*sh.sdf_origin)
                st.sdf_h = sh.sdf_h
            arr.append(st)
        self._sdf_bufs = bufs
        return arr


class Sim(_Handle):
    """One scene: an n^3 grid of one material."""

    def __init__(self, n: int, dt: float, material, max_particles: int, gravity=(0.0, -9.8, 0.0), bound: int = 3,
                 max_colliders: int = 8, device=None):
        self.device = torch.device(device if device is not None else "cuda")
        self.cfg = mpm.mpm_config(n, dt, (ctypes.c_float * 3)(*gravity), bound, max_particles, max_colliders)
        self.mat = _material(material)
        nbytes = mpm.mpm_workspace_size(self.cfg, self.mat)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self.handle = mpm.mpm_create(self.cfg, self.mat, self.workspace.data_ptr(), nbytes, _stream())
        self.n = n
        self.kinds = [material.kind]
        self.k = 0

    def set_particles(self, x, v=None, C=None, F=None, stream=None):
        if isinstance(x, torch.Tensor) and x.is_cuda:
            n = x.shape[1]
            mpm.mpm_set_particles(self.handle, n, _dev_ptr(x), _dev_ptr(v), _dev_ptr(C), _dev_ptr(F), 1,
                                  _stream(stream))
            return
        arrs = [None if a is None else np.ascontiguousarray(np.asarray(a, dtype=np.float32)) for a in (x, v, C, F)]
        n = arrs[0].shape[1]
        ptrs = [0 if a is None else a.ctypes.data for a in arrs]
        mpm.mpm_set_particles(self.handle, n, *ptrs, 0, _stream(stream))

    def read_grid(self, stream=None):
        g = torch.zeros((self.n, self.n, self.n, 4), dtype=torch.float32, device=self.device)
        mpm.mpm_read_grid(self.handle, g.data_ptr(), _stream(stream))
        return g

    def set_shapes(self, shapes):
        arr = self._shape_structs(shapes)
        mpm.mpm_set_shapes(self.handle, arr)
        self.k = len(arr)


class BatchSim(_Handle):
    """Many independent scenes (envs) in one handle, advanced together by the same launches.

    ``envs`` is a list of ``(n, material, max_particles, max_colliders)``; dt, gravity and the sticky
    wall width are shared. Particle arrays are concatenated in env order (SoA over all particles),
    collider arrays likewise; ``offsets[e]:offsets[e + 1]`` are env e's particles.
    """

    def __init__(self, envs, dt: float, gravity=(0.0, -9.8, 0.0), bound: int = 3, device=None):
        self.device = torch.device(device if device is not None else "cuda")
        self.env_specs = [mpm.mpm_env(int(n), int(cap), int(kmax), _material(m)) for n, m, cap, kmax in envs]
        self.cfg = mpm.mpm_config(int(envs[0][0]), dt, (ctypes.c_float * 3)(*gravity), bound, 1, 0)
        nbytes = mpm.mpm_workspace_size_batch(self.cfg, self.env_specs)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self.handle = mpm.mpm_create_batch(self.cfg, self.env_specs, self.workspace.data_ptr(), nbytes, _stream())
        self.ns = [int(e[0]) for e in envs]
        self.kinds = [int(e[1].kind) for e in envs]
        self.counts = [0] * len(envs)
        self.shape_counts = [0] * len(envs)
        self.k = 0

    @property
    def nenv(self) -> int:
        return mpm.mpm_num_envs(self.handle)

    @property
    def offsets(self):
        return np.concatenate([[0], np.cumsum(self.counts)]).astype(np.int64)

    def set_particles(self, counts, x, v=None, C=None, F=None, stream=None):
        """counts[e] particles per env; arrays (d, sum(counts)) concatenated in env order."""
        counts = [int(c) for c in counts]
        if isinstance(x, torch.Tensor) and x.is_cuda:
            mpm.mpm_set_particles_batch(self.handle, counts, _dev_ptr(x), _dev_ptr(v), _dev_ptr(C), _dev_ptr(F), 1,
                                        _stream(stream))
        else:
            arrs = [None if a is None else np.ascontiguousarray(np.asarray(a, dtype=np.float32))
                    for a in (x, v, C, F)]
            ptrs = [0 if a is None else a.ctypes.data for a in arrs]
            mpm.mpm_set_particles_batch(self.handle, counts, *ptrs, 0, _stream(stream))
        self.counts = counts

    def read_grid(self, stream=None):
        """Per env, its (n, n, n, 4) node array."""
        total = sum(n ** 3 * 4 for n in self.ns)
        flat = torch.zeros(total, dtype=torch.float32, device=self.device)
        mpm.mpm_read_grid(self.handle, flat.data_ptr(), _stream(stream))
        out, off = [], 0
        for n in self.ns:
            out.append(flat[off: off + n ** 3 * 4].view(n, n, n, 4))
            off += n ** 3 * 4
        return out

    def set_shapes(self, shapes_per_env):
        """shapes_per_env[e]: the collider shapes of env e."""
        counts = [len(s) for s in shapes_per_env]
        arr = self._shape_structs([s for env in shapes_per_env for s in env])
        mpm.mpm_set_shapes_batch(self.handle, counts, arr)
        self.shape_counts = counts
        self.k = len(arr)
