"""Thin ctypes binding of ``include/mpm.h`` (libmpm_gb300.so): same entry points, same names.

Argument marshalling only -- every step of the substep runs in the CUDA library.
Pointers are plain integers (device or host addresses), streams are
``cudaStream_t`` values as integers. A non-OK status raises ``MpmError``.
The library is loaded on first use; if it has not been built, loading raises
(there is no fallback).
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

MPM_MAX_COLLIDERS = 32
MPM_MAX_ENVS = 16384
MPM_OK, MPM_ERR_INVALID_ARG, MPM_ERR_CUDA, MPM_ERR_WORKSPACE, MPM_ERR_CAPACITY = range(5)
MPM_FLAG_CLAMPED = 0x1
MPM_FLAG_NONFINITE = 0x2
MPM_FLAG_SV_CLAMPED = 0x4
MPM_FLAG_FAR_MOVE = 0x8
MPM_FLAG_INTERNAL = 0x80000000
MPM_PLASTICINE, MPM_FLUID = 0, 1
MPM_NET_F32, MPM_NET_BF16 = 0, 1
MPM_BOX, MPM_CAPSULE = 0, 1
(MPM_K_LOAD, MPM_K_SCAN, MPM_K_ASSIGN, MPM_K_P2G, MPM_K_GRID, MPM_K_G2P2G, MPM_K_READ,
 MPM_K_COLLIDERS, MPM_K_COUNT) = range(9)
KERNEL_NAMES = ["load", "scan", "assign", "p2g", "grid_update", "g2p2g", "read", "colliders"]

LIB_PATH = _build.LIB_PATH


class mpm_config(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("dt", ctypes.c_float), ("gravity", ctypes.c_float * 3),
                ("bound", ctypes.c_int), ("max_particles", ctypes.c_int), ("max_colliders", ctypes.c_int)]


class mpm_material(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("rho", ctypes.c_float), ("E", ctypes.c_float), ("nu", ctypes.c_float),
                ("yield_stress", ctypes.c_float), ("bulk_modulus", ctypes.c_float), ("p_vol", ctypes.c_float)]


class mpm_shape(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("half", ctypes.c_float * 3), ("friction", ctypes.c_float),
                ("sdf", ctypes.c_void_p), ("res", ctypes.c_int * 3), ("sdf_origin", ctypes.c_float * 3),
                ("sdf_h", ctypes.c_float)]


class mpm_camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int), ("height", ctypes.c_int), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("eye", ctypes.c_float * 3), ("rot", ctypes.c_float * 9),
                ("near_z", ctypes.c_float)]


class mpm_render_params(ctypes.Structure):
    _fields_ = [("radius", ctypes.c_float), ("smooth", ctypes.c_float), ("sigma_depth", ctypes.c_float),
                ("window", ctypes.c_int), ("light", ctypes.c_float * 3), ("albedo", ctypes.c_float * 3),
                ("ambient", ctypes.c_float), ("background", ctypes.c_float * 3)]


class mpm_env(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("max_particles", ctypes.c_int), ("max_colliders", ctypes.c_int),
                ("material", mpm_material)]


class mpm_box(ctypes.Structure):
    _fields_ = [("i0", ctypes.c_int), ("j0", ctypes.c_int), ("k0", ctypes.c_int), ("D", ctypes.c_int),
                ("H", ctypes.c_int), ("W", ctypes.c_int)]

    def dims(self):
        return (self.D, self.H, self.W)


class mpm_surrogate_net(ctypes.Structure):
    _fields_ = [("w_packed", ctypes.c_void_p * 4), ("bias", ctypes.c_void_p * 4), ("m_scale", ctypes.c_float),
                ("v_scale", ctypes.c_float), ("dv_unit", ctypes.c_float), ("v_ref", ctypes.c_double),
                ("threshold", ctypes.c_double), ("k", ctypes.c_int), ("margin", ctypes.c_int)]


class MpmError(RuntimeError):
    def __init__(self, fn, status, detail=""):
        self.status = status
        super().__init__(f"{fn}: {status_string(status)}{(' (' + detail + ')') if detail else ''}")


_lib = None
_vp = ctypes.c_void_p


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing (run __graft_entry__.build())")
    L = ctypes.CDLL(LIB_PATH)
    st = ctypes.c_int
    sig = {
        "mpm_workspace_size": (st, [ctypes.POINTER(mpm_config), ctypes.POINTER(mpm_material), ctypes.POINTER(ctypes.c_size_t)]),
        "mpm_create": (st, [ctypes.POINTER(mpm_config), ctypes.POINTER(mpm_material), _vp, ctypes.c_size_t, _vp,
                            ctypes.POINTER(_vp)]),
        "mpm_workspace_size_batch": (st, [ctypes.POINTER(mpm_config), ctypes.c_int, ctypes.POINTER(mpm_env),
                                          ctypes.POINTER(ctypes.c_size_t)]),
        "mpm_create_batch": (st, [ctypes.POINTER(mpm_config), ctypes.c_int, ctypes.POINTER(mpm_env), _vp,
                                  ctypes.c_size_t, _vp, ctypes.POINTER(_vp)]),
        "mpm_set_particles_batch": (st, [_vp, ctypes.POINTER(ctypes.c_int), _vp, _vp, _vp, _vp, ctypes.c_int, _vp]),
        "mpm_set_shapes_batch": (st, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(mpm_shape)]),
        "mpm_num_envs": (ctypes.c_int, [_vp]),
        "mpm_set_launch": (st, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
        "mpm_set_contact": (st, [_vp, ctypes.c_int, ctypes.c_float, ctypes.c_float]),
        "mpm_render_workspace_size": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int]),
        "mpm_render": (st, [ctypes.POINTER(mpm_camera), ctypes.POINTER(mpm_render_params), ctypes.c_int, ctypes.c_int,
                            _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_size_t, _vp]),
        "mpm_render_sim": (st, [_vp, ctypes.POINTER(mpm_camera), ctypes.POINTER(mpm_render_params), _vp, _vp, _vp, _vp,
                                _vp, ctypes.c_size_t, _vp]),
        "mpm_get_launch": (st, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_int)]),
        "mpm_set_particles": (st, [_vp, ctypes.c_int, _vp, _vp, _vp, _vp, ctypes.c_int, _vp]),
        "mpm_set_shapes": (st, [_vp, ctypes.c_int, ctypes.POINTER(mpm_shape)]),
        "mpm_set_colliders": (st, [_vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp]),
        "mpm_substep": (st, [_vp, ctypes.c_int, _vp]),
        "mpm_read_state": (st, [_vp, _vp, _vp, _vp, _vp, ctypes.c_int, _vp]),
        "mpm_read_wrench": (st, [_vp, _vp, ctypes.POINTER(ctypes.c_int), _vp]),
        "mpm_read_wrench_async": (st, [_vp, _vp, _vp, _vp]),
        "mpm_get_status": (st, [_vp, ctypes.POINTER(ctypes.c_uint), ctypes.c_int, _vp]),
        "mpm_num_particles": (ctypes.c_int, [_vp]),
        "mpm_read_grid": (st, [_vp, _vp, _vp]),
        "mpm_set_timing": (st, [_vp, ctypes.c_uint]),
        "mpm_set_graphs": (st, [_vp, ctypes.c_int]),
        "mpm_read_timing": (st, [_vp, _vp, _vp, ctypes.c_int]),
        "mpm_launch_count": (ctypes.c_longlong, [_vp]),
        "mpm_destroy": (None, [_vp]),
        "mpm_p2g_static": (st, [ctypes.POINTER(mpm_config), ctypes.POINTER(mpm_material), ctypes.c_int, _vp, _vp, _vp,
                                _vp, _vp, _vp]),
        "mpm_conv3d_forward": (st, [ctypes.c_int] * 6 + [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp]),
        "mpm_conv3d_forward_tiled": (st, [ctypes.c_int] * 5 + [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp,
                                                               _vp]),
        "mpm_conv3d_tile_count": (ctypes.c_int, [ctypes.c_int] * 3),
        "mpm_conv3d_tile_flags": (st, [ctypes.c_int] * 3 + [_vp, ctypes.c_int, _vp, _vp]),
        "mpm_conv3d_forward_tc": (st, [ctypes.c_int] * 5 + [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp,
                                                            ctypes.c_int, _vp]),
        "mpm_conv3d_tc_packed_bytes": (ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
        "mpm_conv3d_pack_tc": (st, [ctypes.c_int, ctypes.c_int, _vp, _vp, _vp]),
        "mpm_conv3d_tc_adjoint_packed_bytes": (ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
        "mpm_conv3d_pack_tc_adjoint": (st, [ctypes.c_int, ctypes.c_int, _vp, _vp, _vp]),
        "mpm_conv3d_backward_data_tc": (st, [ctypes.c_int] * 5 + [_vp, _vp, _vp, _vp, _vp]),
        "mpm_conv3d_backward_weight_tc": (st, [ctypes.c_int] * 5 + [_vp, _vp, _vp, _vp, _vp]),
        "mpm_pad_channels_bf16": (st, [ctypes.c_int] * 3 + [_vp, _vp, _vp]),
        "mpm_conv3d_tc_tile_count": (ctypes.c_int, [ctypes.c_int] * 3),
        "mpm_conv3d_tc_tile_dist": (st, [ctypes.c_int] * 3 + [_vp, _vp, _vp]),
        "mpm_net_tc_status": (st, [ctypes.POINTER(ctypes.c_uint), ctypes.c_int, _vp]),
        "mpm_conv3d_backward_data": (st, [ctypes.c_int] * 6 + [_vp, _vp, _vp, _vp, _vp]),
        "mpm_conv3d_backward_weight": (st, [ctypes.c_int] * 6 + [_vp, _vp, _vp, _vp, _vp]),
        "mpm_mse_loss": (st, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int, _vp, _vp, _vp, _vp, _vp]),
        "mpm_adam_step": (st, [ctypes.c_int, _vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                               ctypes.c_float, ctypes.c_float, _vp, _vp]),
        "mpm_cast_f32_to_bf16": (st, [ctypes.c_int, _vp, _vp, _vp]),
        "mpm_cast_bf16_to_f32": (st, [ctypes.c_int, _vp, _vp, _vp]),
        "mpm_surrogate_box": (st, [_vp, ctypes.c_int, ctypes.POINTER(mpm_box), _vp]),
        "mpm_surrogate_features": (st, [_vp, ctypes.POINTER(mpm_box), ctypes.c_float, ctypes.c_float, _vp, _vp, _vp]),
        "mpm_surrogate_check": (st, [_vp, ctypes.POINTER(mpm_box), _vp, ctypes.c_float, ctypes.c_int, ctypes.c_double,
                                     ctypes.POINTER(ctypes.c_double), _vp]),
        "mpm_surrogate_advance": (st, [_vp, ctypes.POINTER(mpm_box), _vp, ctypes.c_float, ctypes.c_int, _vp]),
        "mpm_surrogate_workspace_size": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_int]),
        "mpm_surrogate_attach": (st, [_vp, ctypes.POINTER(mpm_surrogate_net), _vp, ctypes.c_size_t, ctypes.c_int]),
        "mpm_surrogate_step": (st, [_vp, ctypes.c_int, ctypes.c_int, _vp]),
        "mpm_surrogate_stats": (st, [_vp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                                     ctypes.POINTER(ctypes.c_double), ctypes.c_int, _vp]),
        "mpm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "mpm_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def lib():
    return _load()


def _check(fn, status):
    if status != MPM_OK:
        detail = _load().mpm_last_error().decode() if status == MPM_ERR_CUDA else ""
        raise MpmError(fn, status, detail)


def status_string(status: int) -> str:
    return _load().mpm_status_string(status).decode()


def mpm_workspace_size(cfg: mpm_config, mat: mpm_material) -> int:
    out = ctypes.c_size_t(0)
    _check("mpm_workspace_size", _load().mpm_workspace_size(ctypes.byref(cfg), ctypes.byref(mat), ctypes.byref(out)))
    return out.value


def mpm_create(cfg: mpm_config, mat: mpm_material, d_workspace: int, nbytes: int, stream: int = 0) -> int:
    h = _vp()
    _check("mpm_create", _load().mpm_create(ctypes.byref(cfg), ctypes.byref(mat), d_workspace, nbytes, stream,
                                            ctypes.byref(h)))
    return h.value


def _env_array(envs):
    return (mpm_env * max(1, len(envs)))(*envs)


def mpm_workspace_size_batch(cfg: mpm_config, envs) -> int:
    out = ctypes.c_size_t(0)
    _check("mpm_workspace_size_batch", _load().mpm_workspace_size_batch(ctypes.byref(cfg), len(envs),
                                                                        _env_array(envs), ctypes.byref(out)))
    return out.value


def mpm_create_batch(cfg: mpm_config, envs, d_workspace: int, nbytes: int, stream: int = 0) -> int:
    h = _vp()
    _check("mpm_create_batch", _load().mpm_create_batch(ctypes.byref(cfg), len(envs), _env_array(envs), d_workspace,
                                                        nbytes, stream, ctypes.byref(h)))
    return h.value


def mpm_set_particles_batch(sim: int, counts, x: int, v: int = 0, C: int = 0, F: int = 0, src_on_device: int = 1,
                            stream: int = 0) -> None:
    c = (ctypes.c_int * max(1, len(counts)))(*counts)
    _check("mpm_set_particles_batch", _load().mpm_set_particles_batch(sim, c, x or None, v or None, C or None,
                                                                      F or None, src_on_device, stream))


def mpm_set_shapes_batch(sim: int, counts, shapes) -> None:
    c = (ctypes.c_int * max(1, len(counts)))(*counts)
    arr = (mpm_shape * max(1, len(shapes)))(*shapes)
    _check("mpm_set_shapes_batch", _load().mpm_set_shapes_batch(sim, c, arr))


def mpm_num_envs(sim: int) -> int:
    return _load().mpm_num_envs(sim)


def mpm_set_launch(sim: int, chunk: int = 0, fused_ctas_per_sm: int = 0, grid_ctas_per_sm: int = 0) -> None:
    _check("mpm_set_launch", _load().mpm_set_launch(sim, chunk, fused_ctas_per_sm, grid_ctas_per_sm))


MPM_CONTACT_GRID = 0
MPM_CONTACT_PARTICLE = 1
MPM_SDF_VOLUME = 2


def mpm_set_contact(sim: int, mode: int, stiffness: float = 0.0, damping: float = 0.0) -> None:
    _check("mpm_set_contact", _load().mpm_set_contact(sim, mode, stiffness, damping))


def mpm_render_workspace_size(width: int, height: int) -> int:
    return _load().mpm_render_workspace_size(width, height)


def mpm_render(cam: mpm_camera, params: mpm_render_params, n: int, stride: int, d_x: int, d_depth: int, d_smooth: int,
               d_normal: int, d_rgb: int, d_ws: int, nbytes: int, stream: int = 0) -> None:
    _check("mpm_render", _load().mpm_render(ctypes.byref(cam), ctypes.byref(params), n, stride, d_x, d_depth, d_smooth,
                                            d_normal, d_rgb, d_ws, nbytes, stream))


def mpm_render_sim(sim: int, cam: mpm_camera, params: mpm_render_params, d_depth: int, d_smooth: int, d_normal: int,
                   d_rgb: int, d_ws: int, nbytes: int, stream: int = 0) -> None:
    _check("mpm_render_sim", _load().mpm_render_sim(sim, ctypes.byref(cam), ctypes.byref(params), d_depth, d_smooth,
                                                    d_normal, d_rgb, d_ws, nbytes, stream))


def mpm_get_launch(sim: int):
    a, b, c = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    _check("mpm_get_launch", _load().mpm_get_launch(sim, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def mpm_set_particles(sim: int, n: int, x: int, v: int = 0, C: int = 0, F: int = 0, src_on_device: int = 1,
                      stream: int = 0) -> None:
    _check("mpm_set_particles", _load().mpm_set_particles(sim, n, x or None, v or None, C or None, F or None,
                                                          src_on_device, stream))


def mpm_set_shapes(sim: int, shapes) -> None:
    arr = (mpm_shape * max(1, len(shapes)))(*shapes)
    _check("mpm_set_shapes", _load().mpm_set_shapes(sim, len(shapes), arr))


def mpm_set_colliders(sim: int, k: int, pose: int, lin_vel: int, ang_vel: int = 0, com: int = 0,
                      stream: int = 0) -> None:
    _check("mpm_set_colliders", _load().mpm_set_colliders(sim, k, pose or None, lin_vel or None, ang_vel or None,
                                                          com or None, stream))


def mpm_substep(sim: int, n_substeps: int, stream: int = 0) -> None:
    _check("mpm_substep", _load().mpm_substep(sim, n_substeps, stream))


def mpm_read_state(sim: int, x: int = 0, v: int = 0, C: int = 0, F: int = 0, dst_on_device: int = 1,
                   stream: int = 0) -> None:
    _check("mpm_read_state", _load().mpm_read_state(sim, x or None, v or None, C or None, F or None, dst_on_device,
                                                    stream))


def mpm_read_wrench(sim: int, out: int, stream: int = 0) -> int:
    n = ctypes.c_int(0)
    _check("mpm_read_wrench", _load().mpm_read_wrench(sim, out or None, ctypes.byref(n), stream))
    return n.value


def mpm_read_wrench_async(sim: int, out: int, n_substeps: int, stream: int = 0) -> None:
    """Enqueue the wrench and substep count into page-locked host memory (pointers), without waiting."""
    _check("mpm_read_wrench_async", _load().mpm_read_wrench_async(sim, out or None, n_substeps or None, stream))


def mpm_get_status(sim: int, clear: int = 0, stream: int = 0) -> int:
    f = ctypes.c_uint(0)
    _check("mpm_get_status", _load().mpm_get_status(sim, ctypes.byref(f), clear, stream))
    return f.value


def mpm_num_particles(sim: int) -> int:
    return _load().mpm_num_particles(sim)


def mpm_read_grid(sim: int, d_out: int, stream: int = 0) -> None:
    _check("mpm_read_grid", _load().mpm_read_grid(sim, d_out, stream))


def mpm_set_timing(sim: int, kernel_mask: int) -> None:
    _check("mpm_set_timing", _load().mpm_set_timing(sim, kernel_mask & 0xFFFFFFFF))


def mpm_set_graphs(sim: int, enable: int) -> None:
    _check("mpm_set_graphs", _load().mpm_set_graphs(sim, enable))


def mpm_read_timing(sim: int, reset: int = 0):
    ms = (ctypes.c_double * MPM_K_COUNT)()
    cnt = (ctypes.c_longlong * MPM_K_COUNT)()
    _check("mpm_read_timing", _load().mpm_read_timing(sim, ms, cnt, reset))
    return list(ms), list(cnt)


def mpm_launch_count(sim: int) -> int:
    return _load().mpm_launch_count(sim)


def mpm_destroy(sim: int) -> None:
    _load().mpm_destroy(sim)


def mpm_p2g_static(cfg: mpm_config, mat: mpm_material, n: int, x: int, v: int = 0, C: int = 0, F: int = 0,
                   grid_out: int = 0, stream: int = 0) -> None:
    """Particle-to-grid transfer into a caller grid with the library's own scratch (no allocation)."""
    _check("mpm_p2g_static", _load().mpm_p2g_static(ctypes.byref(cfg), ctypes.byref(mat), n, x or None, v or None,
                                                    C or None, F or None, grid_out or None, stream))


def mpm_last_error() -> str:
    return _load().mpm_last_error().decode()


# ---------------------------------------------------------------------------- network kernels (mpm_net.h)

def mpm_conv3d_forward(dtype, D, H, W, cin, cout, x, w, bias, relu, y_f32, y, stream=0):
    _check("mpm_conv3d_forward", _load().mpm_conv3d_forward(dtype, D, H, W, cin, cout, x, w, bias or None, relu,
                                                            y_f32, y, stream))


def mpm_conv3d_forward_tiled(D, H, W, cin, cout, x, w, bias, relu, y_f32, y, tile_flags, stream=0):
    _check("mpm_conv3d_forward_tiled", _load().mpm_conv3d_forward_tiled(D, H, W, cin, cout, x, w, bias or None, relu,
                                                                        y_f32, y, tile_flags, stream))


def mpm_conv3d_forward_tc(D, H, W, cin, cout, x, w_packed, bias, relu, y_f32, y, tile_dist=0, radius=0, stream=0):
    _check("mpm_conv3d_forward_tc", _load().mpm_conv3d_forward_tc(D, H, W, cin, cout, x, w_packed, bias or None, relu,
                                                                  y_f32, y, tile_dist or None, radius, stream))


def mpm_conv3d_tc_packed_bytes(cin, cout) -> int:
    return _load().mpm_conv3d_tc_packed_bytes(cin, cout)


def mpm_conv3d_pack_tc(cin, cout, w, packed, stream=0):
    _check("mpm_conv3d_pack_tc", _load().mpm_conv3d_pack_tc(cin, cout, w, packed, stream))


def mpm_conv3d_tc_adjoint_packed_bytes(cin, cout) -> int:
    return _load().mpm_conv3d_tc_adjoint_packed_bytes(cin, cout)


def mpm_conv3d_pack_tc_adjoint(cin, cout, w, packed, stream=0):
    _check("mpm_conv3d_pack_tc_adjoint", _load().mpm_conv3d_pack_tc_adjoint(cin, cout, w, packed, stream))


def mpm_conv3d_backward_data_tc(D, H, W, cin, cout, dy, w_adj_packed, act_in, dx, stream=0):
    _check("mpm_conv3d_backward_data_tc", _load().mpm_conv3d_backward_data_tc(D, H, W, cin, cout, dy, w_adj_packed,
                                                                              act_in or None, dx, stream))


def mpm_pad_channels_bf16(nvox, c, c_pad, src, dst, stream=0):
    _check("mpm_pad_channels_bf16", _load().mpm_pad_channels_bf16(nvox, c, c_pad, src, dst, stream))


def mpm_conv3d_tc_tile_count(D, H, W) -> int:
    return _load().mpm_conv3d_tc_tile_count(D, H, W)


def mpm_conv3d_tc_tile_dist(D, H, W, mask, dist, stream=0):
    _check("mpm_conv3d_tc_tile_dist", _load().mpm_conv3d_tc_tile_dist(D, H, W, mask, dist, stream))


def mpm_net_tc_status(clear=0, stream=0) -> int:
    f = ctypes.c_uint(0)
    _check("mpm_net_tc_status", _load().mpm_net_tc_status(ctypes.byref(f), clear, stream))
    return f.value


def mpm_conv3d_tile_count(D, H, W) -> int:
    return _load().mpm_conv3d_tile_count(D, H, W)


def mpm_conv3d_tile_flags(D, H, W, mask, dilate, flags, stream=0):
    _check("mpm_conv3d_tile_flags", _load().mpm_conv3d_tile_flags(D, H, W, mask, dilate, flags, stream))


def mpm_conv3d_backward_data(dtype, D, H, W, cin, cout, dy, w, act_in, dx, stream=0):
    _check("mpm_conv3d_backward_data", _load().mpm_conv3d_backward_data(dtype, D, H, W, cin, cout, dy, w,
                                                                        act_in or None, dx, stream))


def mpm_conv3d_backward_weight_tc(D, H, W, cin, cout, x, dy, dw, db, stream=0):
    _check("mpm_conv3d_backward_weight_tc", _load().mpm_conv3d_backward_weight_tc(D, H, W, cin, cout, x, dy, dw, db,
                                                                                  stream))


def mpm_conv3d_backward_weight(dtype, D, H, W, cin, cout, x, dy, dw, db, stream=0):
    _check("mpm_conv3d_backward_weight", _load().mpm_conv3d_backward_weight(dtype, D, H, W, cin, cout, x, dy, dw,
                                                                            db, stream))


def mpm_mse_loss(dtype, nvox, C, pred, pred_f32, target, mask, loss, dpred, stream=0):
    _check("mpm_mse_loss", _load().mpm_mse_loss(dtype, nvox, C, pred, pred_f32, target, mask, loss, dpred, stream))


def mpm_adam_step(n, p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, p_bf16=0, stream=0):
    _check("mpm_adam_step", _load().mpm_adam_step(n, p, g, m, v, t, lr, beta1, beta2, eps, p_bf16 or None, stream))


def mpm_cast_f32_to_bf16(n, src, dst, stream=0):
    _check("mpm_cast_f32_to_bf16", _load().mpm_cast_f32_to_bf16(n, src, dst, stream))


def mpm_cast_bf16_to_f32(n, src, dst, stream=0):
    _check("mpm_cast_bf16_to_f32", _load().mpm_cast_bf16_to_f32(n, src, dst, stream))


# ---------------------------------------------------------------------------- surrogate window (mpm.h)

def mpm_surrogate_box(sim, margin, stream=0) -> mpm_box:
    b = mpm_box()
    _check("mpm_surrogate_box", _load().mpm_surrogate_box(sim, margin, ctypes.byref(b), stream))
    return b


def mpm_surrogate_features(sim, box: mpm_box, m_scale, v_scale, feat, mask, stream=0):
    _check("mpm_surrogate_features", _load().mpm_surrogate_features(sim, ctypes.byref(box), m_scale, v_scale, feat,
                                                                    mask, stream))


def mpm_surrogate_check(sim, box: mpm_box, dv, dv_unit, k, v_ref, stream=0):
    """Returns (mass residual, momentum residual, grid mass, |P_hat - P_exp|)."""
    out = (ctypes.c_double * 4)()
    _check("mpm_surrogate_check", _load().mpm_surrogate_check(sim, ctypes.byref(box), dv, dv_unit, k, v_ref, out,
                                                              stream))
    return tuple(out)


def mpm_surrogate_advance(sim, box: mpm_box, dv, dv_unit, k, stream=0):
    _check("mpm_surrogate_advance", _load().mpm_surrogate_advance(sim, ctypes.byref(box) if box is not None else None,
                                                                  dv or None, dv_unit, k, stream))


def mpm_surrogate_workspace_size(max_voxels, max_particles) -> int:
    return _load().mpm_surrogate_workspace_size(max_voxels, max_particles)


def mpm_surrogate_attach(sim, net, d_workspace, nbytes, max_voxels):
    _check("mpm_surrogate_attach", _load().mpm_surrogate_attach(sim, ctypes.byref(net) if net is not None else None,
                                                                d_workspace, nbytes, max_voxels))


def mpm_surrogate_step(sim, n_substeps, gate=1, stream=0):
    _check("mpm_surrogate_step", _load().mpm_surrogate_step(sim, n_substeps, gate, stream))


def mpm_surrogate_stats(sim, reset=0, stream=0):
    """Returns (windows, fallbacks, (mass residual, momentum residual) of the last window)."""
    w, f = ctypes.c_longlong(0), ctypes.c_longlong(0)
    r = (ctypes.c_double * 2)()
    _check("mpm_surrogate_stats", _load().mpm_surrogate_stats(sim, ctypes.byref(w), ctypes.byref(f), r, reset, stream))
    return w.value, f.value, (r[0], r[1])
