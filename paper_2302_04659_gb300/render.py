"""Particle renderer binding (App. D.2 screen-space splatting; the kernels are in csrc/render_kernels.cu).

``Renderer`` owns the device images of one camera and renders either positions the caller holds
(``render``) or a simulation handle's particles in place (``render_sim``). Argument marshalling only:
every step runs in the library's kernels."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from . import _native as mpm


def look_at(eye, target, up=(0.0, 1.0, 0.0)) -> np.ndarray:
    """World -> camera rotation (rows: camera x right, y down, z forward) looking from eye at target."""
    eye, target, up = (np.asarray(a, np.float64) for a in (eye, target, up))
    z = target - eye
    z /= np.linalg.norm(z)
    x = np.cross(z, up)  # right, with y pointing down the image
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    return np.stack([x, y, z])


@dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    eye: tuple
    rot: np.ndarray
    near_z: float = 1e-3

    @staticmethod
    def looking(width, height, fov_y_deg, eye, target, up=(0.0, 1.0, 0.0)) -> "Camera":
        f = 0.5 * height / np.tan(np.radians(fov_y_deg) / 2)
        return Camera(width, height, f, f, width / 2, height / 2, tuple(eye), look_at(eye, target, up))

    def c(self) -> mpm.mpm_camera:
        f3 = ctypes.c_float * 3
        return mpm.mpm_camera(self.width, self.height, self.fx, self.fy, self.cx, self.cy, f3(*self.eye),
                              (ctypes.c_float * 9)(*np.asarray(self.rot, np.float32).reshape(9)), self.near_z)


@dataclass
class Style:
    radius: float
    smooth: float
    sigma_depth: float
    window: int = 4
    light: tuple = (0.3, -0.6, -0.75)
    albedo: tuple = (0.85, 0.6, 0.4)
    ambient: float = 0.25
    background: tuple = (0.0, 0.0, 0.0)

    def c(self) -> mpm.mpm_render_params:
        f3 = ctypes.c_float * 3
        return mpm.mpm_render_params(self.radius, self.smooth, self.sigma_depth, self.window, f3(*self.light),
                                     f3(*self.albedo), self.ambient, f3(*self.background))


class Renderer:
    """Device images of one camera: depth, smoothed depth (H, W), normals and colour (H, W, 3)."""

    def __init__(self, camera: Camera, style: Style, device=None):
        self.device = torch.device(device if device is not None else "cuda")
        self.camera, self.style = camera, style
        H, W = camera.height, camera.width
        kw = dict(dtype=torch.float32, device=self.device)
        self.depth = torch.empty((H, W), **kw)
        self.smooth = torch.empty((H, W), **kw)
        self.normal = torch.empty((H, W, 3), **kw)
        self.rgb = torch.empty((H, W, 3), **kw)
        self.ws_bytes = mpm.mpm_render_workspace_size(W, H)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        self._cam, self._style = camera.c(), style.c()

    def _outs(self):
        return (self.depth.data_ptr(), self.smooth.data_ptr(), self.normal.data_ptr(), self.rgb.data_ptr(),
                self.ws.data_ptr(), self.ws_bytes)

    def render(self, x: torch.Tensor, stream=None):
        """x: device positions (3, N) (FP32, rows contiguous)."""
        x = x.to(self.device, torch.float32).contiguous()
        n = x.shape[1]
        mpm.mpm_render(self._cam, self._style, n, n, x.data_ptr(), *self._outs(), _stream(stream))
        return self.rgb

    def render_sim(self, sim, stream=None):
        """The particles of a ``Sim`` / ``BatchSim``, read where the simulation keeps them."""
        mpm.mpm_render_sim(sim.handle, self._cam, self._style, *self._outs(), _stream(stream))
        return self.rgb


def _stream(stream) -> int:
    if stream is None:
        return int(torch.cuda.current_stream().cuda_stream)
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def save_ppm(rgb, path: str) -> None:
    """Write an (H, W, 3) colour image in [0, 1] as a binary PPM file."""
    a = rgb.detach().cpu().numpy() if isinstance(rgb, torch.Tensor) else np.asarray(rgb)
    img = (np.clip(a, 0.0, 1.0) * 255.0 + 0.5).astype(np.uint8)
    with open(path, "wb") as f:
        f.write(f"P6 {img.shape[1]} {img.shape[0]} 255\n".encode())
        f.write(img.tobytes())
