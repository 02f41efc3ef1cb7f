"""Learned grid surrogate: a small 3D convolutional network that replaces k = 5 MPM substeps at a time.

An extension of the method (the paper's simulator has no learned component). A window of k substeps
runs as: one plain grid update (gravity, colliders, sticky walls), the network's correction of the
updated node velocities, and one grid-to-particle transfer with time step k*dt (``mpm_surrogate_*`` in
include/mpm.h).
The network sees, over a box around the material, each node's mass and updated velocity; it predicts
the change that turns the updated velocity into the mass-weighted mean velocity of the node's particles
over the next k substeps (the velocity a single k*dt transfer needs to move them where k plain substeps
would). A gate compares the corrected grid's mass and momentum with the plain method's first-order
prediction and falls back to k plain substeps when either residual exceeds 1e-3.

Network: four 3x3x3 convolutions, 4 -> 32 -> 32 -> 32 -> 3 channels, ReLU between them, zero padding;
BF16 weights and activations with FP32 accumulation, trained with Adam on windows the plain MPM
generates from the pinch-scene distribution. Every step of training and inference runs in the
library's kernels (mpm_net.h, mpm.h); this module only allocates buffers and sequences the calls.

    python -m paper_2302_04659_gb300.surrogate train --out FILE [--rollouts 2000] [--epochs 48]
    python -m paper_2302_04659_gb300.surrogate eval --weights FILE [--scenes 256]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np
import torch

from . import _native as mpm
from . import scenes

CHANNELS = (4, 32, 32, 32, 3)
K = 5                 # substeps per window
V_SCALE = 10.0        # network input units per m/s
DV_UNIT = 0.01        # m/s per network output unit
V_REF = 0.0           # velocity scale of the momentum residual: 0 = the scene's RMS node speed at the window start
THRESHOLD = 1e-3      # fallback when the mass or momentum residual exceeds this
MARGIN = 5            # nodes around the material's bins: 4 for the receptive field, 1 for motion in a step
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "surrogate_pinch64.npz")


def mass_scale(rho: float, n: int) -> float:
    """Input scale of node mass: 1 / (rho dx^3), the mass of a node fully inside the material."""
    return float(n ** 3 / rho)


def _stream(stream=None) -> int:
    return int((stream or torch.cuda.current_stream()).cuda_stream)


class Network:
    """The convolutional net: FP32 master weights, BF16 mirrors, Adam moments, per-box buffers."""

    def __init__(self, device="cuda", seed: int = 0):
        self.device = torch.device(device)
        rng = np.random.default_rng(seed)
        self.w, self.b = [], []
        for i in range(4):
            cin, cout = CHANNELS[i], CHANNELS[i + 1]
            std = math.sqrt(2.0 / (27 * cin)) * (0.1 if i == 3 else 1.0)  # He init; a small last layer
            self.w.append(torch.from_numpy(rng.normal(0.0, std, size=(27, cout, cin)).astype(np.float32)).to(self.device))
            self.b.append(torch.zeros(cout, dtype=torch.float32, device=self.device))
        self._init_state()

    def _init_state(self):
        self.wbf = [w.to(torch.bfloat16) for w in self.w]
        for wf, wb in zip(self.w, self.wbf):  # the library's rounding, so the mirrors match Adam's
            mpm.mpm_cast_f32_to_bf16(wf.numel(), wf.data_ptr(), wb.data_ptr(), _stream())
        # the tensor-core forward's layout of every layer's BF16 weights
        self.wtc = [torch.zeros(mpm.mpm_conv3d_tc_packed_bytes(CHANNELS[i], CHANNELS[i + 1]), dtype=torch.uint8,
                                device=self.device) for i in range(4)]
        # the adjoint layers of the tensor-core input gradient (layers 1-3; the input's gradient is not needed)
        self.wadj = [None] + [torch.zeros(mpm.mpm_conv3d_tc_adjoint_packed_bytes(CHANNELS[i], CHANNELS[i + 1]),
                                          dtype=torch.uint8, device=self.device) for i in range(1, 4)]
        self._pack()
        self.engine = "tc"
        self.backward_engine = "tc"  # weight and input gradients on the tensor cores ("mma": mma.sync kernels)
        self.params = [t for pair in zip(self.w, self.b) for t in pair]
        self.grads = [torch.zeros_like(p) for p in self.params]
        self.m = [torch.zeros_like(p) for p in self.params]
        self.v = [torch.zeros_like(p) for p in self.params]
        self.t = 0
        self._bufs = {}

    def _pack(self, stream=None):
        s = _stream(stream)
        for i in range(4):
            mpm.mpm_conv3d_pack_tc(CHANNELS[i], CHANNELS[i + 1], self.wbf[i].data_ptr(), self.wtc[i].data_ptr(), s)
        for i in range(1, 4):
            mpm.mpm_conv3d_pack_tc_adjoint(CHANNELS[i], CHANNELS[i + 1], self.wbf[i].data_ptr(),
                                           self.wadj[i].data_ptr(), s)

    # ---------------------------------------------------------------- persistence
    def save(self, path: str, meta: dict | None = None):
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        arrays = {f"w{i}": self.w[i].cpu().numpy() for i in range(4)}
        arrays.update({f"b{i}": self.b[i].cpu().numpy() for i in range(4)})
        arrays["meta"] = np.array(json.dumps(meta or {}))
        np.savez(path, **arrays)

    @classmethod
    def load(cls, path: str, device="cuda") -> "Network":
        d = np.load(path)
        net = cls.__new__(cls)
        net.device = torch.device(device)
        net.w = [torch.from_numpy(d[f"w{i}"]).to(net.device) for i in range(4)]
        net.b = [torch.from_numpy(d[f"b{i}"]).to(net.device) for i in range(4)]
        net.meta = json.loads(str(d["meta"])) if "meta" in d else {}
        net._init_state()
        return net

    # ---------------------------------------------------------------- buffers
    def _buffers(self, dims):
        if dims not in self._bufs:
            dev = self.device
            acts = [None] + [torch.empty(dims + (CHANNELS[i + 1],), dtype=torch.bfloat16, device=dev)
                             for i in range(3)]
            out = torch.empty(dims + (3,), dtype=torch.float32, device=dev)
            gbuf = [torch.empty(dims + (c,), dtype=torch.bfloat16, device=dev) for c in CHANNELS[1:]]
            gpad = torch.empty(dims + (4,), dtype=torch.bfloat16, device=dev)  # the output gradient, 3 -> 4 channels
            nt = mpm.mpm_conv3d_tile_count(*dims)
            self._bufs[dims] = {"acts": acts, "out": out, "g": gbuf, "gpad": gpad,
                                "loss": torch.zeros(2, dtype=torch.float32, device=dev),
                                "flags": torch.zeros((2, nt), dtype=torch.uint8, device=dev),
                                "dist": torch.zeros(mpm.mpm_conv3d_tc_tile_count(*dims), dtype=torch.uint8,
                                                    device=dev)}
        return self._bufs[dims]

    # ---------------------------------------------------------------- passes
    def forward(self, x_bf16: torch.Tensor, mask: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """x: (D, H, W, 4) BF16 -> (D, H, W, 3) FP32 (in DV_UNIT units). Keeps activations for backward.

        With a voxel mask (one byte per voxel), outputs are needed only on it: the last layer computes
        the 4 x 8 x 8 tiles holding masked voxels, the hidden layers those tiles and their neighbours (the
        three hidden layers reach 3 voxels, less than a tile), the rest is written as zeros. Outputs on
        the mask are the same as without it."""
        dims = tuple(x_bf16.shape[:3])
        bufs = self._buffers(dims)
        bufs["acts"][0] = x_bf16
        s = _stream(stream)
        if self.engine == "tc":  # tensor-core forward: tiles within 3 - i voxels of the mask for layer i
            dist = bufs["dist"]
            if mask is not None:
                mpm.mpm_conv3d_tc_tile_dist(*dims, mask.data_ptr(), dist.data_ptr(), s)
            for i in range(4):
                last = i == 3
                y = bufs["out"] if last else bufs["acts"][i + 1]
                mpm.mpm_conv3d_forward_tc(*dims, CHANNELS[i], CHANNELS[i + 1], bufs["acts"][i].data_ptr(),
                                          self.wtc[i].data_ptr(), self.b[i].data_ptr(), 0 if last else 1,
                                          1 if last else 0, y.data_ptr(), dist.data_ptr() if mask is not None else 0,
                                          3 - i, s)
            return bufs["out"]
        flags = bufs["flags"]
        if mask is not None:
            mpm.mpm_conv3d_tile_flags(*dims, mask.data_ptr(), 0, flags[0].data_ptr(), s)
            mpm.mpm_conv3d_tile_flags(*dims, mask.data_ptr(), 1, flags[1].data_ptr(), s)
        for i in range(4):
            last = i == 3
            y = bufs["out"] if last else bufs["acts"][i + 1]
            if mask is None:
                mpm.mpm_conv3d_forward(mpm.MPM_NET_BF16, *dims, CHANNELS[i], CHANNELS[i + 1],
                                       bufs["acts"][i].data_ptr(), self.wbf[i].data_ptr(), self.b[i].data_ptr(),
                                       0 if last else 1, 1 if last else 0, y.data_ptr(), s)
            else:
                mpm.mpm_conv3d_forward_tiled(*dims, CHANNELS[i], CHANNELS[i + 1], bufs["acts"][i].data_ptr(),
                                             self.wbf[i].data_ptr(), self.b[i].data_ptr(), 0 if last else 1,
                                             1 if last else 0, y.data_ptr(), flags[0 if last else 1].data_ptr(), s)
        return bufs["out"]

    def loss_and_backward(self, target: torch.Tensor, mask: torch.Tensor, stream=None) -> torch.Tensor:
        """Masked MSE of the last forward's output against target (FP32, DV_UNIT units); fills the
        gradients. Returns the loss as a 2-float device tensor (loss, masked voxels)."""
        dims = tuple(target.shape[:3])
        bufs = self._buffers(dims)
        s = _stream(stream)
        nvox = dims[0] * dims[1] * dims[2]
        g = bufs["g"][3]
        mpm.mpm_mse_loss(mpm.MPM_NET_BF16, nvox, 3, bufs["out"].data_ptr(), 1, target.data_ptr(), mask.data_ptr(),
                         bufs["loss"].data_ptr(), g.data_ptr(), s)
        for i in range(3, -1, -1):
            tc = self.backward_engine == "tc"
            dy = g
            if tc and CHANNELS[i + 1] < 4:  # the tensor-core kernels read 4, 16 or 32 channels
                mpm.mpm_pad_channels_bf16(nvox, CHANNELS[i + 1], 4, g.data_ptr(), bufs["gpad"].data_ptr(), s)
                dy = bufs["gpad"]
            if tc:  # tcgen05: voxels as the contraction, both operands read MN-major from channel planes
                mpm.mpm_conv3d_backward_weight_tc(*dims, CHANNELS[i], CHANNELS[i + 1], bufs["acts"][i].data_ptr(),
                                                  dy.data_ptr(), self.grads[2 * i].data_ptr(),
                                                  self.grads[2 * i + 1].data_ptr(), s)
            else:
                mpm.mpm_conv3d_backward_weight(mpm.MPM_NET_BF16, *dims, CHANNELS[i], CHANNELS[i + 1],
                                               bufs["acts"][i].data_ptr(), g.data_ptr(), self.grads[2 * i].data_ptr(),
                                               self.grads[2 * i + 1].data_ptr(), s)
            if i > 0:
                gx = bufs["g"][i - 1]
                if tc:  # tcgen05: the forward kernel on the adjoint weights
                    mpm.mpm_conv3d_backward_data_tc(*dims, CHANNELS[i], CHANNELS[i + 1], dy.data_ptr(),
                                                    self.wadj[i].data_ptr(), bufs["acts"][i].data_ptr(),
                                                    gx.data_ptr(), s)
                else:
                    mpm.mpm_conv3d_backward_data(mpm.MPM_NET_BF16, *dims, CHANNELS[i], CHANNELS[i + 1], g.data_ptr(),
                                                 self.wbf[i].data_ptr(), bufs["acts"][i].data_ptr(), gx.data_ptr(), s)
                g = gx
        return bufs["loss"]

    def step(self, lr: float, stream=None):
        self.t += 1
        s = _stream(stream)
        for j, p in enumerate(self.params):
            mirror = self.wbf[j // 2].data_ptr() if j % 2 == 0 else 0
            mpm.mpm_adam_step(p.numel(), p.data_ptr(), self.grads[j].data_ptr(), self.m[j].data_ptr(),
                              self.v[j].data_ptr(), self.t, lr, 0.9, 0.999, 1e-8, mirror, s)
        self._pack(stream)


# -------------------------------------------------------------------- windows on a simulation

class Window:
    """Device buffers for one box: FP32 features, BF16 network input, mask."""

    def __init__(self, dims, device):
        self.dims = dims
        self.feat = torch.empty(dims + (4,), dtype=torch.float32, device=device)
        self.xbf = torch.empty(dims + (4,), dtype=torch.bfloat16, device=device)
        self.mask = torch.empty(dims, dtype=torch.uint8, device=device)


class Attached:
    """The network attached to a one-env ``Sim``: environment steps run inside the library as graph-replayed
    windows with the gate on the device (``mpm_surrogate_step``)."""

    def __init__(self, sim, net: Network, rho: float, max_voxels: int = 96 ** 3, k: int = K,
                 threshold: float = THRESHOLD):
        self.sim, self.net = sim, net
        cfg = mpm.mpm_surrogate_net()
        for i in range(4):
            cfg.w_packed[i] = net.wtc[i].data_ptr()
            cfg.bias[i] = net.b[i].data_ptr()
        cfg.m_scale, cfg.v_scale, cfg.dv_unit = mass_scale(rho, sim.n), V_SCALE, DV_UNIT
        cfg.v_ref, cfg.threshold, cfg.k, cfg.margin = V_REF, threshold, k, MARGIN
        self.cfg = cfg
        nbytes = mpm.mpm_surrogate_workspace_size(max_voxels, sim.cfg.max_particles)
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=sim.device)
        mpm.mpm_surrogate_attach(sim.handle, cfg, self.ws.data_ptr(), nbytes, max_voxels)

    def env_step(self, pose, lin, ang, com, substeps: int = 25, gate=True, stream=None):
        # gate: False/0 off, True/1 per-step fallback, 2 per-window branches (mpm_surrogate_step)
        self.sim.set_colliders(pose, lin, ang, com, stream=stream)
        mpm.mpm_surrogate_step(self.sim.handle, substeps, int(gate), _stream(stream))

    def stats(self, reset: bool = False):
        return mpm.mpm_surrogate_stats(self.sim.handle, int(reset), _stream())

    def detach(self):
        mpm.mpm_surrogate_attach(self.sim.handle, None, 0, 0, 0)


class Runner:
    """Advances a one-env ``Sim`` by environment steps made of surrogate windows, with the gate, driving
    each window from the host (used to generate training data and in tests)."""

    def __init__(self, sim, net: Network | None, rho: float, k: int = K, threshold: float = THRESHOLD):
        self.sim, self.net, self.k, self.threshold = sim, net, k, threshold
        self.m_scale = mass_scale(rho, sim.n)
        self.windows = 0
        self.fallbacks = 0
        self.residuals = []
        self._win = {}
        self._zero = {}

    def window_buffers(self, box):
        dims = box.dims()
        if dims not in self._win:
            self._win[dims] = Window(dims, self.sim.device)
        return self._win[dims]

    def box(self, stream=None):
        return mpm.mpm_surrogate_box(self.sim.handle, MARGIN, _stream(stream))

    def start(self, box, stream=None) -> Window:
        w = self.window_buffers(box)
        s = _stream(stream)
        mpm.mpm_surrogate_features(self.sim.handle, box, self.m_scale, V_SCALE, w.feat.data_ptr(), w.mask.data_ptr(), s)
        return w

    def correction(self, w: Window, stream=None) -> torch.Tensor:
        """The network's output for a started window (zeros without a network)."""
        if self.net is None:
            if w.dims not in self._zero:
                self._zero[w.dims] = torch.zeros(w.dims + (3,), dtype=torch.float32, device=self.sim.device)
            return self._zero[w.dims]
        s = _stream(stream)
        n = w.feat.numel()
        mpm.mpm_cast_f32_to_bf16(n, w.feat.data_ptr(), w.xbf.data_ptr(), s)
        return self.net.forward(w.xbf, w.mask, stream)

    def window(self, box, gate: bool = True, stream=None):
        """One window of k substeps: surrogate if the gate passes, else plain."""
        w = self.start(box, stream)
        dv = self.correction(w, stream)
        s = _stream(stream)
        ok = True
        if gate:
            r = mpm.mpm_surrogate_check(self.sim.handle, box, dv.data_ptr(), DV_UNIT, self.k, V_REF, s)
            self.residuals.append(r[:2])
            ok = r[0] <= self.threshold and r[1] <= self.threshold
        self.windows += 1
        if ok:
            mpm.mpm_surrogate_advance(self.sim.handle, box, dv.data_ptr(), DV_UNIT, self.k, s)
        else:
            self.fallbacks += 1
            mpm.mpm_surrogate_advance(self.sim.handle, box, 0, DV_UNIT, self.k, s)
        return ok

    def env_step(self, pose, lin, ang, com, substeps: int = 25, gate: bool = True, stream=None):
        """Upload the collider inputs and advance ``substeps`` (a multiple of k) by windows."""
        self.sim.set_colliders(pose, lin, ang, com, stream=stream)
        box = self.box(stream)
        if box.D == 0:
            self.sim.substep(substeps, stream=stream)
            return
        for _ in range(substeps // self.k):
            self.window(box, gate, stream)


# -------------------------------------------------------------------- data, training, evaluation

def make_sim(sc, device="cuda"):
    from .sim import Sim
    sim = Sim(sc.n, sc.dt, sc.material, sc.N, gravity=sc.gravity, bound=sc.bound, max_colliders=len(sc.shapes),
              device=device)
    sim.set_shapes(sc.shapes)
    return sim


def _upload(sim, sc):
    d = sim.device
    sim.set_particles(*(torch.from_numpy(a).to(d) for a in (sc.x, sc.v, sc.C, sc.F)))


def _read_x(sim) -> torch.Tensor:
    x = torch.empty((3, sim.N), dtype=torch.float32, device=sim.device)
    mpm.mpm_read_state(sim.handle, x.data_ptr(), 0, 0, 0, 1, _stream())
    return x


def wall_mask(box, n, bound, device):
    """Nodes of the box outside the sticky wall band."""
    idx = [torch.arange(o, o + d, device=device) for o, d in ((box.i0, box.D), (box.j0, box.H), (box.k0, box.W))]
    ok = [(a >= bound) & (a < n - bound) for a in idx]
    return ok[0][:, None, None] & ok[1][None, :, None] & ok[2][None, None, :]


def window_sample(sim, scratch, sc, box, m_scale, k=K):
    """Run one plain window from the sim's current state and return the training pair
    (features BF16 (D,H,W,4), mask u8 (D,H,W), target FP32 (D,H,W,3) in DV_UNIT units)."""
    dev = sim.device
    x0 = _read_x(sim)
    dims = box.dims()
    feat = torch.empty(dims + (4,), dtype=torch.float32, device=dev)
    mask = torch.empty(dims, dtype=torch.uint8, device=dev)
    s = _stream()
    mpm.mpm_surrogate_features(sim.handle, box, m_scale, V_SCALE, feat.data_ptr(), mask.data_ptr(), s)
    mpm.mpm_surrogate_advance(sim.handle, box, 0, DV_UNIT, k, s)
    x1 = _read_x(sim)
    vbar = ((x1 - x0) / (k * sc.dt)).contiguous()
    # mass-weighted mean window velocity at the nodes: a transfer of (x0, vbar) with no stress or C
    scratch.set_particles(x0, vbar)
    g = scratch.read_grid()[box.i0:box.i0 + box.D, box.j0:box.j0 + box.H, box.k0:box.k0 + box.W]
    m = g[..., 0]
    has = m > 0
    vstar = torch.where(has[..., None], g[..., 1:] / torch.where(has, m, 1.0)[..., None], 0.0)
    v1 = feat[..., 1:] / V_SCALE
    keep = has & (mask > 0) & wall_mask(box, sc.n, sc.bound, dev)
    target = torch.where(keep[..., None], (vstar - v1) / DV_UNIT, 0.0).contiguous()
    xbf = torch.empty(dims + (4,), dtype=torch.bfloat16, device=dev)
    mpm.mpm_cast_f32_to_bf16(feat.numel(), feat.data_ptr(), xbf.data_ptr(), s)
    return xbf, keep.to(torch.uint8).contiguous(), target


def generate(seeds, particles=200_000, env_steps=4, sample_steps=(1, 2, 3), windows_per_step=(0, 2),
             device="cuda", log=None):
    """Training windows from plain MPM rollouts of pinch scenes with the given seeds."""
    samples = []
    sim = scratch = None
    t0 = time.perf_counter()
    for i, seed in enumerate(seeds):
        sc = scenes.pinch_scene(seed=seed, N=particles)
        if sim is None:
            sim = make_sim(sc, device)
            from .sim import Sim
            scratch = Sim(sc.n, sc.dt, scenes.Material(scenes.PLASTICINE, rho=sc.material.rho, E=sc.material.E,
                                                       nu=sc.material.nu, yield_stress=sc.material.yield_stress,
                                                       p_vol=sc.material.p_vol), sc.N, gravity=sc.gravity,
                          bound=sc.bound, device=device)
        _upload(sim, sc)
        m_scale = mass_scale(sc.material.rho, sc.n)
        for step in range(env_steps):
            sim.set_colliders(*scenes.finger_state(sc, step * sc.substeps_per_env_step * sc.dt))
            if step not in sample_steps:
                sim.substep(sc.substeps_per_env_step)
                continue
            box = mpm.mpm_surrogate_box(sim.handle, MARGIN, _stream())
            for wi in range(sc.substeps_per_env_step // K):
                if wi in windows_per_step:
                    samples.append(window_sample(sim, scratch, sc, box, m_scale))
                else:
                    sim.substep(K)
        if log and (i + 1) % 100 == 0:
            log(f"generated {i + 1}/{len(seeds)} rollouts, {len(samples)} windows, {time.perf_counter() - t0:.1f}s")
    for s_ in (sim, scratch):
        if s_ is not None:
            s_.close()
    return samples


def train(net: Network, samples, epochs=6, lr=1e-3, lr_end=1e-4, seed=0, log=None):
    rng = np.random.default_rng(seed)
    steps = epochs * len(samples)
    it = 0
    history = []
    for ep in range(epochs):
        order = rng.permutation(len(samples))
        acc = torch.zeros((), dtype=torch.float64, device=net.device)
        for idx in order:
            x, mask, target = samples[idx]
            frac = it / max(steps - 1, 1)
            rate = lr_end + 0.5 * (lr - lr_end) * (1.0 + math.cos(math.pi * frac))  # cosine decay
            net.forward(x, mask)
            loss = net.loss_and_backward(target, mask)
            net.step(rate)
            acc += loss[0].double()
            it += 1
        mean = float(acc) / len(samples)
        history.append(mean)
        if log:
            log(f"epoch {ep + 1}/{epochs}: mean loss {mean:.5f}")
    return history


_ZERO = {}


def zero_net(device):
    """A network whose output is zero (all weights and biases zero): the window without a correction."""
    if device not in _ZERO:
        z = Network(device=device, seed=0)
        for t in z.w + z.b:
            t.zero_()
        z._init_state()
        _ZERO[device] = z
    return _ZERO[device]


def evaluate(net: Network | None, seeds, particles=200_000, warm_steps=2, device="cuda", gate=True, warmup=True,
             steps=4):
    """Per held-out scene: after ``warm_steps`` plain env steps, ``steps`` env steps by the plain method and
    the same by windows (with ``net``, or with a zero correction when None) from the same state, the fingers
    following their scripts. Errors compare the positions after the first env step; the timings are the
    mean time per env step over the ``steps`` consecutive steps (graphs captured beforehand, off the
    clock)."""
    out = {"rel_x": [], "mean_abs": [], "rel_disp": [], "rel_x_last": [], "windows": 0, "fallbacks": 0,
           "ms_plain": [], "ms_surrogate": []}
    sim = None
    for seed in seeds:
        sc = scenes.pinch_scene(seed=seed, N=particles)
        if sim is None:
            sim = make_sim(sc, device)
        _upload(sim, sc)
        for step in range(warm_steps):
            sim.set_colliders(*scenes.finger_state(sc, step * 25 * sc.dt))
            sim.substep(25)
        snap = sim.read_state(on_device=True)
        cols = [scenes.finger_state(sc, (warm_steps + i) * 25 * sc.dt) for i in range(steps)]

        def restore():
            sim.set_particles(snap["x"], snap["v"], snap["C"], snap["F"])

        def run(step_fn, n):
            for i in range(n):
                step_fn(cols[i])

        def timed(step_fn):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            run(step_fn, steps)
            b.record()
            b.synchronize()
            return a.elapsed_time(b) / steps

        def plain_step(c):
            sim.set_colliders(*c)
            sim.substep(25)

        runner = Attached(sim, net if net is not None else zero_net(sim.device), sc.material.rho)

        def sur_step(c):
            runner.env_step(*c, gate=gate)

        # accuracy: positions after the first env step and after all of them (this also captures the
        # graphs of both state parities, so the timed runs below replay only)
        run(plain_step, 1)
        x_plain = _read_x(sim).double()
        restore()
        run(plain_step, steps)
        x_plain_last = _read_x(sim).double()
        restore()
        run(sur_step, 1)
        x_sur = _read_x(sim).double()
        restore()
        run(sur_step, steps)
        x_sur_last = _read_x(sim).double()
        runner.stats(reset=True)
        # timing: consecutive env steps, nothing read back in between
        if warmup:
            restore()
            run(plain_step, min(2, steps))
        restore()
        ms_p = timed(plain_step)
        restore()
        ms_s = timed(sur_step)
        w_, f_, _ = runner.stats(reset=True)
        runner.detach()
        d = x_sur - x_plain
        out["rel_x"].append(float(d.norm() / x_plain.norm()))
        out["mean_abs"].append(float(d.norm(dim=0).mean()))
        disp = x_plain - snap["x"].double()
        out["rel_disp"].append(float(d.norm() / disp.norm().clamp_min(1e-30)))
        out["rel_x_last"].append(float((x_sur_last - x_plain_last).norm() / x_plain_last.norm()))
        out["windows"] += w_ if gate else 5 * steps
        out["fallbacks"] += f_ if gate else 0
        out["ms_plain"].append(ms_p)
        out["ms_surrogate"].append(ms_s)
    if sim is not None:
        sim.close()
    return out


def summarize(res):
    return {
        "scenes": len(res["rel_x"]),
        "rel_x_mean": float(np.mean(res["rel_x"])),
        "rel_x_max": float(np.max(res["rel_x"])),
        "mean_abs_dx": float(np.mean(res["mean_abs"])),
        "rel_to_displacement_mean": float(np.mean(res["rel_disp"])),
        "rel_x_after_all_steps_mean": float(np.mean(res["rel_x_last"])),
        "fallback_rate": res["fallbacks"] / max(res["windows"], 1),
        "ms_per_env_step_plain": float(np.median(res["ms_plain"])),
        "ms_per_env_step_surrogate": float(np.median(res["ms_surrogate"])),
    }


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    tr = sub.add_parser("train")
    tr.add_argument("--out", default=WEIGHTS)
    tr.add_argument("--rollouts", type=int, default=2000)
    tr.add_argument("--first-seed", type=int, default=10000)
    tr.add_argument("--epochs", type=int, default=48)
    tr.add_argument("--lr", type=float, default=1e-3)
    tr.add_argument("--eval-scenes", type=int, default=32)
    ev = sub.add_parser("eval")
    ev.add_argument("--weights", default=WEIGHTS)
    ev.add_argument("--scenes", type=int, default=256)
    args = ap.parse_args()
    from . import build
    build.build()

    def log(msg):
        print(msg, flush=True)

    if args.cmd == "train":
        t0 = time.perf_counter()
        samples = generate(range(args.first_seed, args.first_seed + args.rollouts), log=log)
        t_gen = time.perf_counter() - t0
        net = Network(seed=0)
        t1 = time.perf_counter()
        hist = train(net, samples, epochs=args.epochs, lr=args.lr, log=log)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t1
        res = summarize(evaluate(net, range(20000, 20000 + args.eval_scenes)))
        meta = {"rollouts": args.rollouts, "seeds": [args.first_seed, args.first_seed + args.rollouts - 1],
                "windows": len(samples), "epochs": args.epochs, "lr": args.lr, "loss_history": hist,
                "generation_s": t_gen, "training_s": t_train, "eval": res, "k": K, "v_scale": V_SCALE,
                "dv_unit": DV_UNIT, "margin": MARGIN}
        net.save(args.out, meta)
        log(json.dumps(meta))
    else:
        net = Network.load(args.weights)
        seeds = range(20000, 20000 + args.scenes)
        res = {"surrogate": summarize(evaluate(net, seeds)), "no_network": summarize(evaluate(None, seeds))}
        log(json.dumps(res))


if __name__ == "__main__":
    main()
