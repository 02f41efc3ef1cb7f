"""Benchmark of the MLS-MPM substep: particle-substeps/s on the 200k-particle pinch scene.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

A step is one environment step of the pinch scene: the fingers' poses and velocities are copied in
(mpm_set_colliders), then 25 substeps run (mpm_substep), each a full pass of the hot path (bin sort,
grid update with colliders, fused G2P/P2G). Inputs are resident in HBM when the timed region starts;
L2 (129 MB) is flushed by writing a 512 MB buffer before every timed step, outside the events.
The metric counts particles x substeps per second over all ranks (N > 1 runs independent replicas,
one scene per GPU, seeds 1000 + rank).

The JSON line also carries:
  e2e          the same metric measured through the C-ABI with host buffers: collider poses copied in
               from pinned host memory, positions and per-finger impulses read back to pinned host
               memory, every step, inside the timed region;
  roofline     the fused G2P/P2G kernel (the dominant one): algorithmic bytes (192 B per
               particle-substep: x, v, C, F read and written in FP32) per launch / mean launch time
               from CUDA events bracketing each launch during the timed region, against the measured
               HBM copy bandwidth; plus its DRAM traffic per launch from the committed ncu summary when
               it was taken on the current kernel source;
  cpu_baseline the FP64 oracle (single thread) on one environment step of the same scene;
  clocks       nvidia-smi samples taken during the timed region;
  batched      256 envs (64^3 grids, 20k-120k particles, plasticine and fluid, a box tool each) in one
               handle: env-steps/s, particle-substeps/s, autotuned launch shape, and the same envs run
               one handle per env (the per-scene form) for comparison;
  serving      1,024 envs (2k-200k particles log-uniform, 48^3-96^3 grids, a box and a capsule each):
               env-steps/s and p50/p99 latency of an env step that reads its impulses back.
--impl reference times the oracle itself on a bounded particle sample of the same scene.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "pinch_200k_64cubed"
METRIC = "MPM particle-substeps/s on 1 GB300; batched env-steps/s at ≤1e-3 rel. error"
UNIT = "particle-substeps/s"
BYTES_PER_PARTICLE_SUBSTEP = 192  # x, v, C, F in FP32, read and written
SUBSTEPS = 25


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def code_digest(sources) -> str:
    """Hash of the code of C/CUDA source texts: comments, blank lines and trailing spaces are left out, so
    a change of wording alone keeps the hash."""
    h = hashlib.sha256()
    for src in sources:
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        h.update("\n".join(line.rstrip() for line in src.splitlines() if line.strip()).encode())
    return h.hexdigest()[:16]


FLAG_NAMES = {0x1: "clamped (a particle reached the 2 dx margin of the domain)",
              0x2: "nonfinite", 0x4: "singular value clamped", 0x8: "far move (slow path)",
              0x80000000: "internal"}


def flag_names(flags: int):
    """The sticky device flags (MPM_FLAG_*) set, by name."""
    return [name for bit, name in FLAG_NAMES.items() if flags & bit]


def kernel_source_hash() -> str:
    """code_digest of the sources the fused substep kernel (k_g2p2g) is compiled from."""
    csrc = os.path.join(ROOT, "paper_2302_04659_gb300", "csrc")
    return code_digest(open(os.path.join(csrc, fn), encoding="utf-8").read()
                       for fn in ("mpm_device.cuh", "mpm_internal.h", "mpm_kernels.cu"))


# FP32 flops per particle-substep of the fused kernel (FMA counted as 2): ncu instruction counters of
# the 600k-particle pinch capture, 8.30e8 flops per launch / 600,000 particles.
FP32_FLOPS_PER_PARTICLE_SUBSTEP = 1383


def fp32_peak_tflops(sm_mhz: float | None) -> float:
    """Dense FP32 FMA peak of a GB300: 152 SMs x 128 lanes x 2 flops at the given SM clock."""
    return 152 * 128 * 2 * (sm_mhz or 2070.0) * 1e6 / 1e12


def measured_peak_gbs():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def traffic_per_launch(src_hash: str):
    """DRAM bytes per g2p2g launch from the committed ncu summary, if it was taken on this source."""
    p = os.path.join(ROOT, "profiles", "g2p2g_traffic.json")
    try:
        d = json.load(open(p))
    except Exception:
        return None
    if d.get("kernel_source_hash") != src_hash:
        return None
    return d.get("dram_bytes_per_launch_full_size")


class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons during the timed region."""

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        self.out = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is None:
            return
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        self.out = out

    def summary(self):
        if not self.out:
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.strip().splitlines():
            f = [c.strip() for c in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def job_throughput(local_units, local_seconds, device=None):
    """Whole-job throughput over the ranks of an initialized process group (one rank: just local):
    units summed over ranks divided by the slowest rank's time. Returns (value, max seconds, units)."""
    import torch
    import torch.distributed as dist
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return u.item() / t.item(), t.item(), u.item()


def pinch_inputs(seed, N=200_000):
    from paper_2302_04659_gb300 import scenes
    return scenes.pinch_scene(seed=seed, N=N)


def run_native(args):
    import torch
    import torch.distributed as dist

    from paper_2302_04659_gb300 import build as b
    from paper_2302_04659_gb300 import scenes
    from paper_2302_04659_gb300.sim import Sim

    rank, world, local = env_rank()
    b.build()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    sc = pinch_inputs(1000 + rank, args.particles)
    N = sc.N
    sim = Sim(sc.n, sc.dt, sc.material, N, gravity=sc.gravity, bound=sc.bound, max_colliders=len(sc.shapes),
              device=dev)
    xd = torch.from_numpy(sc.x).to(dev)
    vd = torch.from_numpy(sc.v).to(dev)
    Cd = torch.from_numpy(sc.C).to(dev)
    Fd = torch.from_numpy(sc.F).to(dev)
    sim.set_shapes(sc.shapes)
    stream = torch.cuda.current_stream(dev)
    k = len(sc.shapes)
    # pinned host buffers for the collider inputs of every step
    pose_h = torch.empty((k, 7), dtype=torch.float32).pin_memory()
    lin_h = torch.empty((k, 3), dtype=torch.float32).pin_memory()
    ang_h = torch.empty((k, 3), dtype=torch.float32).pin_memory()
    com_h = torch.empty((k, 3), dtype=torch.float32).pin_memory()
    from paper_2302_04659_gb300 import _native as mpm

    def set_colliders(step):
        pose, lin, ang, com = scenes.finger_state(sc, step * SUBSTEPS * sc.dt)
        pose_h.numpy()[:] = pose
        lin_h.numpy()[:] = lin
        ang_h.numpy()[:] = ang
        com_h.numpy()[:] = com
        mpm.mpm_set_colliders(sim.handle, k, pose_h.data_ptr(), lin_h.data_ptr(), ang_h.data_ptr(),
                              com_h.data_ptr(), int(stream.cuda_stream))

    def env_step(step):
        set_colliders(step)
        mpm.mpm_substep(sim.handle, SUBSTEPS, int(stream.cuda_stream))

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    sim.set_particles(xd, vd, Cd, Fd)
    for s in range(args.warmup):
        env_step(s)
    def timed_pass(first_step):
        """K env steps, each bracketed by events on the launching stream, L2 flushed before each."""
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        barrier()
        for s in range(args.steps):
            flush.fill_(float(s))
            ev[s][0].record(stream)
            env_step(first_step + s)
            ev[s][1].record(stream)
        barrier()
        return sum(a.elapsed_time(b) for a, b in ev) / 1e3

    # ---------------- timed region (device-resident inputs), no instrumentation inside the steps
    l0 = sim.launches
    wall0 = time.perf_counter()
    with ClockSampler(local) as clk:
        elapsed = timed_pass(args.warmup)
    wall = time.perf_counter() - wall0
    launches = sim.launches - l0
    # ---------------- the same steps again with CUDA events bracketing every launch of every kernel (event
    # nodes inside the replayed graphs): the fused G2P/P2G kernel's share of the device time. Events between
    # kernels remove the programmatic launch overlap, so this pass is slower; the kernel's time per launch is
    # its share of this pass times the headline pass's time per substep
    sim.set_timing(True)
    sim.read_timing(reset=True)
    elapsed_instrumented = timed_pass(args.warmup + args.steps)
    ktime = sim.read_timing(reset=True)
    sim.set_timing(False)
    # ---------------- the same steps with plain launches (no graph replay), for comparison
    sim.set_graphs(False)
    elapsed_plain = timed_pass(args.warmup + 2 * args.steps)
    sim.set_graphs(True)
    value, elapsed, total_units = job_throughput(N * SUBSTEPS * args.steps, elapsed, dev)
    flags = sim.status()
    g_ms, g_n = ktime["g2p2g"]
    g_evt = g_ms / max(g_n, 1) / 1e3  # seconds per launch with events around every launch
    share = g_ms / max(sum(v[0] for v in ktime.values()), 1e-30)
    substeps = SUBSTEPS * args.steps
    g_avg = share * elapsed / substeps  # seconds per launch, consistent with the headline pass
    if g_n != substeps or g_avg > elapsed / substeps * (1 + 1e-9):
        raise RuntimeError(f"k_g2p2g timing: {g_n} launches for {substeps} substeps, {g_avg:.3e} s per launch")
    # ---------------- end-to-end through the C-ABI with host buffers: the same env steps as the device
    # pass (same warm-up, L2 flushed before each step outside its events), each step's events bracketing
    # the collider upload from pinned host memory, the substeps, and the read-back of the step's positions,
    # impulses and substep count into page-locked host memory (asynchronous, in stream order: the host
    # never waits inside the loop, the closing barrier waits for the last copy)
    e2e_steps = args.steps if not args.no_e2e else 0
    x_h = torch.empty((3, N), dtype=torch.float32).pin_memory()
    wr_h = torch.empty((k, 6), dtype=torch.float64).pin_memory()
    cnt_h = torch.empty(1, dtype=torch.int32).pin_memory()
    sim.set_particles(xd, vd, Cd, Fd)
    for s in range(args.warmup):
        env_step(s)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(e2e_steps)]
    barrier()
    for s in range(e2e_steps):
        flush.fill_(float(s))
        ev[s][0].record(stream)
        env_step(args.warmup + s)
        mpm.mpm_read_state(sim.handle, x_h.data_ptr(), 0, 0, 0, 2, int(stream.cuda_stream))
        mpm.mpm_read_wrench_async(sim.handle, wr_h.data_ptr(), cnt_h.data_ptr(), int(stream.cuda_stream))
        ev[s][1].record(stream)
    barrier()
    e2e_value = (job_throughput(N * SUBSTEPS * e2e_steps, sum(a.elapsed_time(b) for a, b in ev) / 1e3, dev)[0]
                 if e2e_steps else None)
    h2d = k * (7 + 3 + 3 + 3) * 4
    d2h = 3 * N * 4 + k * 6 * 8 + 4
    if e2e_steps and int(cnt_h[0]) != SUBSTEPS:  # the last step's read arrived: 25 substeps since its upload
        raise RuntimeError(f"e2e read-back: substep count {int(cnt_h[0])}, expected {SUBSTEPS}")
    sim.close()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return None
    peak, peak_kind = measured_peak_gbs()
    src_hash = kernel_source_hash()
    clk_mhz = (clk.summary() or {}).get("sm_mhz")
    achieved = BYTES_PER_PARTICLE_SUBSTEP * N / g_avg / 1e9 if g_avg > 0 else None
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": elapsed / args.steps * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded ellipsoid of plasticine, scripted capsule fingers)",
        "config": {
            "workload": WORKLOAD,
            "particles_per_gpu": N,
            "grid": f"{sc.n}^3",
            "substeps_per_step": SUBSTEPS,
            "colliders": "2 capsules r=0.02, friction 0.5",
            "material": "plasticine E=5e3 nu=0.3 yield=50 rho=1e3",
            "dt": sc.dt,
            "l2": "flushed before every timed step (512 MB write, outside the events)",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "rollout_phase": (f"env steps {args.warmup}-{args.warmup + args.steps - 1} of a rollout from the "
                              "initial ellipsoid (the blob settles and spreads: later steps touch more bins)"),
        },
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e2e_steps,
                "what": "collider upload from pinned host memory + 25 substeps + positions, impulses and substep "
                        "count read back to page-locked host memory, per env step, L2 flushed between steps"},
        "gpu_launches": launches,
        "plain_launches": {"value": N * SUBSTEPS * args.steps / elapsed_plain, "unit": UNIT,
                           "ms_per_step": elapsed_plain / args.steps * 1e3,
                           "what": "the same env steps launched kernel by kernel instead of replayed from a graph"},
        "roofline": {
            "kernel": "k_g2p2g",
            "bound": "hbm",
            "achieved": achieved,
            "peak": peak,
            "peak_kind": f"{peak_kind} HBM copy bandwidth",
            "unit": "GB/s",
            "frac": achieved / peak if achieved else None,
            "traffic": traffic_per_launch(src_hash),
            "algorithmic_bytes_per_launch": BYTES_PER_PARTICLE_SUBSTEP * N,
            "mean_launch_us": g_avg * 1e6,
            "share_of_substep": share,
            "launches": g_n,
            "timing": ("share of k_g2p2g in the device time of every kernel (CUDA events around each launch, "
                       "second pass) x the headline ms per substep"),
            "event_bracketed_us": g_evt * 1e6,
            "kernel_source_hash": src_hash,
            "note": "state (38 MB) fits the 129 MB L2 inside a step; L2 flushed between steps",
            "fp32": {
                "bound": "alu",
                "flops_per_particle_substep": FP32_FLOPS_PER_PARTICLE_SUBSTEP,
                "achieved": FP32_FLOPS_PER_PARTICLE_SUBSTEP * N / g_avg / 1e12 if g_avg > 0 else None,
                "peak": fp32_peak_tflops(clk_mhz),
                "unit": "TFLOP/s",
                "frac": (FP32_FLOPS_PER_PARTICLE_SUBSTEP * N / g_avg / 1e12 / fp32_peak_tflops(clk_mhz)
                         if g_avg > 0 else None),
                "what": ("FP32 flops of k_g2p2g per particle-substep (FMA = 2) counted by ncu on the 600k pinch "
                         "capture (profiles/g2p2g_pinch200k.md); peak = 152 SMs x 128 FP32 lanes x 2 x the "
                         "median SM clock sampled during the timed region"),
            },
        },
        "kernel_ms": {kname: {"ms": v[0], "launches": v[1]} for kname, v in ktime.items() if v[1]},
        "status_flags": flags,
        "status_flags_set": flag_names(flags),
        "wall_s": wall,
    }
    line["clocks"] = clk.summary()
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(sc)
    # the sections below come last in the line, the most read ones at the very end, in compact form
    batched = serving = None
    if world == 1 and not args.no_batched:
        batched = run_batched(dev, "batch256", args.batched_steps, 3, per_scene=True, tune=True)
        serving = run_batched(dev, "serve1024", args.batched_steps, 3, per_scene=False, tune=True)
        line["contact_forms"] = run_contact(dev, args.batched_steps * 4)
        line["render"] = run_render(dev, args.batched_steps * 5)
    if world == 1 and args.surrogate_scenes > 0:
        line["surrogate"] = run_surrogate(dev, args.surrogate_scenes)
    if batched is not None:
        line["batched_detail"] = {k: batched.pop(k) for k in ("autotune", "clocks", "status_flags_set", "grids")}
        line["batched"] = batched
        line["serving"] = serving
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return line


def run_batched(dev, which: str, steps: int, warmup: int, per_scene: bool, tune: bool, nenv: int = 0):
    """A batched workload in one handle: all envs advance together, one graph replay per env step.

    ``batch256``: 256 envs, 64^3 grids, 20k-120k particles (uniform, seeded), plasticine and fluid
    alternating, a box tool each. ``serve1024``: 1,024 envs, 2k-200k particles (log-uniform), 48^3-96^3
    grids, a box tool and a capsule finger each. Inputs are far larger than L2, so no flush is needed.
    Reports env-steps/s (envs x steps / time) and particle-substeps/s from a back-to-back pass, step
    latency percentiles from a pass that reads every step's impulses back to the host, and for
    ``batch256`` the same envs run one handle per env (the per-scene form) with the largest relative
    difference in positions between the two forms after one env step."""
    import torch

    from paper_2302_04659_gb300 import _native as mpm
    from paper_2302_04659_gb300 import autotune, scenes
    from paper_2302_04659_gb300.sim import BatchSim, Sim

    t_gen = time.perf_counter()
    if which == "batch256":
        envs = scenes.batch_workload(nenv or 256)
    else:
        envs = scenes.serving_workload(nenv or 1024)
    counts, (x, v, C, F) = scenes.concat_states(envs)
    t_gen = time.perf_counter() - t_gen
    sc0 = envs[0]
    dt = sc0.dt
    sim = BatchSim([(sc.n, sc.material, sc.N, len(sc.shapes)) for sc in envs], dt, gravity=sc0.gravity,
                   bound=sc0.bound, device=dev)
    xd, vd, Cd, Fd = (torch.from_numpy(a).to(dev) for a in (x, v, C, F))
    sim.set_particles(counts, xd, vd, Cd, Fd)
    sim.set_shapes([sc.shapes for sc in envs])
    paths = scenes.ToolPaths(envs)
    k = paths.k
    stream = torch.cuda.current_stream(dev)
    pin = {name: torch.empty((k, d), dtype=torch.float32).pin_memory()
           for name, d in (("pose", 7), ("lin", 3), ("ang", 3), ("com", 3))}
    wr_h = torch.empty((k, 6), dtype=torch.float64).pin_memory()
    N = int(sum(counts))

    def set_colliders(step, handle=sim.handle):
        for name, arr in zip(("pose", "lin", "ang", "com"), paths.at(step * SUBSTEPS * dt)):
            pin[name].numpy()[:] = arr
        mpm.mpm_set_colliders(handle, k, pin["pose"].data_ptr(), pin["lin"].data_ptr(), pin["ang"].data_ptr(),
                              pin["com"].data_ptr(), int(stream.cuda_stream))

    def env_step(step):
        set_colliders(step)
        mpm.mpm_substep(sim.handle, SUBSTEPS, int(stream.cuda_stream))

    def reset():
        sim.set_particles(counts, xd, vd, Cd, Fd)
        set_colliders(0)

    tuned = None
    if tune:
        shape, ms, trials = autotune.tune(sim, substeps=4, reps=2, prepare=lambda: set_colliders(0), restore=reset)
        tuned = {"shape": {"chunk": shape[0], "fused_ctas_per_sm": shape[1], "grid_ctas_per_sm": shape[2]},
                 "ms_per_substep": ms, "trials_ms_per_substep": trials}
    # positions after one env step from the initial state (compared with the per-scene form below)
    reset()
    mpm.mpm_substep(sim.handle, SUBSTEPS, int(stream.cuda_stream))
    x_batch = sim.read_state(on_device=True)["x"]
    reset()
    for s_ in range(warmup):
        env_step(s_)
    torch.cuda.synchronize(dev)
    # ---- throughput: back-to-back env steps, device-resident
    l0 = sim.launches
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index or 0) as clk:
        a.record(stream)
        for s_ in range(steps):
            env_step(warmup + s_)
        b.record(stream)
        torch.cuda.synchronize(dev)
    secs = a.elapsed_time(b) / 1e3
    launches = sim.launches - l0
    # ---- the fused kernel's share of the device time (events around every launch, a second pass), for its
    # roofline fraction with the state in HBM: algorithmic bytes 192 per plasticine particle-substep, 128
    # per fluid one (x, v, C and F or J, read and written in FP32)
    sim.set_timing(True)
    sim.read_timing(reset=True)
    for s_ in range(steps):
        env_step(warmup + s_)
    torch.cuda.synchronize(dev)
    kt = sim.read_timing(reset=True)
    sim.set_timing(False)
    share = kt["g2p2g"][0] / max(sum(v[0] for v in kt.values()), 1e-30)
    bytes_substep = sum(sc.N * (192 if sc.material.kind == scenes.PLASTICINE else 128) for sc in envs)
    g_s = share * secs / (steps * SUBSTEPS)
    peak, peak_kind = measured_peak_gbs()
    # ---- latency: every step reads its impulses back (host waits), per-step events
    lat = []
    for s_ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        env_step(warmup + steps + s_)
        mpm.mpm_read_wrench(sim.handle, wr_h.data_ptr(), int(stream.cuda_stream))
        e1.record(stream)
        e1.synchronize()
        lat.append(e0.elapsed_time(e1))
    # ---- per-env request latency: closed-loop clients, one per env, each sending its next request (its
    # tool's poses) a random think time (uniform in [0, one step]) after its previous answer. The server runs
    # batched env steps back to back; each step serves every request that has arrived when it starts (all
    # envs step; those without a new request keep their scripted poses) and ends when the impulses are back
    # on the host. A request's latency runs from its arrival to that read-back (host wall clock).
    rng = np.random.default_rng(7)
    T = secs / steps
    arrival = time.perf_counter() + rng.uniform(0.0, T, size=len(envs))
    req_lat = []
    for s_ in range(steps):
        start = time.perf_counter()
        if not (arrival <= start).any():  # nobody waiting: idle until the next request arrives
            time.sleep(max(0.0, float(arrival.min()) - start))
            start = time.perf_counter()
        served = arrival <= start
        env_step(warmup + 2 * steps + s_)
        mpm.mpm_read_wrench(sim.handle, wr_h.data_ptr(), int(stream.cuda_stream))
        end = time.perf_counter()
        req_lat.extend(((end - arrival[served]) * 1e3).tolist())
        arrival[served] = end + rng.uniform(0.0, T, size=int(served.sum()))
    flags = sim.status()
    shape_now = sim.get_launch()
    nenv = len(envs)
    out = {
        "workload": which,
        "envs": nenv,
        "particles": N,
        "grids": sorted({sc.n for sc in envs}),
        "materials": "plasticine/fluid alternating",
        "colliders": k,
        "substeps_per_env_step": SUBSTEPS,
        "steps": steps,
        "env_steps_per_s": nenv * steps / secs,
        "particle_substeps_per_s": N * SUBSTEPS * steps / secs,
        "ms_per_env_step": secs / steps * 1e3,
        "step_latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                            "what": "one batched env step of all envs: set colliders + 25 substeps + impulses "
                                    "read back to pinned host memory"},
        "request_latency_ms": {"p50": float(np.percentile(req_lat, 50)), "p99": float(np.percentile(req_lat, 99)),
                               "requests": len(req_lat),
                               "what": "per env request, closed-loop clients with think time U[0, one step]: "
                                       "arrival to its env's impulses on the host"},
        "gpu_launches": launches,
        "roofline": {"kernel": "k_g2p2g", "bound": "hbm", "achieved": bytes_substep / g_s / 1e9, "peak": peak,
                     "unit": "GB/s", "frac": bytes_substep / g_s / 1e9 / peak, "share_of_substep": share,
                     "mean_launch_us": g_s * 1e6, "algorithmic_bytes_per_launch": bytes_substep,
                     "peak_kind": f"{peak_kind} HBM copy bandwidth"},
        "launch_shape": {"chunk": shape_now[0], "fused_ctas_per_sm": shape_now[1], "grid_ctas_per_sm": shape_now[2]},
        "autotune": tuned,
        "status_flags": flags,
        "status_flags_set": flag_names(flags),
        "clocks": clk.summary(),
        "input_generation_s": t_gen,
        "l2": "inputs larger than L2 (not flushed)",
    }
    sim.close()
    del xd, vd, Cd, Fd
    if per_scene:
        # ---- the per-scene form: one handle per env, stepped one after another on the same stream
        sims = []
        off = np.concatenate([[0], np.cumsum(counts)])
        col_off = np.concatenate([[0], np.cumsum([len(sc.shapes) for sc in envs])])
        for e, sc in enumerate(envs):
            s1 = Sim(sc.n, sc.dt, sc.material, max(sc.N, 1), gravity=sc.gravity, bound=sc.bound,
                     max_colliders=len(sc.shapes), device=dev)
            s1.set_particles(*(torch.from_numpy(np.ascontiguousarray(a[:, off[e]:off[e + 1]])).to(dev)
                               for a in (x, v, C, F)))
            s1.set_shapes(sc.shapes)
            sims.append(s1)

        def per_scene_step(step):
            st = paths.at(step * SUBSTEPS * dt)
            for e, s1 in enumerate(sims):
                c0, c1 = col_off[e], col_off[e + 1]
                s1.set_colliders(*(arr[c0:c1] for arr in st), stream=stream)
                s1.substep(SUBSTEPS, stream=stream)

        per_scene_step(0)
        x_single = torch.cat([s1.read_state(on_device=True)["x"] for s1 in sims], dim=1)
        diffs = []
        for e in range(nenv):
            xs = x_single[:, off[e]:off[e + 1]].double()
            xb = x_batch[:, off[e]:off[e + 1]].double()
            diffs.append(float((xb - xs).norm() / xs.norm().clamp_min(1e-30)))
        ps_steps = max(2, min(steps, 4))
        for s_ in range(1, 2):
            per_scene_step(s_)
        torch.cuda.synchronize(dev)
        a.record(stream)
        for s_ in range(ps_steps):
            per_scene_step(2 + s_)
        b.record(stream)
        torch.cuda.synchronize(dev)
        ps_secs = a.elapsed_time(b) / 1e3
        for s1 in sims:
            s1.close()
        out["per_scene"] = {
            "env_steps_per_s": nenv * ps_steps / ps_secs,
            "particle_substeps_per_s": N * SUBSTEPS * ps_steps / ps_secs,
            "steps": ps_steps,
            "form": "one handle per env, each env step a collider upload and one graph replay, envs in turn",
        }
        out["speedup_vs_per_scene"] = out["env_steps_per_s"] / out["per_scene"]["env_steps_per_s"]
        out["max_rel_x_diff_vs_per_scene_after_one_env_step"] = max(diffs)
    return out


def run_contact(dev, steps: int, warmup: int = 3):
    """The two contact forms (Sec. 3) side by side on 200,000-particle plasticine scenes, 64^3 grid:
    the pinch scene (two capsule fingers) and the ring press (a spinning torus tool held as an SDF
    volume at half the grid spacing). Per scene and form: `steps` env steps of 25 substeps, graph
    replay, L2 flushed before each step (outside the events), the mean time per env step. Particle
    form: penalty stiffness 0.2/dt^2, damping 0.5/dt."""
    import torch

    from paper_2302_04659_gb300 import scenes
    from paper_2302_04659_gb300.sim import Sim

    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out = {"stiffness_dt2": 0.2, "damping_dt": 0.5, "l2": "flushed before every timed step"}
    for name, sc in (("pinch_capsules", scenes.pinch_scene(seed=1000, N=200_000)),
                     ("ring_press_sdf_volume", scenes.ring_press_scene(seed=4000, N=200_000))):
        res = {}
        for mode in ("grid", "particle"):
            sim = Sim(sc.n, sc.dt, sc.material, sc.N, gravity=sc.gravity, bound=sc.bound,
                      max_colliders=len(sc.shapes), device=dev)
            sim.set_shapes(sc.shapes)
            if mode == "particle":
                sim.set_contact("particle", 0.2 / sc.dt ** 2, 0.5 / sc.dt)
            sim.set_particles(*(torch.from_numpy(a).to(dev) for a in (sc.x, sc.v, sc.C, sc.F)))

            def env_step(i):
                sim.set_colliders(*scenes.finger_state(sc, i * SUBSTEPS * sc.dt), stream=stream)
                sim.substep(SUBSTEPS, stream=stream)

            for i in range(warmup):
                env_step(i)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            torch.cuda.synchronize(dev)
            for i in range(steps):
                flush.fill_(float(i))
                ev[i][0].record(stream)
                env_step(warmup + i)
                ev[i][1].record(stream)
            torch.cuda.synchronize(dev)
            ms = sum(a.elapsed_time(b) for a, b in ev) / steps
            wr, _ = sim.read_wrench()
            res[mode] = {"ms_per_env_step": ms, "particle_substeps_per_s": sc.N * SUBSTEPS / (ms / 1e3),
                         "status_flags": sim.status(), "last_impulse_norm": float(np.linalg.norm(wr[:, :3]))}
            sim.close()
        res["particle_over_grid_time"] = res["particle"]["ms_per_env_step"] / res["grid"]["ms_per_env_step"]
        out[name] = res
    return out


def run_render(dev, frames: int, warmup: int = 3):
    """The particle renderer (App. D.2 splatting) on the 200,000-particle pinch scene after one env step,
    rendered in place from the simulation's buffers (no copy): splat, distance-scaled bilateral filter
    (half window 4), normals and shading, at 640x480 and 1280x960. Mean time per frame over `frames`
    frames bracketed by CUDA events, L2 flushed before each (outside the events)."""
    import torch

    from paper_2302_04659_gb300 import scenes
    from paper_2302_04659_gb300.render import Camera, Renderer, Style
    from paper_2302_04659_gb300.sim import Sim

    sc = scenes.pinch_scene(seed=1000, N=200_000)
    sim = Sim(sc.n, sc.dt, sc.material, sc.N, gravity=sc.gravity, bound=sc.bound, max_colliders=len(sc.shapes),
              device=dev)
    sim.set_shapes(sc.shapes)
    sim.set_particles(*(torch.from_numpy(a).to(dev) for a in (sc.x, sc.v, sc.C, sc.F)))
    sim.set_colliders(*scenes.finger_state(sc, 0.1))
    sim.substep(SUBSTEPS)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out = {"particles": sc.N, "style": "radius 0.004, smooth 0.008, sigma_depth 0.01, half window 4",
           "l2": "flushed before every frame"}
    for W, H in ((640, 480), (1280, 960)):
        r = Renderer(Camera.looking(W, H, 40.0, (0.55, 0.55, -0.35), (0.5, 0.2, 0.5)),
                     Style(radius=0.004, smooth=0.008, sigma_depth=0.01, window=4), device=dev)
        for _ in range(warmup):
            r.render_sim(sim, stream=stream)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(frames)]
        torch.cuda.synchronize(dev)
        for i in range(frames):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            r.render_sim(sim, stream=stream)
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        ms = sum(a.elapsed_time(b) for a, b in ev) / frames
        drawn = float(torch.isfinite(r.depth).float().mean())
        out[f"{W}x{H}"] = {"ms_per_frame": ms, "frames_per_s": 1e3 / ms, "drawn_pixel_fraction": drawn,
                           "launches_per_frame": 4}
    sim.close()
    return out


def run_conv_scan(dev, reps: int = 20):
    """The surrogate network's tcgen05 convolution alone, per layer shape (4 -> 32, 32 -> 32, 32 -> 3)
    and box size, from one tile to a 64^3 box: mean time per launch over `reps` launches replayed from a
    CUDA graph (no host launch cost), and the dense TFLOP/s that implies. Random BF16 inputs."""
    import torch

    from paper_2302_04659_gb300 import _native as mpm

    torch.manual_seed(0)
    out = []
    for cin, cout in ((4, 32), (32, 32), (32, 3)):
        w = (torch.randn(27, cout, cin, device=dev) * 0.05).to(torch.bfloat16).contiguous()
        wp = torch.empty(mpm.mpm_conv3d_tc_packed_bytes(cin, cout), dtype=torch.uint8, device=dev)
        st = torch.cuda.Stream(dev)
        mpm.mpm_conv3d_pack_tc(cin, cout, w.data_ptr(), wp.data_ptr(), st.cuda_stream)
        bias = torch.zeros(cout, device=dev)
        for D, H, W in ((1, 16, 8), (1, 16, 8 * 152), (2, 16, 8 * 152), (4, 16, 8 * 152), (33, 38, 40),
                        (64, 64, 64)):
            x = torch.randn(D, H, W, cin, device=dev).to(torch.bfloat16).contiguous()
            y = torch.empty(D, H, W, cout, device=dev, dtype=torch.bfloat16)

            def conv():
                mpm.mpm_conv3d_forward_tc(D, H, W, cin, cout, x.data_ptr(), wp.data_ptr(), bias.data_ptr(), 1, 0,
                                          y.data_ptr(), 0, 0, st.cuda_stream)

            with torch.cuda.stream(st):
                for _ in range(3):
                    conv()
            torch.cuda.synchronize(dev)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=st):
                for _ in range(reps):
                    conv()
            with torch.cuda.stream(st):
                g.replay()
            torch.cuda.synchronize(dev)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(st):  # the graph replays on the current stream: time it there
                a.record()
                g.replay()
                b.record()
            b.synchronize()
            us = a.elapsed_time(b) / reps * 1e3
            out.append({"cin": cin, "cout": cout, "box": [D, H, W], "tiles": mpm.mpm_conv3d_tc_tile_count(D, H, W),
                        "us_per_launch": us, "tflops": 2.0 * D * H * W * 27 * cin * cout / us / 1e6})
    return {"what": "k_conv_tc forward, graph-replayed launches, CUDA events", "rows": out}


def run_train_timing(dev, reps: int = 20):
    """The surrogate network's training kernels on the pinch window box (33 x 38 x 40 nodes): per layer,
    the weight and bias gradients with the tcgen05 kernel (mpm_conv3d_backward_weight_tc) and with the
    mma.sync kernel it replaced (mpm_conv3d_backward_weight), each `reps` calls replayed from a CUDA graph
    (device time, no host launch cost), with the largest relative difference of their dW; then one
    training step (forward, masked MSE, backward) per backward engine, launched eagerly. Random inputs."""
    import torch

    from paper_2302_04659_gb300 import _native as mpm
    from paper_2302_04659_gb300 import surrogate as sur

    torch.manual_seed(0)
    D, H, W = 33, 38, 40
    C = sur.CHANNELS
    st = torch.cuda.Stream(dev)

    def graph_time(fn):
        with torch.cuda.stream(st):
            for _ in range(3):
                fn()
        torch.cuda.synchronize(dev)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            for _ in range(reps):
                fn()
        with torch.cuda.stream(st):
            g.replay()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            a.record()
            g.replay()
            b.record()
        b.synchronize()
        return a.elapsed_time(b) / reps * 1e3

    layers = []
    for i in range(4):
        cin, cout = C[i], C[i + 1]
        cd = 4 if cout <= 4 else (16 if cout <= 16 else 32)
        x = torch.randn(D, H, W, cin, device=dev).to(torch.bfloat16).contiguous()
        dy = torch.randn(D, H, W, cout, device=dev).to(torch.bfloat16).contiguous()
        dyp = torch.zeros(D, H, W, cd, device=dev, dtype=torch.bfloat16)
        dyp[..., :cout] = dy
        dw_m, db_m = torch.zeros(27 * cout * cin, device=dev), torch.zeros(cout, device=dev)
        dw_t, db_t = torch.zeros_like(dw_m), torch.zeros_like(db_m)
        s = st.cuda_stream

        def mma():
            mpm.mpm_conv3d_backward_weight(mpm.MPM_NET_BF16, D, H, W, cin, cout, x.data_ptr(), dy.data_ptr(),
                                           dw_m.data_ptr(), db_m.data_ptr(), s)

        def tc():
            mpm.mpm_conv3d_backward_weight_tc(D, H, W, cin, cout, x.data_ptr(), dyp.data_ptr(), dw_t.data_ptr(),
                                              db_t.data_ptr(), s)

        t_m, t_t = graph_time(mma), graph_time(tc)
        diff = float((dw_t - dw_m).abs().max() / dw_m.abs().max().clamp_min(1e-30))
        flops = 2.0 * D * H * W * 27 * cin * cout
        layers.append({"cin": cin, "cout": cout, "us_mma_sync": t_m, "us_tcgen05": t_t,
                       "tflops_tcgen05": flops / t_t / 1e6, "max_rel_diff_dw": diff})
    net = sur.Network(device=dev)
    xin = torch.randn(D, H, W, 4, device=dev).to(torch.bfloat16)
    mask = torch.ones(D, H, W, dtype=torch.uint8, device=dev)
    target = torch.randn(D, H, W, 3, device=dev)
    steps = {}
    for eng in ("mma", "tc"):
        net.backward_engine = eng

        def step():
            net.forward(xin, mask)
            net.loss_and_backward(target, mask)

        step()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            step()
        b.record()
        b.synchronize()
        steps["us_" + ("mma_sync" if eng == "mma" else "tcgen05")] = a.elapsed_time(b) / reps * 1e3
    return {"box": [D, H, W], "weight_gradient": layers,
            "train_step": dict(steps, what="forward + masked MSE + backward, eager launches, CUDA events"),
            "what": "weight gradients graph-replayed (device time); dW compared between the two kernels"}


def run_surrogate(dev, n_scenes: int):
    """The learned grid surrogate (the committed trained weights) against the plain method on held-out
    pinch scenes (seeds 20000 + i, 200,000 particles, 64^3 grid, two capsule fingers; none of them among the
    training seeds 10000-11999). Per scene, from the state after two plain env steps: four env steps by
    each form from the same state; errors compare positions after the first env step; times are the mean
    of four back-to-back env steps (median over scenes), graphs captured beforehand. The surrogate runs
    with the per-step gate (a step whose windows fail the mass or momentum check is redone by plain
    substeps) and without a gate."""
    from paper_2302_04659_gb300 import surrogate as sur

    if not os.path.exists(sur.WEIGHTS):
        return {"unavailable": "trained weights not present"}
    t0 = time.perf_counter()
    net = sur.Network.load(sur.WEIGHTS, device=dev)
    seeds = range(20000, 20000 + n_scenes)
    gated = sur.summarize(sur.evaluate(net, seeds, device=dev, gate=True))
    ungated = sur.summarize(sur.evaluate(net, seeds, device=dev, gate=False))
    # the same windows without the network (zero correction), on a quarter of the scenes: what the
    # network adds, and whether the gate catches a window that is not corrected
    few = seeds[: max(1, len(seeds) // 4)]
    none_ungated = sur.summarize(sur.evaluate(None, few, device=dev, gate=False, steps=1))
    none_gated = sur.summarize(sur.evaluate(None, few, device=dev, gate=True, steps=1))
    meta = net.meta
    return {
        "workload": "pinch scenes, held out",
        "seeds": [seeds[0], seeds[-1]],
        "particles": 200_000,
        "window_substeps": sur.K,
        "gate": {"threshold": sur.THRESHOLD, "v_ref": "scene RMS node speed" if sur.V_REF == 0.0 else sur.V_REF,
                 "what": "mass and momentum residuals"},
        "training": {k: meta.get(k) for k in ("rollouts", "seeds", "windows", "epochs")},
        "gated": gated,
        "ungated": ungated,
        "env_steps_per_s_plain": 1e3 / gated["ms_per_env_step_plain"],
        "env_steps_per_s_surrogate_gated": 1e3 / gated["ms_per_env_step_surrogate"],
        "env_steps_per_s_surrogate_ungated": 1e3 / ungated["ms_per_env_step_surrogate"],
        "speedup_gated": gated["ms_per_env_step_plain"] / gated["ms_per_env_step_surrogate"],
        "speedup_ungated": ungated["ms_per_env_step_plain"] / ungated["ms_per_env_step_surrogate"],
        "no_network": {"scenes": none_ungated["scenes"], "rel_x_mean": none_ungated["rel_x_mean"],
                       "rel_to_displacement_mean": none_ungated["rel_to_displacement_mean"],
                       "fallback_rate_gated": none_gated["fallback_rate"],
                       "what": "the same windows with a zero correction, ungated; and the gate's verdict on them"},
        "network_over_no_network_displacement_error": (ungated["rel_to_displacement_mean"]
                                                       / max(none_ungated["rel_to_displacement_mean"], 1e-30)),
        "wall_s": time.perf_counter() - t0,
    }


def oracle_setup(sc, sample=None):
    import oracle
    m = sc.material
    idx = np.arange(sc.N) if sample is None else np.linspace(0, sc.N - 1, sample).astype(np.int64)
    p_vol = m.p_vol * sc.N / len(idx)
    P = oracle.Params(n=sc.n, dt=sc.dt, gravity=tuple(sc.gravity), bound=sc.bound, kind=m.kind, E=m.E, nu=m.nu,
                      yield_stress=m.yield_stress, rho=m.rho, p_vol=p_vol)
    s = oracle.State.from_arrays(sc.x[:, idx], sc.v[:, idx], sc.C[:, idx], sc.F[:, idx])
    return P, s


def oracle_colliders(sc, step):
    import oracle
    from paper_2302_04659_gb300 import scenes
    pose, lin, ang, com = scenes.finger_state(sc, step * SUBSTEPS * sc.dt)
    return [oracle.Collider(sh.type, tuple(map(float, sh.half)), float(sh.friction), tuple(map(float, pose[i, :3])),
                            tuple(map(float, pose[i, 3:])), tuple(map(float, lin[i])), tuple(map(float, ang[i])),
                            tuple(map(float, com[i]))) for i, sh in enumerate(sc.shapes)]


def _oracle_replica(job):
    """One replica of the oracle timing (run in a spawned process): `warmup` untimed then `substeps` timed
    substeps of the pinch scene (seed, particles, optional sample) from its initial state, colliders at env
    step 0. Returns the timed seconds."""
    seed, N, sample, warmup, substeps = job
    sys.path.insert(0, ROOT)
    import oracle
    sc = pinch_inputs(seed, N)
    P, s = oracle_setup(sc, sample)
    cols = oracle_colliders(sc, 0)
    oracle.rollout(P, s, warmup, cols, 0.0)
    t0 = time.perf_counter()
    oracle.rollout(P, s, substeps, cols, 0.0)
    return time.perf_counter() - t0


def oracle_on_all_cores(seed, N, sample, warmup, substeps):
    """The oracle as it stands (single-threaded FP64 C) as independent replicas, one per host core, each
    on its own copy of the workload: aggregate particle-substeps/s of the whole host. Processes are
    spawned (never forked after CUDA is initialised). Returns (value, cores, seconds of the slowest)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(cores) as pool:
        secs = pool.map(_oracle_replica, [(seed, N, sample, warmup, substeps)] * cores)
    n = N if sample is None else sample
    return cores * n * substeps / max(secs), cores, max(secs)


def cpu_baseline(sc):
    """The FP64 oracle on one environment step (25 substeps) of the full scene: single-threaded, and as one
    replica per host core running at the same time (the host's aggregate throughput)."""
    import oracle
    oracle.build()
    P, s = oracle_setup(sc)
    cols = oracle_colliders(sc, 0)
    t0 = time.perf_counter()
    oracle.rollout(P, s, SUBSTEPS, cols, 0.0)
    dt = time.perf_counter() - t0
    single = sc.N * SUBSTEPS / dt
    value, cores, secs = oracle_on_all_cores(1000, sc.N, None, 1, SUBSTEPS)
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"one env step ({SUBSTEPS} substeps) of all {sc.N} particles, FP64, one oracle replica per "
                       f"host core ({cores}) at once"),
            "seconds": secs, "single_thread_value": single, "single_thread_seconds": dt,
            "cpu": cpu_model(), "host_cores": os.cpu_count()}


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def run_reference(args):
    """The oracle as it stands, one replica per host core, each on a bounded particle sample of the same
    scene: warm-up then timed substeps (one substep per step)."""
    rank, world, _ = env_rank()
    if rank != 0:
        return None
    import oracle
    oracle.build()
    sc = pinch_inputs(1000, args.particles)
    total = args.steps + args.warmup
    budget = 90.0  # seconds of oracle work per core for the whole run
    per_unit = 1.6e-6  # seconds per particle-substep of the oracle (about, one core)
    sample = int(min(sc.N, max(2000, budget / max(total, 1) / per_unit)))
    value, cores, secs = oracle_on_all_cores(1000, sc.N, sample, args.warmup, args.steps)
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": secs / args.steps * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (seeded ellipsoid of plasticine, scripted capsule fingers)",
        "config": {"workload": WORKLOAD, "particles_per_gpu": sc.N, "grid": f"{sc.n}^3",
                   "substeps_per_step": 1, "parallelism": f"host CPU, {cores} oracle replicas (one per core)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": (f"{sample} of the {sc.N} particles (mass-preserving) per replica, one substep "
                                    f"per step, {cores} replicas at once"),
                         "cpu": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--particles", type=int, default=200_000, help="particles of the pinch scene")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched and serving workloads")
    ap.add_argument("--batched-steps", type=int, default=10, help="timed env steps of the batched workloads")
    ap.add_argument("--surrogate-scenes", type=int, default=256,
                    help="held-out scenes of the surrogate evaluation (0 skips it)")
    ap.add_argument("--only", choices=["batched", "serving", "surrogate", "contact", "render", "conv", "train"], default=None,
                    help="run one batched workload alone and print its section (profiling runs)")
    ap.add_argument("--envs", type=int, default=0, help="with --only: number of envs (default: the workload's)")
    ap.add_argument("--no-tune", action="store_true", help="with --only: keep the default launch shape")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.only:
        import torch
        from paper_2302_04659_gb300 import build as b
        b.build()
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        if args.only == "surrogate":
            out = run_surrogate(dev, args.surrogate_scenes)
        elif args.only == "contact":
            out = run_contact(dev, args.batched_steps * 4)
        elif args.only == "render":
            out = run_render(dev, args.batched_steps * 5)
        elif args.only == "conv":
            out = run_conv_scan(dev)
        elif args.only == "train":
            out = run_train_timing(dev)
        else:
            out = run_batched(dev, "batch256" if args.only == "batched" else "serve1024", args.batched_steps,
                              3, per_scene=False, tune=not args.no_tune, nenv=args.envs)
        print(json.dumps(out), flush=True)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
