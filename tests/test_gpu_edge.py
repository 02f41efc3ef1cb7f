"""GPU edge cases through the C-ABI: empty and ragged inputs, contention, far moves, bad inputs,
checkpoint/resume, device-side I/O and the wrench/status bookkeeping."""
import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import TOL_V, TOL_X, make_sim, oracle_params, oracle_state, rel, rel_C
from paper_2302_04659_gb300 import _native as mpm
from paper_2302_04659_gb300 import scenes
from test_gpu_parity import assert_state_close, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2302_04659_gb300 import build
    build.build()
    yield


def random_scene(N, seed, n=32, lo=0.3, hi=0.7, v_std=0.5, C_std=5.0, gravity=(0.0, -9.8, 0.0), bound=3):
    x = (lo + (hi - lo) * scenes.uniform(seed, 3 * N).reshape(3, N)).astype(np.float32)
    v, C, F = scenes.random_state(N, seed + 1, v_std=v_std, C_std=C_std)
    mat = scenes.Material(scenes.PLASTICINE, p_vol=(0.25 ** 3) / 8192)
    return scenes.Scene(n=n, dt=2e-4, material=mat, x=x, v=v, C=C, F=F, gravity=gravity, bound=bound)


def one_step_parity(sc, nsub=1):
    out, flags, _ = run_gpu(sc, nsub)
    ref = oracle_state(sc)
    oracle.rollout(oracle_params(sc), ref, nsub)
    assert_state_close(out, ref, dx=1.0 / sc.n)
    return flags


def test_empty_scene():
    sc = scenes.cube_scene("floor")
    sim = make_sim(sc)
    sim.set_particles(np.zeros((3, 0), np.float32))
    sim.substep(3)
    assert sim.N == 0
    st = sim.read_state(on_device=False)
    assert st["x"].shape == (3, 0)
    sim.close()


@pytest.mark.parametrize("N", [1, 2, 31, 33, 129, 4097])
def test_ragged_counts(N):
    flags = one_step_parity(random_scene(N, 100 + N))
    assert not (flags & mpm.MPM_FLAG_INTERNAL)


def test_many_particles_in_one_cell():
    """2,000 particles inside one cell: every atomic of the shared tile hits the same 27 nodes."""
    N = 2000
    n = 32
    dx = 1.0 / n
    sc = random_scene(N, 7, n=n, lo=0.5 + 0.1 * dx, hi=0.5 + 0.9 * dx)
    one_step_parity(sc)


def test_bins_spanning_several_chunks():
    """A dense blob whose bins hold several chunks each, and a sparse tail of lone particles."""
    N = 20000
    sc = random_scene(N, 11, n=32, lo=0.45, hi=0.55)
    one_step_parity(sc)


def test_far_move_served_by_slow_path():
    """Particles crossing more than a cell per substep still transfer exactly (global-atomic path)."""
    N = 3000
    sc = random_scene(N, 13, n=32, lo=0.4, hi=0.6, v_std=0.1, C_std=0.5, gravity=(0.0, 0.0, 0.0), bound=0)
    sc.v[0] += 300.0  # 300 m/s * 2e-4 s = 0.06 = 1.9 cells
    flags = one_step_parity(sc, nsub=2)
    assert flags & mpm.MPM_FLAG_FAR_MOVE


def test_out_of_domain_and_nonfinite_inputs_are_flagged():
    sc = random_scene(256, 17)
    sc.x[0, 3] = 1.5
    sc.x[1, 5] = -0.2
    sim = make_sim(sc)
    sim.set_particles(sc.x, sc.v, sc.C, sc.F)
    assert sim.status() & mpm.MPM_FLAG_CLAMPED
    st = sim.read_state(on_device=False)
    dx = 1.0 / sc.n
    assert st["x"][0, 3] == np.float32(1 - 2 * dx) and st["x"][1, 5] == np.float32(2 * dx)
    sc.x[2, 7] = np.nan
    sim.set_particles(sc.x, sc.v, sc.C, sc.F)
    sim.substep(2)
    f = sim.status(clear=True)
    assert f & mpm.MPM_FLAG_NONFINITE
    assert sim.status() == 0
    st = sim.read_state(on_device=False)
    assert np.all(st["x"] >= 2 * dx - 1e-7) or np.isnan(st["x"]).any() is False
    sim.close()


def test_checkpoint_resume_matches_uninterrupted():
    sc = scenes.cube_scene("floor")
    a, _, _ = run_gpu(sc, 20)
    sim = make_sim(sc)
    sim.set_particles(sc.x, sc.v, sc.C, sc.F)
    sim.substep(10)
    mid = sim.read_state(on_device=False)
    sim.close()
    sim2 = make_sim(sc)
    sim2.set_particles(mid["x"], mid["v"], mid["C"], mid["F"])
    sim2.substep(10)
    b = sim2.read_state(on_device=False)
    sim2.close()
    for k in ("x", "v", "F"):
        assert rel(b[k], a[k]) <= 1e-5, k
    assert rel_C(b["C"], a["C"], a["v"], 1.0 / sc.n) <= 1e-5


def test_device_io_matches_host_io():
    sc = scenes.cube_scene("rand")
    sim = make_sim(sc)
    dev = {k: torch.from_numpy(getattr(sc, k)).cuda() for k in ("x", "v", "C", "F")}
    sim.set_particles(dev["x"], dev["v"], dev["C"], dev["F"])
    sim.substep(2)
    d = sim.read_state(on_device=True)
    h = sim.read_state(on_device=False)
    for k in ("x", "v", "C", "F"):
        assert np.array_equal(d[k].cpu().numpy(), h[k]), k
    ref = oracle_state(sc)
    oracle.rollout(oracle_params(sc), ref, 2)
    assert rel(h["x"], ref.x) <= TOL_X and rel(h["v"], ref.v) <= TOL_V
    sim.close()


def test_async_host_reads_match_blocking_reads():
    """Reads into page-locked host memory, enqueued without waiting, hold what the blocking reads return
    once the stream has reached them -- also when the next substeps are already queued behind them;
    pageable destinations are refused."""
    sc = scenes.pinch_scene(seed=1003, N=20000)
    pose, lin, ang, com = scenes.finger_state(sc, 0.1)
    sim = make_sim(sc)
    sim.set_particles(sc.x, sc.v, sc.C, sc.F)
    sim.set_shapes(sc.shapes)
    sim.set_colliders(pose, lin, ang, com)
    sim.substep(7)
    h = sim.read_state(on_device=False)
    w, n = sim.read_wrench()
    st = torch.cuda.current_stream().cuda_stream
    x_p = torch.empty((3, sc.N), dtype=torch.float32).pin_memory()
    F_p = torch.empty((9, sc.N), dtype=torch.float32).pin_memory()
    w_p = torch.empty((len(sc.shapes), 6), dtype=torch.float64).pin_memory()
    n_p = torch.zeros(1, dtype=torch.int32).pin_memory()
    mpm.mpm_read_state(sim.handle, x_p.data_ptr(), 0, 0, F_p.data_ptr(), 2, st)
    mpm.mpm_read_wrench_async(sim.handle, w_p.data_ptr(), n_p.data_ptr(), st)
    sim.substep(3)  # queued behind the reads: it reuses the staging buffer the reads copy from
    torch.cuda.synchronize()
    assert np.array_equal(x_p.numpy(), h["x"]) and np.array_equal(F_p.numpy(), h["F"])
    assert np.array_equal(w_p.numpy(), w) and int(n_p[0]) == n == 7
    pageable = np.empty((3, sc.N), np.float32)
    with pytest.raises(mpm.MpmError):
        mpm.mpm_read_state(sim.handle, pageable.ctypes.data, 0, 0, 0, 2, st)
    with pytest.raises(mpm.MpmError):
        mpm.mpm_read_wrench_async(sim.handle, np.empty((2, 6)).ctypes.data, 0, st)
    with pytest.raises(mpm.MpmError):
        mpm.mpm_read_state(sim.handle, x_p.data_ptr(), 0, 0, 0, 3, st)
    sim.close()


def test_wrench_bookkeeping_and_timing():
    sc = scenes.pinch_scene(seed=1002, N=20000)
    pose, lin, ang, com = scenes.finger_state(sc, 0.2)
    sim = make_sim(sc)
    sim.set_particles(sc.x, sc.v, sc.C, sc.F)
    sim.set_shapes(sc.shapes)
    sim.set_colliders(pose, lin, ang, com)
    sim.set_timing(True)
    sim.substep(5)
    w1, n1 = sim.read_wrench()
    assert n1 == 5 and np.abs(w1).max() > 0
    sim.set_colliders(pose, lin, ang, com)
    w0, n0 = sim.read_wrench()
    assert n0 == 0 and np.all(w0 == 0)
    sim.substep(1)
    t = sim.read_timing(reset=True)
    assert t["g2p2g"][1] == 6 and t["grid_update"][1] == 6 and t["g2p2g"][0] > 0
    assert sim.launches > 0
    sim.close()


def test_graph_replay_matches_direct_launches():
    """Substeps replayed from captured CUDA graphs (odd and even counts, so both buffer parities are
    captured and replayed) agree with directly issued launches."""
    sc = scenes.pinch_scene(seed=1003, N=30000)
    pose, lin, ang, com = scenes.finger_state(sc, 0.2)
    outs = []
    for graphs in (True, False):
        sim = make_sim(sc)
        sim.set_graphs(graphs)
        sim.set_particles(sc.x, sc.v, sc.C, sc.F)
        sim.set_shapes(sc.shapes)
        sim.set_colliders(pose, lin, ang, com)
        for n in (5, 5, 4, 5, 4):
            sim.substep(n)
        outs.append((sim.read_state(on_device=False), sim.read_wrench()))
        assert not (sim.status() & mpm.MPM_FLAG_INTERNAL)
        sim.close()
    (a, (wa, na)), (b, (wb, nb)) = outs
    assert na == nb == 23
    for k in ("x", "v", "F"):
        assert rel(a[k], b[k]) <= 1e-5, k
    assert rel_C(a["C"], b["C"], b["v"], 1.0 / sc.n) <= 1e-5
    assert rel(wa, wb) <= 1e-4


def test_capacity_and_argument_errors():
    sc = scenes.cube_scene("floor")
    sim = make_sim(sc, max_particles=100)
    with pytest.raises(mpm.MpmError) as e:
        sim.set_particles(sc.x, sc.v, sc.C, sc.F)
    assert e.value.status == mpm.MPM_ERR_CAPACITY
    with pytest.raises(mpm.MpmError):
        mpm.mpm_substep(sim.handle, -1, 0)
    sim.close()
