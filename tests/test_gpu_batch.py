"""GPU parity of the batched handle: many envs with their own grids, materials, particle counts and
colliders advanced by the same launches.

Each env of a batch is compared with the FP64 oracle run on that env alone (one substep, element-wise,
the tolerances of ``gpu_helpers``), and with a single-scene handle running the same env (several
substeps; atomic ordering differs, so to a tolerance well below the parity bound). Both bin-scan paths
are covered: the fused pass's last CTA (few bins) and the two grid-wide scan kernels (many bins).
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import (TOL_C, TOL_F, TOL_V, TOL_X, make_sim, oracle_colliders, oracle_params, oracle_state,
                         rel, rel_C)
from paper_2302_04659_gb300 import scenes

pytestmark = pytest.mark.gpu

# bins above which the grid-wide scan kernels replace the fused pass's tail scan
TAIL_SCAN_MAX_BINS = 16384


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2302_04659_gb300 import build
    build.build()
    yield


def make_batch(envs, max_colliders=None):
    from paper_2302_04659_gb300.sim import BatchSim
    sc0 = envs[0]
    spec = [(sc.n, sc.material, max(sc.N, 1), max(len(sc.shapes), 0) if max_colliders is None else max_colliders)
            for sc in envs]
    return BatchSim(spec, sc0.dt, gravity=sc0.gravity, bound=sc0.bound)


def run_batch(envs, nsub, t=0.0, with_colliders=True):
    sim = make_batch(envs)
    counts, (x, v, C, F) = scenes.concat_states(envs)
    sim.set_particles(counts, x, v, C, F)
    cols = None
    if with_colliders:
        sim.set_shapes([sc.shapes for sc in envs])
        cols = scenes.concat_tool_states(envs, t)
        sim.set_colliders(*cols)
    sim.substep(nsub)
    out = sim.read_state(on_device=False)
    wr, n = sim.read_wrench() if with_colliders else (None, None)
    flags = sim.status()
    sim.close()
    return out, counts, wr, n, flags


def split(out, counts):
    off = np.concatenate([[0], np.cumsum(counts)])
    return [{k: a[:, off[e]:off[e + 1]] for k, a in out.items()} for e in range(len(counts))]


def ambiguous_mask(sc, amb):
    """Particles whose stencil touches a node the oracle marks as within 1e-6 of a collider branch flip."""
    keep = np.ones(sc.N, bool)
    if amb is not None and amb.any():
        base = np.floor(sc.x.astype(np.float64) * sc.n - 0.5).astype(int)
        bad = np.zeros(sc.N, bool)
        for node in np.argwhere(amb):
            bad |= np.all((node[:, None] >= base) & (node[:, None] <= base + 2), axis=0)
        keep = ~bad
    return keep


def assert_env_matches_oracle(sc, got, t, wr_env):
    P = oracle_params(sc)
    ref = oracle_state(sc)
    pose, lin, ang, com = scenes.finger_state(sc, t) if sc.shapes else (None, None, None, None)
    cols = oracle_colliders(sc, pose, lin, ang, com) if sc.shapes else ()
    # the poses were set at time t; the oracle's collider clock counts from there
    _, wref, amb = oracle.substep(P, ref, cols, 0.0, want_ambiguous=True)
    keep = ambiguous_mask(sc, amb)
    assert (~keep).sum() <= 1e-3 * max(sc.N, 1)
    dx = 1.0 / sc.n
    m = keep
    ex = rel(got["x"][:, m], ref.x[:, m])
    ev = rel(got["v"][:, m], ref.v[:, m])
    ec = rel_C(got["C"][:, m], ref.C[:, m], ref.v[:, m], dx)
    if sc.material.kind == scenes.PLASTICINE:
        ef = rel(got["F"][:, m], ref.F[:, m])
    else:
        J = np.prod(got["F"][[0, 4, 8]].astype(np.float64), axis=0)
        ef = rel(J[m], ref.J[m])
    assert ex <= TOL_X and ev <= TOL_V and ec <= TOL_C and ef <= TOL_F, (ex, ev, ec, ef)
    if sc.shapes:
        # relative where the tool pushes (impulses ~1e-2); a graze of a few nodes is held to the same
        # absolute error as a 1e-3 impulse
        scale = max(np.abs(wref).max(), 1e-3)
        assert np.abs(wr_env[:, :3] - wref[:, :3]).max() <= 1e-4 * scale
        assert np.abs(wr_env[:, 3:] - wref[:, 3:]).max() <= 1e-4 * scale
    return np.abs(wref).max() if sc.shapes else 0.0


def mixed_envs():
    """Uneven envs: plasticine and fluid, grids 16^3 to 48^3, 0 to 9k particles, with and without tools."""
    cube = scenes.cube_scene("rand")
    return [
        scenes.tool_scene(11, scenes.PLASTICINE, 6000, n=32),
        scenes.tool_scene(12, scenes.FLUID, 4000, n=24),
        cube,
        scenes.tool_scene(13, scenes.FLUID, 9000, n=48, extra_capsule=True),
        scenes.tool_scene(14, scenes.PLASTICINE, 0, n=16),
        scenes.tool_scene(15, scenes.PLASTICINE, 1, n=16),
    ]


@pytest.mark.parametrize("t", [0.0, 0.2])
def test_mixed_batch_one_substep_matches_oracle(t):
    envs = mixed_envs()
    out, counts, wr, nsub, flags = run_batch(envs, 1, t=t)
    assert nsub == 1
    assert flags & 0x80000000 == 0
    touched = 0.0
    col = 0
    for sc, got in zip(envs, split(out, counts)):
        k = len(sc.shapes)
        if sc.N:
            touched = max(touched, assert_env_matches_oracle(sc, got, t, wr[col:col + k]))
        col += k
    if t > 0:
        assert touched > 0, "the tools should touch their bodies at t > 0"


def test_many_bins_grid_scan_matches_oracle():
    """Six 64^3 envs (24,576 bins): bins are counted and scanned by the grid-wide kernels."""
    envs = [scenes.tool_scene(100 + e, scenes.PLASTICINE if e % 2 == 0 else scenes.FLUID, 3000 + 1500 * e, n=64)
            for e in range(6)]
    assert sum((sc.n // 4) ** 3 for sc in envs) > TAIL_SCAN_MAX_BINS
    t = 0.15
    out, counts, wr, nsub, flags = run_batch(envs, 1, t=t)
    col = 0
    for sc, got in zip(envs, split(out, counts)):
        assert_env_matches_oracle(sc, got, t, wr[col:col + 1])
        col += 1


@pytest.mark.parametrize("many_bins", [False, True])
def test_batch_matches_single_handles_over_substeps(many_bins):
    """30 substeps: every env of a batch against its own single-scene handle."""
    n = 64 if many_bins else 32
    envs = [scenes.tool_scene(200 + e, scenes.PLASTICINE if e % 2 == 0 else scenes.FLUID, 2000 + 700 * e, n=n)
            for e in range(6)]
    t = 0.1
    out, counts, wr, nsub, _ = run_batch(envs, 30, t=t)
    assert nsub == 30
    col = 0
    for sc, got in zip(envs, split(out, counts)):
        sim = make_sim(sc)
        sim.set_particles(sc.x, sc.v, sc.C, sc.F)
        sim.set_shapes(sc.shapes)
        sim.set_colliders(*scenes.finger_state(sc, t))
        sim.substep(30)
        ref = sim.read_state(on_device=False)
        wref, _ = sim.read_wrench()
        sim.close()
        assert rel(got["x"], ref["x"]) <= 1e-5
        assert rel(got["v"], ref["v"]) <= 1e-3
        if np.abs(wref).max() > 0:
            assert rel(wr[col:col + 1], wref) <= 1e-3
        col += 1


def test_batch_graph_replay_matches_direct_launches():
    envs = mixed_envs()
    res = []
    for graphs in (True, False):
        sim = make_batch(envs)
        sim.set_graphs(graphs)
        counts, (x, v, C, F) = scenes.concat_states(envs)
        sim.set_particles(counts, x, v, C, F)
        sim.set_shapes([sc.shapes for sc in envs])
        sim.set_colliders(*scenes.concat_tool_states(envs, 0.2))
        for _ in range(3):
            sim.substep(5)
        res.append(sim.read_state(on_device=False)["x"])
        sim.close()
    assert rel(res[0], res[1]) <= 1e-5


def test_launch_shapes_agree():
    """The autotuner's knobs change only the schedule: every launch shape gives the same substep."""
    from paper_2302_04659_gb300 import _native
    envs = [scenes.tool_scene(300 + e, scenes.PLASTICINE if e % 2 == 0 else scenes.FLUID, 5000, n=32)
            for e in range(4)]
    counts, (x, v, C, F) = scenes.concat_states(envs)
    outs = []
    for shape in [(0, 0, 0), (32, 1, 1), (96, 3, 4), (256, 4, 8)]:
        sim = make_batch(envs)
        if shape != (0, 0, 0):
            sim.set_launch(*shape)
            assert sim.get_launch() == shape
        sim.set_particles(counts, x, v, C, F)
        sim.set_shapes([sc.shapes for sc in envs])
        sim.set_colliders(*scenes.concat_tool_states(envs, 0.2))
        sim.substep(10)
        outs.append(sim.read_state(on_device=False)["x"])
        for bad in [(16, 0, 0), (100, 0, 0), (288, 0, 0), (0, 99, 0), (0, 0, 99), (0, -1, 0)]:
            with pytest.raises(_native.MpmError):
                sim.set_launch(*bad)
        sim.close()
    for o in outs[1:]:
        assert rel(o, outs[0]) <= 1e-5


def test_batch_capacity_and_argument_errors():
    from paper_2302_04659_gb300 import _native
    envs = mixed_envs()[:3]
    sim = make_batch(envs)
    assert sim.nenv == 3
    counts, (x, v, C, F) = scenes.concat_states(envs)
    with pytest.raises(_native.MpmError) as e:
        sim.set_particles([counts[0] + 1, counts[1], counts[2] - 1], x, v, C, F)
    assert e.value.status == _native.MPM_ERR_CAPACITY
    with pytest.raises(_native.MpmError):
        sim.set_particles([counts[0], -1, counts[2]], x, v, C, F)
    sim.set_particles(counts, x, v, C, F)
    assert sim.N == sum(counts)
    with pytest.raises(_native.MpmError) as e:
        sim.set_shapes([envs[0].shapes * 2, [], []])  # more shapes than env 0's capacity
    assert e.value.status == _native.MPM_ERR_CAPACITY
    sim.set_shapes([sc.shapes for sc in envs])
    pose, lin, ang, com = scenes.concat_tool_states(envs, 0.0)
    sim.k = len(pose) - 1  # a count that differs from the shapes set
    with pytest.raises(_native.MpmError):
        sim.set_colliders(pose[:-1], lin[:-1], ang[:-1], com[:-1])
    sim.close()


def test_many_colliders_pose_table_matches_single_handles():
    """20 envs with a tool each (more colliders than the grid update keeps per CTA): poses come from the
    table filled at upload for 64 substeps, then are evaluated on the fly; 70 substeps against single
    handles, whose few colliders are posed per CTA."""
    envs = [scenes.tool_scene(400 + e, scenes.PLASTICINE if e % 2 == 0 else scenes.FLUID, 600 + 37 * e, n=24)
            for e in range(20)]
    t = 0.12
    out, counts, wr, nsub, _ = run_batch(envs, 70, t=t)
    assert nsub == 70
    hit = 0
    for e, (sc, got) in enumerate(zip(envs, split(out, counts))):
        sim = make_sim(sc)
        sim.set_particles(sc.x, sc.v, sc.C, sc.F)
        sim.set_shapes(sc.shapes)
        sim.set_colliders(*scenes.finger_state(sc, t))
        sim.substep(70)
        ref = sim.read_state(on_device=False)
        wref, _ = sim.read_wrench()
        sim.close()
        assert rel(got["x"], ref["x"]) <= 1e-5
        scale = max(np.abs(wref).max(), 1e-3)
        assert np.abs(wr[e:e + 1] - wref).max() <= 1e-3 * scale
        hit += np.abs(wref).max() > 1e-3
    assert hit >= 5, "several tools should push their bodies"


def test_chunk_size_change_mid_run():
    """A chunk-size change between substeps recuts the chunk list: the fused pass of a smaller CTA never
    meets a chunk cut for the larger one (every particle still moves, no internal-error flag), and the
    state equals a run that used the final size throughout."""
    from paper_2302_04659_gb300.sim import Sim
    sc = scenes.pinch_scene(seed=1008, N=100_000)
    cols = scenes.finger_state(sc, 0.1)
    outs = []
    for sizes in ((256, 64), (64, 64), (128, 256)):
        sim = Sim(sc.n, sc.dt, sc.material, sc.N, gravity=sc.gravity, bound=sc.bound, max_colliders=2)
        sim.set_shapes(sc.shapes)
        sim.set_launch(sizes[0])
        sim.set_particles(sc.x, sc.v, sc.C, sc.F)
        sim.set_colliders(*cols)
        sim.substep(3)
        sim.set_launch(sizes[1])
        sim.substep(3)
        assert sim.status() & 0x80000000 == 0
        outs.append(sim.read_state(on_device=False)["x"])
        sim.close()
    for o in outs[1:]:
        assert rel(o, outs[0]) <= 1e-5


def test_chunk_size_change_with_grid_scan():
    """The recut after a chunk-size change on the grid-wide scan path (more bins than the fused pass's
    last CTA scans): same state as a batch that used the final size throughout, no internal-error flag."""
    envs = [scenes.tool_scene(120 + e, scenes.PLASTICINE if e % 2 == 0 else scenes.FLUID, 20_000, n=64)
            for e in range(6)]
    assert sum((sc.n // 4) ** 3 for sc in envs) > TAIL_SCAN_MAX_BINS
    counts, (x, v, C, F) = scenes.concat_states(envs)
    cols = scenes.concat_tool_states(envs, 0.1)
    outs = []
    for sizes in ((256, 64), (64, 64)):
        sim = make_batch(envs)
        sim.set_launch(sizes[0])
        sim.set_particles(counts, x, v, C, F)
        sim.set_shapes([sc.shapes for sc in envs])
        sim.set_colliders(*cols)
        sim.substep(3)
        sim.set_launch(sizes[1])
        sim.substep(3)
        assert sim.status() & 0x80000000 == 0
        outs.append(sim.read_state(on_device=False)["x"])
        sim.close()
    assert rel(outs[0], outs[1]) <= 1e-5
