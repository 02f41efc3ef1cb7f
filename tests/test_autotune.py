"""Host logic of the launch-shape autotuner: the coordinate descent finds the best shape of a synthetic
cost surface, respects the fused kernel's occupancy limit, and caches per workload signature. The GPU
test tunes a real batch and checks the chosen shape is applied and valid."""
import pytest

from paper_2302_04659_gb300 import autotune


class FakeSim:
    """Launch shapes as the library checks them: chunks above 128 run 256-thread CTAs, which fit at
    most 4 per SM (max_fused caps both CTA sizes further)."""

    def __init__(self, max_fused=7):
        self.max_fused = max_fused
        self.shape = (128, min(7, max_fused), 2)
        self.N = 123456
        self.ns = [64]
        self.kinds = [0, 1]
        self.nenv = 4
        self.device = None
        self.restored = 0

    def set_launch(self, c, f, g):
        c = c or self.shape[0]
        limit = min(4 if c > 128 else 7, self.max_fused)
        if f and f > limit:
            raise autotune.mpm.MpmError("mpm_set_launch", 1)
        self.shape = (c, f or self.shape[1], g or self.shape[2])

    def get_launch(self):
        return self.shape


def cost(shape):
    c, f, g = shape
    return 1.0 + 0.01 * abs(c - 192) + 0.05 * abs(f - 3) + 0.02 * abs(g - 4)


@pytest.fixture
def fake_env(monkeypatch, tmp_path):
    monkeypatch.setattr(autotune, "CACHE_PATH", str(tmp_path / "autotune.json"))
    monkeypatch.setattr(autotune.torch.cuda, "get_device_name", lambda dev=None: "FakeGPU")
    calls = []

    def fake_time(sim, shape, substeps, reps, prepare=None, stream=None):
        calls.append(shape)
        sim.set_launch(*shape)
        return cost(shape)

    monkeypatch.setattr(autotune, "time_shape", fake_time)
    return calls


def test_descent_finds_optimum_and_caches(fake_env):
    sim = FakeSim()
    shape, ms, trials = autotune.tune(sim, restore=lambda: setattr(sim, "restored", sim.restored + 1))
    assert shape == (192, 3, 4)
    assert sim.get_launch() == (192, 3, 4)
    assert ms == pytest.approx(cost((192, 3, 4)))
    assert sim.restored == 1
    assert len(trials) == len(set(fake_env)) < 4 * 3 * 3  # fewer trials than the full grid
    # second call: served from the cache, no trials, shape applied
    sim2 = FakeSim()
    n_calls = len(fake_env)
    shape2, ms2, trials2 = autotune.tune(sim2)
    assert shape2 == (192, 3, 4) and trials2 == {} and len(fake_env) == n_calls
    assert sim2.get_launch() == (192, 3, 4)


def test_signature_separates_workloads(fake_env):
    a, b = FakeSim(), FakeSim()
    b.N = 4 * a.N
    c = FakeSim()
    c.kinds = [0]
    assert autotune.signature(a) != autotune.signature(b)
    assert autotune.signature(a) != autotune.signature(c)
    d = FakeSim()
    d.N = a.N + 1000  # same size bucket
    assert autotune.signature(a) == autotune.signature(d)


def test_occupancy_limit_respected(fake_env):
    sim = FakeSim(max_fused=2)
    shape, _, _ = autotune.tune(sim, use_cache=False)
    assert shape[1] <= 2
    assert all(s[1] <= 2 for s in fake_env)


@pytest.mark.gpu
def test_tune_real_batch():
    from paper_2302_04659_gb300 import build, scenes
    from paper_2302_04659_gb300.sim import BatchSim
    build.build()
    envs = [scenes.tool_scene(500 + e, scenes.PLASTICINE if e % 2 == 0 else scenes.FLUID, 4000, n=32)
            for e in range(8)]
    sim = BatchSim([(sc.n, sc.material, sc.N, len(sc.shapes)) for sc in envs], envs[0].dt)
    counts, (x, v, C, F) = scenes.concat_states(envs)
    sim.set_particles(counts, x, v, C, F)
    sim.set_shapes([sc.shapes for sc in envs])
    cols = scenes.concat_tool_states(envs, 0.1)
    shape, ms, trials = autotune.tune(sim, substeps=2, reps=1, prepare=lambda: sim.set_colliders(*cols),
                                      use_cache=False)
    assert sim.get_launch() == shape
    assert shape[0] in autotune.CHUNKS and shape[2] in autotune.GRID_CTAS
    assert 1 <= shape[1] <= 7
    assert ms > 0 and len(trials) >= 3
    sim.close()
