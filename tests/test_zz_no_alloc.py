"""The allocation-free particle-to-grid entry point (mpm_p2g_static) against the regular path.

mpm_p2g_static is for callers that cannot call cudaMalloc (a plugin inside a host simulator that owns all
device memory, a real-time loop that must not synchronize the device): it keeps its sort scratch in a
device array owned by the library. Its output must match what the regular path returns for the same
particles (mpm_set_particles followed by mpm_read_grid), and it must stay right on consecutive calls,
which reuse that array. This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

from gpu_helpers import rel, make_sim
from paper_2302_04659_gb300 import _native as mpm
from paper_2302_04659_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2302_04659_gb300 import build
    build.build()
    yield


def _cfg_mat(sc):
    m = sc.material
    cfg = mpm.mpm_config(sc.n, sc.dt, (ctypes.c_float * 3)(*sc.gravity), sc.bound, sc.N, 1)
    mat = mpm.mpm_material(m.kind, m.rho, m.E, m.nu, m.yield_stress, m.bulk_modulus, m.p_vol)
    return cfg, mat


def test_static_p2g_matches_regular_path_on_consecutive_calls():
    sc = scenes.cube_scene("rand")
    sim = make_sim(sc)
    sim.set_particles(sc.x, sc.v, sc.C, sc.F)
    ref = sim.read_grid().cpu().numpy().astype(np.float64)
    sim.close()

    cfg, mat = _cfg_mat(sc)
    dev = {k: torch.from_numpy(np.ascontiguousarray(getattr(sc, k))).cuda() for k in ("x", "v", "C", "F")}
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        out = torch.full((sc.n, sc.n, sc.n, 4), 7.0, dtype=torch.float32, device="cuda")  # must be overwritten
        mpm.mpm_p2g_static(cfg, mat, sc.N, dev["x"].data_ptr(), dev["v"].data_ptr(), dev["C"].data_ptr(),
                           dev["F"].data_ptr(), out.data_ptr(), stream)
        g = out.cpu().numpy().astype(np.float64)
        # same tolerances as the regular path's transfer against the FP64 oracle
        assert abs(g[..., 0].sum() - ref[..., 0].sum()) <= 1e-6 * ref[..., 0].sum()
        assert rel(g[..., 0], ref[..., 0]) < 1e-6
        assert rel(g[..., 1:], ref[..., 1:]) < 1e-5


def test_static_p2g_rejects_sizes_beyond_its_scratch():
    sc = scenes.cube_scene("floor")
    cfg, mat = _cfg_mat(sc)
    out = torch.zeros((sc.n, sc.n, sc.n, 4), dtype=torch.float32, device="cuda")
    x = torch.zeros((3, 65537), dtype=torch.float32, device="cuda")
    with pytest.raises(mpm.MpmError) as e:
        mpm.mpm_p2g_static(cfg, mat, 65537, x.data_ptr(), 0, 0, 0, out.data_ptr(), 0)
    assert e.value.status == mpm.MPM_ERR_CAPACITY
