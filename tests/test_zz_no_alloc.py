"""The allocation-free particle-to-grid entry point (mpm_p2g_static) against the FP64 oracle.

mpm_p2g_static is for callers that cannot call cudaMalloc (a plugin inside a host simulator that owns all
device memory, a real-time loop that must not synchronize the device): it keeps its sort scratch in a
device array owned by the library. Its grid must match the oracle's particle-to-grid transfer on the same
FP32 particles, at the documented limits (65,536 particles, 64^3 nodes) where every part of the scratch is
in use, for both materials and with the optional arrays left out, and it must stay right on consecutive
calls, which reuse that array. This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import fluid_scene, oracle_params, oracle_state, rel
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


def _static(sc, arrays, calls=1):
    """Run mpm_p2g_static `calls` times in a row on the same inputs; returns each call's grid (FP64)."""
    cfg, mat = _cfg_mat(sc)
    dev = {k: (torch.from_numpy(np.ascontiguousarray(a)).cuda() if a is not None else None)
           for k, a in arrays.items()}
    ptr = {k: (t.data_ptr() if t is not None else 0) for k, t in dev.items()}
    stream = torch.cuda.current_stream().cuda_stream
    grids = []
    for _ in range(calls):
        out = torch.full((sc.n, sc.n, sc.n, 4), 7.0, dtype=torch.float32, device="cuda")  # must be overwritten
        mpm.mpm_p2g_static(cfg, mat, sc.N, ptr["x"], ptr["v"], ptr["C"], ptr["F"], out.data_ptr(), stream)
        grids.append(out.cpu().numpy().astype(np.float64))
    return grids


def _assert_grid_matches(g, ref):
    # the tolerances of the regular path's transfer against the FP64 oracle (FP32 global atomics here)
    assert abs(g[..., 0].sum() - ref[..., 0].sum()) <= 1e-6 * ref[..., 0].sum()
    assert rel(g[..., 0], ref[..., 0]) < 1e-6
    assert rel(g[..., 1:], ref[..., 1:]) < 1e-5
    assert np.all(g[ref[..., 0] == 0.0] == 0.0)  # nodes no particle reaches stay zero


def test_static_p2g_matches_oracle_at_its_limits_on_consecutive_calls():
    """65,536 particles of plasticine with random v, C, F on a 64^3 grid: the largest inputs the scratch
    takes. Two calls in a row must both equal the oracle's transfer."""
    sc = scenes.pinch_scene(seed=1003, N=65536, n=64)
    v, C, F = scenes.random_state(sc.N, seed=31, v_std=0.3, C_std=3.0, F_std=0.05)
    sc.v, sc.C, sc.F = v, C, F
    ref = oracle.p2g(oracle_params(sc), oracle_state(sc))
    for g in _static(sc, {"x": sc.x, "v": sc.v, "C": sc.C, "F": sc.F}, calls=2):
        _assert_grid_matches(g, ref)


def test_static_p2g_fluid_matches_oracle():
    """The fluid material (J = det F, tau = lambda J (J - 1) I)."""
    sc = fluid_scene()
    ref = oracle.p2g(oracle_params(sc), oracle_state(sc))
    (g,) = _static(sc, {"x": sc.x, "v": sc.v, "C": sc.C, "F": sc.F})
    _assert_grid_matches(g, ref)


@pytest.mark.parametrize("kind", [scenes.PLASTICINE, scenes.FLUID])
def test_static_p2g_optional_arrays_default(kind):
    """v, C and F left out (NULL) mean v = 0, C = 0, F = I (J = 1)."""
    sc = scenes.cube_scene("floor") if kind == scenes.PLASTICINE else fluid_scene()
    N = sc.N
    zeros3, zeros9 = np.zeros((3, N), np.float32), np.zeros((9, N), np.float32)
    eye = np.tile(np.eye(3, dtype=np.float32).reshape(9, 1), (1, N))
    ref = oracle.p2g(oracle_params(sc), oracle_state(sc, v=zeros3, C=zeros9, F=eye))
    (g,) = _static(sc, {"x": sc.x, "v": None, "C": None, "F": None})
    _assert_grid_matches(g, ref)


def test_static_p2g_rejects_sizes_beyond_its_scratch():
    sc = scenes.cube_scene("floor")
    cfg, mat = _cfg_mat(sc)
    out = torch.zeros((sc.n, sc.n, sc.n, 4), dtype=torch.float32, device="cuda")
    x = torch.zeros((3, 65537), dtype=torch.float32, device="cuda")
    with pytest.raises(mpm.MpmError) as e:
        mpm.mpm_p2g_static(cfg, mat, 65537, x.data_ptr(), 0, 0, 0, out.data_ptr(), 0)
    assert e.value.status == mpm.MPM_ERR_CAPACITY
    cfg.n = 68  # a grid the regular path takes, beyond the scratch's 64^3
    with pytest.raises(mpm.MpmError) as e:
        mpm.mpm_p2g_static(cfg, mat, 16, x.data_ptr(), 0, 0, 0, out.data_ptr(), 0)
    assert e.value.status == mpm.MPM_ERR_CAPACITY


def test_static_p2g_checks_only_the_fields_it_uses():
    """max_particles, max_colliders and bound are not used by this entry, so they are not checked."""
    sc = scenes.cube_scene("floor")
    cfg, mat = _cfg_mat(sc)
    cfg.max_particles, cfg.max_colliders, cfg.bound = 0, -1, 1000
    cm = (cfg, mat)
    dev = torch.from_numpy(np.ascontiguousarray(sc.x)).cuda()
    out = torch.zeros((sc.n, sc.n, sc.n, 4), dtype=torch.float32, device="cuda")
    mpm.mpm_p2g_static(*cm, sc.N, dev.data_ptr(), 0, 0, 0, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    eye = np.tile(np.eye(3, dtype=np.float32).reshape(9, 1), (1, sc.N))
    ref = oracle.p2g(oracle_params(sc), oracle_state(sc, v=np.zeros((3, sc.N), np.float32),
                                                       C=np.zeros((9, sc.N), np.float32), F=eye))
    _assert_grid_matches(out.cpu().numpy().astype(np.float64), ref)
    cfg.dt = 0.0
    with pytest.raises(mpm.MpmError) as e:
        mpm.mpm_p2g_static(*cm, sc.N, dev.data_ptr(), 0, 0, 0, out.data_ptr(), 0)
    assert e.value.status == mpm.MPM_ERR_INVALID_ARG
