"""CPU checks of the boundary: the library builds, loads and exports every symbol ``include/mpm.h``
declares, and host-side argument validation rejects bad input before touching the GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2302_04659_gb300 import build
    build.build()
    from paper_2302_04659_gb300 import _native as mpm
    return mpm


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(mpm_[a-z0-9_]+)\s*\(", src, re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["mpm_create", "mpm_set_colliders", "mpm_substep", "mpm_read_state", "mpm_set_particles",
                     "mpm_read_wrench", "mpm_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    L = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_names_match_header(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n) and n not in ("mpm_status_string",)]
    assert not missing, missing


def _cfg(lib, **kw):
    c = dict(n=64, dt=2e-4, gravity=(0.0, -9.8, 0.0), bound=3, max_particles=1000, max_colliders=2)
    c.update(kw)
    return lib.mpm_config(c["n"], c["dt"], (ctypes.c_float * 3)(*c["gravity"]), c["bound"], c["max_particles"],
                          c["max_colliders"])


def _mat(lib, **kw):
    m = dict(kind=0, rho=1e3, E=5e3, nu=0.3, yield_stress=50.0, bulk_modulus=1e4, p_vol=1e-6)
    m.update(kw)
    return lib.mpm_material(m["kind"], m["rho"], m["E"], m["nu"], m["yield_stress"], m["bulk_modulus"], m["p_vol"])


def test_workspace_size_grows_with_capacity(lib):
    a = lib.mpm_workspace_size(_cfg(lib, max_particles=1000), _mat(lib))
    b = lib.mpm_workspace_size(_cfg(lib, max_particles=100000), _mat(lib))
    c = lib.mpm_workspace_size(_cfg(lib, n=32), _mat(lib))
    assert b > a > c > 0
    # two state buffers of 25 floats per particle dominate at large capacity
    assert b - a >= 2 * 25 * 4 * 99000


@pytest.mark.parametrize("bad", [dict(n=30), dict(n=4), dict(n=512), dict(dt=0.0), dict(dt=float("nan")),
                                 dict(bound=40), dict(max_particles=0), dict(max_colliders=33)])
def test_invalid_config_rejected_on_host(lib, bad):
    with pytest.raises(lib.MpmError) as e:
        lib.mpm_workspace_size(_cfg(lib, **bad), _mat(lib))
    assert e.value.status == lib.MPM_ERR_INVALID_ARG


@pytest.mark.parametrize("bad", [dict(kind=2), dict(rho=0.0), dict(p_vol=-1.0), dict(nu=0.5), dict(E=0.0)])
def test_invalid_material_rejected_on_host(lib, bad):
    with pytest.raises(lib.MpmError) as e:
        lib.mpm_workspace_size(_cfg(lib), _mat(lib, **bad))
    assert e.value.status == lib.MPM_ERR_INVALID_ARG


def test_missing_or_small_workspace_rejected_on_host(lib):
    cfg, mat = _cfg(lib), _mat(lib)
    need = lib.mpm_workspace_size(cfg, mat)
    with pytest.raises(lib.MpmError) as e:
        lib.mpm_create(cfg, mat, 0, need)
    assert e.value.status == lib.MPM_ERR_WORKSPACE
    with pytest.raises(lib.MpmError) as e:
        lib.mpm_create(cfg, mat, 4096 * 1024 + 16, need)  # misaligned address, rejected before any use
    assert e.value.status == lib.MPM_ERR_WORKSPACE
    with pytest.raises(lib.MpmError) as e:
        lib.mpm_create(cfg, mat, 4096 * 1024, need - 256)
    assert e.value.status == lib.MPM_ERR_WORKSPACE


def test_status_strings(lib):
    for s in range(5):
        assert lib.status_string(s)
    assert lib.status_string(99) == "unknown status"


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2302_04659_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, fn)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", src, re.M), fn
                assert "mpm_oracle" not in src, fn


def test_network_arguments_rejected_on_host(lib):
    """Bad sizes and channel counts return MPM_ERR_INVALID_ARG before any device work."""
    cases = [
        lambda: lib.mpm_conv3d_forward(lib.MPM_NET_BF16, 0, 4, 4, 32, 32, 1, 1, 0, 0, 0, 1),
        lambda: lib.mpm_conv3d_forward(lib.MPM_NET_BF16, 4, 4, 4, 65, 32, 1, 1, 0, 0, 0, 1),
        lambda: lib.mpm_conv3d_forward(7, 4, 4, 4, 32, 32, 1, 1, 0, 0, 0, 1),
        lambda: lib.mpm_conv3d_backward_data(lib.MPM_NET_F32, 4, -1, 4, 32, 32, 1, 1, 0, 1),
        lambda: lib.mpm_conv3d_backward_weight(lib.MPM_NET_BF16, 4, 4, 4, 40, 32, 1, 1, 1, 1),
        lambda: lib.mpm_mse_loss(lib.MPM_NET_BF16, 0, 3, 1, 1, 1, 1, 1, 1),
        lambda: lib.mpm_adam_step(10, 1, 1, 1, 1, 0, 1e-3),
        # the tensor-core weight gradient: input channels 4, 16 or 32; output 1..32; 16-byte alignment
        lambda: lib.mpm_conv3d_backward_weight_tc(4, 4, 4, 8, 32, 16, 16, 16, 16),
        lambda: lib.mpm_conv3d_backward_weight_tc(4, 4, 4, 32, 0, 16, 16, 16, 16),
        lambda: lib.mpm_conv3d_backward_weight_tc(4, 4, 4, 32, 33, 16, 16, 16, 16),
        lambda: lib.mpm_conv3d_backward_weight_tc(0, 4, 4, 32, 32, 16, 16, 16, 16),
        lambda: lib.mpm_conv3d_backward_weight_tc(4, 4, 4, 32, 32, 8, 16, 16, 16),
        lambda: lib.mpm_conv3d_backward_weight_tc(4, 4, 4, 32, 32, 16, 16, 4, 16),
    ]
    for case in cases:
        with pytest.raises(lib.MpmError) as e:
            case()
        assert e.value.status == lib.MPM_ERR_INVALID_ARG


def test_bin_decode_by_reciprocal_is_exact():
    """The kernels split a local bin index b < nb^3 into block coordinates by multiplying with
    ceil(2^32 / nb) and keeping the high 32 bits, for every block count the library accepts (grids of
    8..256 nodes per axis, nb = n / 4 = 2..64). Checked here against integer division over every bin."""
    for nb in range(2, 65):
        recip = (0xFFFFFFFF // nb) + 1
        assert recip < 2 ** 32
        b = np.arange(nb ** 3, dtype=np.uint64)
        q1 = (b * np.uint64(recip)) >> np.uint64(32)
        q2 = (q1 * np.uint64(recip)) >> np.uint64(32)
        assert np.array_equal(q1, b // nb)
        assert np.array_equal(q2, b // (nb * nb))
