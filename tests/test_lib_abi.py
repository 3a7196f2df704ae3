"""CPU-side checks of the C ABI: libsph builds for sm_103a, loads, and exports
every function include/sph.h declares (no GPU calls)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1606_02738_gb300 import build as sphbuild
from paper_1606_02738_gb300 import sph


@pytest.fixture(scope="module")
def libpath():
    return sphbuild.build()


def test_header_declares_the_boundary():
    names = sph.header_functions()
    for f in ("sph_create", "sph_workspace_size", "sph_set_workspace", "sph_init",
              "sph_density", "sph_force", "sph_step", "sph_get", "sph_get_pair_order",
              "sph_autotune", "sph_fp32_peak", "sph_stats", "sph_last_error", "sph_destroy",
              "sph_default_params"):
        assert f in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in sph.header_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (sph_\w+)", out))
    assert set(sph.header_functions()) <= exported


def test_library_is_built_for_sm_103a(libpath):
    log = open(os.path.join(sphbuild.BUILD, "ptxas.log")).read()
    assert "sm_103a" in log
    assert "spill stores" in log


def test_params_struct_matches_header_defaults(libpath):
    p = sph.sph_default_params()
    assert p.gamma == pytest.approx(5.0 / 3.0)
    assert p.n_ngb == 48.0 and p.h_tol == 1e-6 and p.max_iter == 30 and p.n_split == 64
    assert p.mode == sph.SPH_MODE_BATCHED and p.precision == sph.SPH_PREC_FP32
    assert p.pair_sort == 1 and p.profile == 0 and p.reuse_grid == 1
    assert p.tile == 0 and p.cell_factor == 2.0 and p.reuse_lists == 1 and p.work_queue == 1
    assert ctypes.sizeof(sph.sph_params) == 3 * 8 + 8 * 4 + 8 + 2 * 4
    assert [f for f, _ in sph.sph_params._fields_][-7:] == ["profile", "pair_sort", "reuse_grid",
                                                           "tile", "cell_factor", "reuse_lists",
                                                           "work_queue"]
    assert ctypes.sizeof(sph.sph_stats_t) == (10 * 8 + 4 * 4 + 2 * 8 + 2 * 4 + 5 * 8 + 7 * 8 +
                                              2 * 4 + 8 * 4 + 4 * 8 + 5 * 8)


@pytest.mark.parametrize("field,value", [("pair_sort", 2), ("reuse_lists", 3), ("work_queue", 4),
                                         ("work_queue", -1)])
def test_param_switches_validated(libpath, field, value):
    L = sph.lib()
    bad = sph.sph_default_params()
    setattr(bad, field, value)
    ctx = ctypes.c_void_p()
    assert L.sph_create(ctypes.byref(ctx), ctypes.byref(bad), None) == sph.SPH_EINVAL


def test_invalid_arguments_rejected_without_gpu(libpath):
    L = sph.lib()
    assert L.sph_create(None, None, None) == sph.SPH_EINVAL
    bad = sph.sph_default_params()
    bad.n_split = 1
    ctx = ctypes.c_void_p()
    assert L.sph_create(ctypes.byref(ctx), ctypes.byref(bad), None) == sph.SPH_EINVAL
    assert L.sph_density(None) == sph.SPH_EINVAL
    assert L.sph_stats(None, None) == sph.SPH_EINVAL
    assert L.sph_fp32_peak(0, None, None) == sph.SPH_EINVAL
    L.sph_destroy(None)
