"""The C-ABI library builds for sm_103a, loads, and exports every symbol the
header declares (no compute call is made here)."""
import ctypes
import re

import pytest

from conftest import ROOT, gpu_available


@pytest.fixture(scope="module")
def libso():
    from paper_2407_14783_b300 import build, binding
    build.build()
    return binding.lib()


def _header_functions():
    src = open(f"{ROOT}/include/visfly_b300.h").read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(sim_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_expected_calls():
    names = _header_functions()
    for must in ("sim_create_scene", "sim_step", "sim_render", "sim_step_backward", "sim_create_ctx",
                 "sim_destroy_ctx", "sim_get_status", "sim_last_error"):
        assert must in names


def test_every_header_symbol_is_exported_and_bound(libso):
    from paper_2407_14783_b300 import binding
    for name in _header_functions():
        assert hasattr(libso, name), name
        assert name in binding.SIGNATURES, name


def test_version_and_error_path_without_device(libso):
    assert b"sm_103a" in libso.sim_version()
    if gpu_available():
        pytest.skip("device present")
    from paper_2407_14783_b300 import binding, workloads
    h = ctypes.c_void_p()
    p = binding.make_params(workloads.params())
    rc = libso.sim_create_ctx(ctypes.byref(h), 0, ctypes.byref(p), 0)
    assert rc != 0 and not h.value
    assert len(libso.sim_last_error(None)) > 0


def test_render_config_list(libso):
    from paper_2407_14783_b300.sim import Sim
    cfgs = Sim.render_configs()
    assert len(cfgs) >= 10
    assert all(c["tile_w"] * c["tile_h"] == 32 * c["rays_per_lane"] for c in cfgs)
