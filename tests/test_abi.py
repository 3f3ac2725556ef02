"""The C-ABI library loads and exports every entry point include/rtg.h declares; host-only
argument checks work without a GPU."""

import ctypes
import os
import re

import pytest

from paper_2404_19706_b300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "rtg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rtg_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = _lib.load()
    names = declared_symbols()
    assert len(names) >= 16
    for name in names:
        assert hasattr(lib, name), f"{name} declared in rtg.h but not exported"
    bound = {s[0] for s in _lib.SIGNATURES}
    assert set(names) == bound, set(names) ^ bound


def test_workspace_size_host_only():
    lib = _lib.load()
    cap = _lib.rtg_capacity(1_000_000, 1, 640, 480, 3, 4 << 20)
    n = ctypes.c_size_t()
    assert lib.rtg_workspace_size(ctypes.byref(cap), ctypes.byref(n)) == _lib.RTG_OK
    assert n.value > 1_000_000 * 48  # at least the compositing records
    bad = _lib.rtg_capacity(10, 0, 640, 480, 3, 100)  # zero frames
    assert lib.rtg_workspace_size(ctypes.byref(bad), ctypes.byref(n)) == _lib.RTG_ERR_ARG
    bad = _lib.rtg_capacity(10, 1, 640, 480, 5, 100)  # unsupported channel count
    assert lib.rtg_workspace_size(ctypes.byref(bad), ctypes.byref(n)) == _lib.RTG_ERR_ARG
    assert lib.rtg_workspace_size(None, ctypes.byref(n)) == _lib.RTG_ERR_ARG


def test_host_side_argument_errors_without_gpu():
    lib = _lib.load()
    hp = _lib.rtg_adam_params(1e-3, 4e-3, 1e-3, 0.0, 5e-4, 0.9, 0.999, 1e-15)
    args = [None] * 12
    assert lib.rtg_adam_step(-1, 3, *args, 1, ctypes.byref(hp), None) == _lib.RTG_ERR_ARG
    assert lib.rtg_adam_step(10, 3, *args, 0, ctypes.byref(hp), None) == _lib.RTG_ERR_ARG  # step counts from 1
    assert lib.rtg_adam_step(0, 3, *args, 1, ctypes.byref(hp), None) == _lib.RTG_OK  # nothing to do
    assert lib.rtg_get_status(None) == _lib.RTG_ERR_ARG
    assert lib.rtg_last_error(None)
    assert lib.rtg_destroy(None) == _lib.RTG_OK
    out = ctypes.c_void_p(123)
    assert lib.rtg_create(ctypes.byref(out), None) == _lib.RTG_ERR_ARG and not out.value
    assert lib.rtg_render_forward(None, None, 1, None, None, None, None, None, None, None, None) == _lib.RTG_ERR_ARG
    assert lib.rtg_gather_unstable(-1, 3, *([None] * 11), None) == _lib.RTG_ERR_ARG


def test_struct_layouts_match_header():
    # rtg_camera: 4 floats, 2 ints, 9 + 3 floats
    assert ctypes.sizeof(_lib.rtg_camera) == 4 * 4 + 2 * 4 + 12 * 4
    assert ctypes.sizeof(_lib.rtg_render_params) == 9 * 4
    assert ctypes.sizeof(_lib.rtg_gaussians) == 8 + 8 + 13 * 8 + 8
    assert ctypes.sizeof(_lib.rtg_capacity) == 8 + 4 * 4 + 8
    assert ctypes.sizeof(_lib.rtg_stats) == 5 * 8 + 2 * 4


@pytest.mark.gpu
def test_create_destroy_roundtrip():
    import paper_2404_19706_b300 as rtg
    ctx = rtg.Context(max_gaussians=1000)
    assert ctx.workspace_bytes() > 0
    assert rtg.get_status(ctx) == 0
    ctx.close()
