"""The C-ABI library loads and exports every entry point include/rtg.h declares; host-only
argument checks work without a GPU."""

import ctypes
import os
import re
import shutil
import subprocess
import tempfile

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
    ops = ctypes.c_int64(-7)
    assert lib.rtg_alu_probe(2, 10, 1, ctypes.byref(ops), None) == _lib.RTG_ERR_ARG  # unknown kind
    assert lib.rtg_alu_probe(0, 0, 1, ctypes.byref(ops), None) == _lib.RTG_ERR_ARG   # no iterations
    assert lib.rtg_alu_probe(1, 10, None, ctypes.byref(ops), None) == _lib.RTG_ERR_ARG
    assert ops.value == -7
    # the Adam step that starts under the kernel in front, and the frame-decoding forward:
    # argument errors found on the host, before any launch
    adam_args = [None] * 13
    assert lib.rtg_adam_step_counted_after_gradients(-1, 3, *adam_args, ctypes.byref(hp), None) == _lib.RTG_ERR_ARG
    assert lib.rtg_adam_step_counted_after_gradients(10, 3, *adam_args, None, None) == _lib.RTG_ERR_ARG
    assert lib.rtg_adam_step_counted_after_gradients(10, 0, *adam_args, ctypes.byref(hp), None) == _lib.RTG_ERR_ARG
    assert lib.rtg_adam_step_counted_after_gradients(0, 3, *adam_args[:12], ctypes.c_void_p(8),
                                                     ctypes.byref(hp), None) == _lib.RTG_OK  # nothing to do
    assert lib.rtg_render_forward_l1_frame(None, None, 1, None, None, None, None, None, 1.0, None, None, 1.0, 1.0,
                                           None, None, None, None, None, None) == _lib.RTG_ERR_ARG


def test_struct_layouts_match_header():
    # rtg_camera: 4 floats, 2 ints, 9 + 3 floats
    assert ctypes.sizeof(_lib.rtg_camera) == 4 * 4 + 2 * 4 + 12 * 4
    assert ctypes.sizeof(_lib.rtg_render_params) == 9 * 4
    assert ctypes.sizeof(_lib.rtg_gaussians) == 8 + 8 + 13 * 8 + 8 + 8  # + sh_degree, padded
    assert ctypes.sizeof(_lib.rtg_capacity) == 8 + 4 * 4 + 8
    assert ctypes.sizeof(_lib.rtg_stats) == 6 * 8 + 4 * 4 + 3 * 8  # + window counters, backward steps
    assert ctypes.sizeof(_lib.rtg_tuning) == 8 * 4
    assert ctypes.sizeof(_lib.rtg_add_params) == 6 * 4 + 8
    assert ctypes.sizeof(_lib.rtg_state_params) == 5 * 4
    assert ctypes.sizeof(_lib.rtg_map_arrays) == 9 * 8


@pytest.mark.gpu
def test_create_destroy_roundtrip():
    import paper_2404_19706_b300 as rtg
    ctx = rtg.Context(max_gaussians=1000)
    assert ctx.workspace_bytes() > 0
    assert rtg.get_status(ctx) == 0
    ctx.close()


def test_struct_layouts_match_compiled_header():
    """sizeof / offsetof of every ABI struct as gcc lays out include/rtg.h equal the ctypes
    binding's (a field added to one side only fails here)."""
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    structs = [(n, getattr(_lib, n)) for n in ("rtg_camera", "rtg_render_params", "rtg_gaussians", "rtg_capacity",
                                                 "rtg_stats", "rtg_tuning", "rtg_adam_params", "rtg_add_params",
                                                 "rtg_state_params", "rtg_map_arrays")]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rtg.h"', "int main(void) {"]
    for name, cls in structs:
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{name}.{fname} %zu\\n", offsetof({name}, {fname}));')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines) + "\n")
        subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split("\n")
    got = dict(line.split() for line in out if line.strip())
    for name, cls in structs:
        assert int(got[name]) == ctypes.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert int(got[f"{name}.{fname}"]) == getattr(cls, fname).offset, f"{name}.{fname}"


def test_global_optimisation_entry_points_reject_bad_arguments_without_gpu():
    lib = _lib.load()
    assert lib.rtg_select_top_error(None, 1, 3, 8, 8, None, None, 0.4, None, None) == _lib.RTG_ERR_ARG
    assert lib.rtg_narrow_pixels(None, None, None, None, 1.0, 1.0, None, None) == _lib.RTG_ERR_ARG
    sp = _lib.rtg_state_params(100, 10, 200, 0.1, 0.1)
    assert lib.rtg_confidence_update(-1, 3, None, None, None, None) == _lib.RTG_ERR_ARG
    assert lib.rtg_confidence_update(0, 3, None, None, None, None) == _lib.RTG_OK
    assert lib.rtg_fuse_window(5, 3, *([None] * 13), None) == _lib.RTG_ERR_ARG
    assert lib.rtg_update_states(5, 0, None, ctypes.byref(sp), None, None, None, None, None) == _lib.RTG_ERR_ARG
    assert lib.rtg_error_count(None, 1, 3, 8, 8, *([None] * 6), 0, ctypes.byref(sp), None, None) == _lib.RTG_ERR_ARG
    assert lib.rtg_compact_gaussians(None, 0, 3, None, None, None, None, None) == _lib.RTG_ERR_ARG
    # frame decode: sizes, scale and pointers are checked before any device work
    assert lib.rtg_decode_rgbd(0, 4, 4, 1, 1, 5000.0, 1, 1, None) == _lib.RTG_ERR_ARG
    assert lib.rtg_decode_rgbd(1, 4, 4, 1, 1, 0.0, 1, 1, None) == _lib.RTG_ERR_ARG
    assert lib.rtg_decode_rgbd(1, 4, 4, 1, 1, float("inf"), 1, 1, None) == _lib.RTG_ERR_ARG
    assert lib.rtg_decode_rgbd(1, 4, 4, None, 1, 5000.0, 1, 1, None) == _lib.RTG_ERR_ARG
    p = _lib.rtg_add_params(0.5, 0.1, 0.1, 0.05, 0.99, 0.1, 0)
    assert lib.rtg_add_candidates(None, None, 1, 3, *([None] * 7), 0, ctypes.byref(p), 0,
                                  *([None] * 6), None) == _lib.RTG_ERR_ARG


def test_colour_row_width_comes_from_the_shape_even_without_rows():
    # the binding passes C (values per Gaussian) to Adam and the compaction; with no unstable
    # Gaussian the arrays have no rows, and C must still be the row width, not 0
    import torch
    from paper_2404_19706_b300 import api
    assert api._row_width(torch.empty(0, 3)) == 3
    assert api._row_width(torch.empty(0, 8)) == 8
    assert api._row_width(torch.empty(7, 16, 3)) == 48
    assert api._row_width(torch.empty(0, 16, 3)) == 48
    assert api._row_width(torch.empty(5)) == 1
