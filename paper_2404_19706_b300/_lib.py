"""ctypes view of the C ABI in include/rtg.h (librtg.so, built in-tree for sm_103a).

Loading fails loudly: there is no CPU fallback for any entry point.
"""

from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, Structure, c_char_p, c_float, c_int32, c_int64, c_size_t, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librtg.so")

RTG_OK = 0
RTG_ERR_ARG = -1
RTG_ERR_CUDA = -2
RTG_ERR_WORKSPACE = -3
RTG_ERR_TIMEOUT = -4
RTG_ERR_UNSUPPORTED = -5
RTG_ERR_STATE = -6
STATUS_NAMES = {0: "RTG_OK", -1: "RTG_ERR_ARG", -2: "RTG_ERR_CUDA", -3: "RTG_ERR_WORKSPACE",
                -4: "RTG_ERR_TIMEOUT", -5: "RTG_ERR_UNSUPPORTED", -6: "RTG_ERR_STATE"}
RTG_MAX_FRAMES = 32
RTG_TILE = 16


class rtg_camera(Structure):
    _fields_ = [("fx", c_float), ("fy", c_float), ("cx", c_float), ("cy", c_float),
                ("width", c_int32), ("height", c_int32), ("R", c_float * 9), ("t", c_float * 3)]


class rtg_render_params(Structure):
    _fields_ = [(k, c_float) for k in ("near_z", "alpha_min", "f_max", "t_eps", "delta_alpha", "cos_max_angle",
                                       "lowpass", "guard_band", "tile_discard_frac")]


class rtg_gaussians(Structure):
    _fields_ = [("n", c_int64), ("channels", c_int32)] + [
        (k, c_void_p) for k in ("means", "scales", "quats", "opacity", "colors", "unstable",
                                "u_means", "u_scales", "u_quats", "u_opacity", "u_colors",
                                "rank_map", "unstable_ids")] + [("n_unstable", c_int64), ("sh_degree", c_int32)]


class rtg_capacity(Structure):
    _fields_ = [("max_gaussians", c_int64), ("max_frames", c_int32), ("max_width", c_int32),
                ("max_height", c_int32), ("max_channels", c_int32), ("max_pairs", c_int64)]


class rtg_stats(Structure):
    _fields_ = [("pairs", c_int64), ("fragments", c_int64), ("visible", c_int64), ("masked_pixels", c_int64),
                ("n_unstable", c_int64), ("warp_records", c_int64), ("status", c_int32), ("max_tile_pairs", c_int32), ("tile_w", c_int32),
                ("tile_h", c_int32), ("window_stable", c_int64), ("window_pairs", c_int64),
                ("backward_steps", c_int64)]


class rtg_tuning(Structure):
    _fields_ = [("tile_w", c_int32), ("tile_h", c_int32), ("batch", c_int32), ("schedule", c_int32),
                ("persist_ctas_per_sm", c_int32), ("sort_digit_bits", c_int32), ("sort_rank_max", c_int32),
                ("overlap", c_int32)]


class rtg_adam_params(Structure):
    _fields_ = [(k, c_float) for k in ("lr_means", "lr_scales", "lr_quats", "lr_opacity", "lr_colors", "beta1",
                                       "beta2", "eps", "lr_colors_rest")] + [("colors_dc", c_int32)]


class rtg_add_params(Structure):
    _fields_ = [("delta_T", c_float), ("delta_d", c_float), ("delta_c", c_float), ("sample_rate", c_float),
                ("opacity_opaque", c_float), ("opacity_transparent", c_float), ("seed", ctypes.c_uint64)]


class rtg_state_params(Structure):
    _fields_ = [("delta_eta", c_int32), ("delta_e", c_int32), ("delta_t", c_int32), ("delta_c", c_float),
                ("delta_d", c_float)]


class rtg_map_arrays(Structure):
    _fields_ = [(k, c_void_p) for k in ("means", "scales", "quats", "opacity", "colors", "unstable", "eta", "err",
                                        "t0")]


# (name, restype, argtypes) of every entry point declared in include/rtg.h
SIGNATURES = [
    ("rtg_workspace_size", c_int32, [POINTER(rtg_capacity), POINTER(c_size_t)]),
    ("rtg_create", c_int32, [POINTER(c_void_p), POINTER(rtg_capacity)]),
    ("rtg_destroy", c_int32, [c_void_p]),
    ("rtg_unstable_mask", c_int32, [c_void_p, POINTER(rtg_camera), c_int32, POINTER(rtg_gaussians),
                                    POINTER(rtg_render_params), c_void_p, c_void_p]),
    ("rtg_render_forward", c_int32, [c_void_p, POINTER(rtg_camera), c_int32, POINTER(rtg_gaussians), c_void_p,
                                     POINTER(rtg_render_params), c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("rtg_l1_loss", c_int32, [c_void_p, c_int32, c_int32, c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p,
                              c_void_p, c_float, c_float, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("rtg_render_forward_l1", c_int32, [c_void_p, POINTER(rtg_camera), c_int32, POINTER(rtg_gaussians), c_void_p,
                                        POINTER(rtg_render_params), c_void_p, c_void_p, c_float, c_float, c_void_p,
                                        c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("rtg_render_forward_masked", c_int32, [c_void_p, POINTER(rtg_camera), c_int32, POINTER(rtg_gaussians),
                                            POINTER(rtg_render_params), c_void_p, c_void_p, c_void_p, c_float,
                                            c_float, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("rtg_render_backward_l1", c_int32, [c_void_p] + [c_void_p] * 5 + [c_int32, c_void_p]),
    ("rtg_render_backward", c_int32, [c_void_p] + [c_void_p] * 7 + [c_int32, c_void_p]),
    ("rtg_set_tuning", c_int32, [c_void_p, POINTER(rtg_tuning)]),
    ("rtg_window_begin", c_int32, [c_void_p, POINTER(rtg_camera), c_int32, POINTER(rtg_gaussians),
                                   POINTER(rtg_render_params), c_void_p]),
    ("rtg_window_end", c_int32, [c_void_p]),
    ("rtg_window_is_open", c_int32, [c_void_p]),
    ("rtg_select_top_error", c_int32, [c_void_p, c_int32, c_int32, c_int32, c_int32, c_void_p, c_void_p,
                                       ctypes.c_double, c_void_p, c_void_p]),
    ("rtg_add_candidates", c_int32, [c_void_p, POINTER(rtg_camera), c_int32, c_int32] + [c_void_p] * 7 +
     [c_int64, POINTER(rtg_add_params), c_int64] + [c_void_p] * 6 + [c_void_p]),
    ("rtg_transparent_reg", c_int32, [c_void_p, c_int64] + [c_void_p] * 7 + [c_float, c_float] + [c_void_p] * 4 +
     [c_void_p]),
    ("rtg_confidence_update", c_int32, [c_int64, c_int32, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("rtg_fuse_window", c_int32, [c_int64, c_int32] + [c_void_p] * 13 + [c_void_p]),
    ("rtg_error_count", c_int32, [c_void_p, c_int32, c_int32, c_int32, c_int32] + [c_void_p] * 6 +
     [c_int64, POINTER(rtg_state_params), c_void_p, c_void_p]),
    ("rtg_update_states", c_int32, [c_int64, c_int32, c_void_p, POINTER(rtg_state_params)] + [c_void_p] * 4 +
     [c_void_p]),
    ("rtg_compact_gaussians", c_int32, [c_void_p, c_int64, c_int32, c_void_p, POINTER(rtg_map_arrays),
                                        POINTER(rtg_map_arrays), c_void_p, c_void_p]),
    ("rtg_narrow_pixels", c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_float, c_float, c_void_p,
                                    c_void_p]),
    ("rtg_get_tuning", c_int32, [c_void_p, POINTER(rtg_tuning)]),
    ("rtg_decode_rgbd", c_int32, [c_int32, c_int32, c_int32, c_void_p, c_void_p, c_float, c_void_p, c_void_p,
                                  c_void_p]),
    ("rtg_render_forward_l1_frame", c_int32, [c_void_p, POINTER(rtg_camera), c_int32, POINTER(rtg_gaussians), c_void_p,
                                              POINTER(rtg_render_params), c_void_p, c_void_p, c_float, c_void_p,
                                              c_void_p, c_float, c_float, c_void_p, c_void_p, c_void_p, c_void_p,
                                              c_void_p, c_void_p]),
    ("rtg_adam_step", c_int32, [c_int64, c_int32] + [c_void_p] * 12 + [c_int32, POINTER(rtg_adam_params),
                                                                       c_void_p]),
    ("rtg_adam_step_counted", c_int32, [c_int64, c_int32] + [c_void_p] * 13 + [POINTER(rtg_adam_params),
                                                                                c_void_p]),
    ("rtg_adam_step_counted_after_gradients", c_int32, [c_int64, c_int32] + [c_void_p] * 13 +
     [POINTER(rtg_adam_params), c_void_p]),
    ("rtg_unstable_index", c_int32, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("rtg_unstable_rank", c_int32, [c_void_p, c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("rtg_unstable_index_static", c_int32, [c_int64, c_void_p, c_void_p, c_void_p, c_void_p]),
    ("rtg_gather_unstable", c_int32, [c_int64, c_int32] + [c_void_p] * 11 + [c_void_p]),
    ("rtg_scatter_unstable", c_int32, [c_int64, c_int32] + [c_void_p] * 11 + [c_void_p]),
    ("rtg_get_stats", c_int32, [c_void_p, POINTER(rtg_stats)]),
    ("rtg_get_status", c_int32, [c_void_p]),
    ("rtg_reset_status", c_int32, [c_void_p]),
    ("rtg_last_error", c_char_p, [c_void_p]),
    ("rtg_profile_enable", c_int32, [c_void_p, c_int32]),
    ("rtg_profile_kinds", c_int32, []),
    ("rtg_profile_kind_name", c_char_p, [c_int32]),
    ("rtg_profile_read", c_int32, [c_void_p, POINTER(c_int64), POINTER(ctypes.c_double), c_int32]),
    ("rtg_alu_probe", c_int32, [c_int32, c_int32, c_void_p, POINTER(c_int64), c_void_p]),
    ("rtg_loss_counts", c_int32, [c_void_p, c_void_p, c_void_p]),
    ("rtg_set_loss_scales", c_int32, [c_void_p, c_void_p, c_float, c_float, c_void_p, c_void_p]),
    ("rtg_debug_binning", c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
]

_LIB = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load librtg.so once and attach the prototypes.  Raises if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(f"librtg.so not found at {path}: build it with __graft_entry__.build() "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib
