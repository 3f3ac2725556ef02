"""B300-native masked, depth-split differentiable Gaussian rasterizer (RTG-SLAM, arxiv 2404.19706).

The compute path is librtg.so (CUDA for sm_103a) behind the C ABI in include/rtg.h;
this package is its Python binding.  Importing it loads the library and fails loudly
if it has not been built (there is no CPU fallback).
"""

from . import _lib

_lib.load()

from .api import (  # noqa: E402,F401
    AdamSettings,
    AddSettings,
    MapArrays,
    StateSettings,
    add_candidates,
    compact_gaussians,
    confidence_update,
    error_count,
    fuse_window,
    update_states,
    Context,
    Gaussians,
    RenderSettings,
    Tuning,
    RTGError,
    adam_step,
    adam_step_counted,
    decode_rgbd,
    debug_binning,
    gather_unstable,
    get_stats,
    get_status,
    l1_loss,
    last_error,
    make_camera,
    narrow_pixels,
    profile_enable,
    profile_read,
    alu_probe,
    loss_counts,
    set_loss_scales,
    render_backward,
    render_backward_l1,
    render_forward_l1,
    render_forward_l1_frame,
    render_forward_masked,
    render_forward,
    reset_status,
    scatter_unstable,
    select_top_error,
    transparent_reg,
    unstable_index,
    unstable_rank,
    unstable_mask,
    window_begin,
    window_end,
    window_is_open,
    workspace_size,
)
from .optim import MaskedStep, RasterState, RTGRasterize, rasterize  # noqa: E402,F401
from .keyframes import GlobalStep, KeyframeSet, global_adam  # noqa: E402,F401
from .adding import AddingPass  # noqa: E402,F401
from .state import MapState  # noqa: E402,F401

LIBRARY_PATH = _lib.LIB_PATH
