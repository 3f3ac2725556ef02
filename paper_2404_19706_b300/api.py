"""Python binding of the C ABI (include/rtg.h): argument marshalling only.

Every function here forwards torch CUDA tensors as raw device pointers to the entry
point of the same name in librtg.so and raises ``RTGError`` on a non-OK status.  All
computation happens in the CUDA kernels behind the ABI; PyTorch provides device
memory and streams.
"""

from __future__ import annotations

import ctypes
import dataclasses
import math
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib
from ._lib import (rtg_adam_params, rtg_camera, rtg_capacity, rtg_gaussians, rtg_render_params, rtg_stats)


class RTGError(RuntimeError):
    def __init__(self, status: int, where: str, message: str = ""):
        self.status = status
        super().__init__(f"{where}: {_lib.STATUS_NAMES.get(status, status)} {message}".strip())


def _check(status: int, where: str, ctx=None):
    if status != _lib.RTG_OK:
        lib = _lib.load()
        msg = lib.rtg_last_error(ctx).decode() if ctx is not None else ""
        raise RTGError(status, where, msg)


def _ptr(t: Optional[torch.Tensor], dtype=None, name: str = "tensor") -> Optional[int]:
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must live on a CUDA device (there is no CPU path)")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr() if t.numel() > 0 else None


def _stream(stream) -> Optional[int]:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if isinstance(stream, torch.cuda.Stream) else int(stream)


# ----------------------------------------------------------------------------- value types

@dataclasses.dataclass(frozen=True)
class RenderSettings:
    """Rendering constants (rtg_render_params): Section 3.1 thresholds, the Supplement B
    tile rule and the 3DGS conventions for the values the paper leaves open."""
    near_z: float = 0.2
    alpha_min: float = 1.0 / 255.0
    f_max: float = 0.99
    t_eps: float = 1e-4
    delta_alpha: float = math.exp(-0.5)
    cos_max_angle: float = 0.5
    lowpass: float = 0.3
    guard_band: float = 1.3
    tile_discard_frac: float = 0.5

    def to_c(self) -> rtg_render_params:
        return rtg_render_params(*(float(getattr(self, f.name)) for f in dataclasses.fields(self)))


@dataclasses.dataclass(frozen=True)
class AdamSettings:
    """Supplement C learning rates (Replica/ScanNet++ set); scale is stepped in log space."""
    lr_means: float = 1e-3
    lr_scales: float = 4e-3
    lr_quats: float = 1e-3
    lr_opacity: float = 0.0
    lr_colors: float = 5e-4
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-15
    # SH colour: the first colors_dc values of a colour row (the degree-0 coefficients) use
    # lr_colors, the others lr_colors_rest (0.05 lr_SH0); 0 = every value lr_colors
    lr_colors_rest: float = 2.5e-5
    colors_dc: int = 0

    def to_c(self) -> rtg_adam_params:
        names = ("lr_means", "lr_scales", "lr_quats", "lr_opacity", "lr_colors", "beta1", "beta2", "eps",
                 "lr_colors_rest")
        return rtg_adam_params(*(float(getattr(self, k)) for k in names), int(self.colors_dc))


@dataclasses.dataclass(frozen=True)
class AddSettings:
    """Thresholds of the Gaussian-adding masks (Section 3.2, Eq. 6), the sampled fraction and
    the opacities of new opaque / transparent Gaussians (rtg_add_params, without the seed)."""
    delta_T: float = 0.5
    delta_d: float = 0.1
    delta_c: float = 0.1
    sample_rate: float = 0.05
    opacity_opaque: float = 0.99
    opacity_transparent: float = 0.1

    def to_c(self, seed: int) -> "_lib.rtg_add_params":
        return _lib.rtg_add_params(self.delta_T, self.delta_d, self.delta_c, self.sample_rate, self.opacity_opaque,
                                   self.opacity_transparent, int(seed) & ((1 << 64) - 1))


def make_camera(cam) -> rtg_camera:
    """Any object with fx, fy, cx, cy, width, height, R [3,3] (camera-to-world), t [3]."""
    c = rtg_camera()
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    R = np.asarray(cam.R, dtype=np.float32).reshape(9)
    t = np.asarray(cam.t, dtype=np.float32).reshape(3)
    for k in range(9):
        c.R[k] = float(R[k])
    for k in range(3):
        c.t[k] = float(t[k])
    return c


def _cams(cams) -> tuple:
    if not isinstance(cams, (list, tuple)):
        cams = [cams]
    arr = (rtg_camera * len(cams))(*[make_camera(c) for c in cams])
    return arr, len(cams)


@dataclasses.dataclass
class Gaussians:
    """Structure-of-arrays Gaussian parameters on the GPU (rtg_gaussians)."""
    means: torch.Tensor      # [N,3] f32
    scales: torch.Tensor     # [N,3] f32
    quats: torch.Tensor      # [N,4] f32 (w,x,y,z)
    opacity: torch.Tensor    # [N] f32
    colors: torch.Tensor     # [N,C] f32
    unstable: torch.Tensor   # [N] u8
    u_means: Optional[torch.Tensor] = None  # optional compact overrides [Nu, .]
    u_scales: Optional[torch.Tensor] = None
    u_quats: Optional[torch.Tensor] = None
    u_opacity: Optional[torch.Tensor] = None
    u_colors: Optional[torch.Tensor] = None
    rank_map: Optional[torch.Tensor] = None      # optional precomputed unstable index (int32 [N])
    unstable_ids: Optional[torch.Tensor] = None  # int32 [Nu], ascending
    n_unstable: int = 0
    sh_degree: int = 0  # 1..3: colors holds SH coefficients [N, (d+1)^2, 3]

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @property
    def channels(self) -> int:
        """Colour channels of a render (3 with SH colour)."""
        return 3 if self.sh_degree > 0 else int(self.colors.shape[1])

    @property
    def color_width(self) -> int:
        """Colour values per Gaussian: the channels, or 3 (d+1)^2 SH coefficients."""
        return int(np.prod(self.colors.shape[1:]))

    @staticmethod
    def from_scene(scene, device="cuda") -> "Gaussians":
        def t(a, dt=torch.float32):
            return torch.as_tensor(np.ascontiguousarray(a)).to(device=device, dtype=dt).contiguous()
        colors = np.asarray(scene.colors)
        deg = int(round(np.sqrt(colors.shape[1]))) - 1 if colors.ndim == 3 else 0
        return Gaussians(t(scene.means), t(scene.scales), t(scene.quats), t(scene.opacity), t(colors),
                         t(scene.unstable, torch.uint8), sh_degree=deg)

    def to_c(self) -> rtg_gaussians:
        g = rtg_gaussians()
        g.n, g.channels, g.sh_degree = self.n, self.channels, int(self.sh_degree)
        for name in ("means", "scales", "quats", "opacity", "colors"):
            setattr(g, name, _ptr(getattr(self, name), torch.float32, name))
        g.unstable = _ptr(self.unstable, torch.uint8, "unstable")
        for name in ("u_means", "u_scales", "u_quats", "u_opacity", "u_colors"):
            v = getattr(self, name)
            setattr(g, name, _ptr(v, torch.float32, name) if v is not None else None)
        if self.rank_map is not None:
            g.rank_map = _ptr(self.rank_map, torch.int32, "rank_map")
            g.unstable_ids = _ptr(self.unstable_ids, torch.int32, "unstable_ids") if self.n_unstable else None
            g.n_unstable = int(self.n_unstable)
        if self.u_means is not None and any(getattr(self, k).numel() == 0 for k in ("u_means",)):
            # an empty compact set is the same as no override
            for name in ("u_means", "u_scales", "u_quats", "u_opacity", "u_colors"):
                setattr(g, name, None)
        return g


# ----------------------------------------------------------------------------- context

class Context:
    """Owns an rtg_ctx (the preallocated workspace) on the current CUDA device."""

    def __init__(self, max_gaussians: int, max_frames: int = 1, max_width: int = 640, max_height: int = 480,
                 max_channels: int = 3, max_pairs: Optional[int] = None):
        lib = _lib.load()
        if max_pairs is None:
            max_pairs = max(1 << 20, 32 * max_gaussians * max_frames)
        self.cap = rtg_capacity(int(max_gaussians), int(max_frames), int(max_width), int(max_height),
                                int(max_channels), int(min(max_pairs, 0xFFFFFFFF)))
        h = ctypes.c_void_p()
        st = lib.rtg_create(ctypes.byref(h), ctypes.byref(self.cap))
        if st != _lib.RTG_OK:
            raise RTGError(st, "rtg_create", f"capacity {self.cap.max_gaussians} Gaussians, "
                                             f"{self.cap.max_pairs} pairs")
        self.handle = h

    def workspace_bytes(self) -> int:
        n = ctypes.c_size_t()
        _check(_lib.load().rtg_workspace_size(ctypes.byref(self.cap), ctypes.byref(n)), "rtg_workspace_size")
        return int(n.value)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            _lib.load().rtg_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def ptr(self):
        return self.handle

    def set_tuning(self, t: "Tuning"):
        c = t.to_c()
        _check(_lib.load().rtg_set_tuning(self.ptr, ctypes.byref(c)), "rtg_set_tuning", self.ptr)

    def get_tuning(self) -> "Tuning":
        c = _lib.rtg_tuning()
        _check(_lib.load().rtg_get_tuning(self.ptr, ctypes.byref(c)), "rtg_get_tuning", self.ptr)
        return Tuning(c.tile_w, c.tile_h, c.batch, c.schedule, c.persist_ctas_per_sm, c.sort_digit_bits,
                      c.sort_rank_max, c.overlap)


@dataclasses.dataclass(frozen=True)
class Tuning:
    """Launch configuration of the render path (rtg_tuning); never changes a rendered value."""
    tile_w: int = 16
    tile_h: int = 16
    batch: int = 32
    schedule: int = 0          # 0: CTA per tile; 1: persistent warps over the cost-ordered queue
    persist_ctas_per_sm: int = 4
    sort_digit_bits: int = 8
    sort_rank_max: int = 0
    overlap: int = 1           # programmatic dependent launch between the kernels of a call

    def to_c(self):
        return _lib.rtg_tuning(self.tile_w, self.tile_h, self.batch, self.schedule, self.persist_ctas_per_sm,
                               self.sort_digit_bits, self.sort_rank_max, self.overlap)

    def as_dict(self) -> dict:
        return {"tile": f"{self.tile_w}x{self.tile_h}", "batch": self.batch, "schedule": self.schedule,
                "persist_ctas_per_sm": self.persist_ctas_per_sm, "sort_digit_bits": self.sort_digit_bits,
                "sort_rank_max": self.sort_rank_max, "overlap": self.overlap}


def workspace_size(max_gaussians, max_frames=1, max_width=640, max_height=480, max_channels=3, max_pairs=1 << 20):
    cap = rtg_capacity(int(max_gaussians), int(max_frames), int(max_width), int(max_height), int(max_channels),
                       int(max_pairs))
    n = ctypes.c_size_t()
    _check(_lib.load().rtg_workspace_size(ctypes.byref(cap), ctypes.byref(n)), "rtg_workspace_size")
    return int(n.value)


# ----------------------------------------------------------------------------- entry points

def window_begin(ctx: Context, cams, g: Gaussians, settings: RenderSettings, stream=None):
    """Open an optimisation window: project the stable Gaussians into ``cams`` once; later
    forwards with the same cameras, settings, arrays and unstable index reuse them."""
    if g.rank_map is None:
        raise ValueError("window_begin needs a Gaussians with the precomputed unstable index (rank_map)")
    arr, F = _cams(cams)
    gc = g.to_c()
    prm = settings.to_c()
    st = _lib.load().rtg_window_begin(ctx.ptr, arr, F, ctypes.byref(gc), ctypes.byref(prm), _stream(stream))
    _check(st, "rtg_window_begin", ctx.ptr)


def window_end(ctx: Context):
    _check(_lib.load().rtg_window_end(ctx.ptr), "rtg_window_end", ctx.ptr)


def window_is_open(ctx: Context) -> bool:
    return bool(_lib.load().rtg_window_is_open(ctx.ptr))


def unstable_mask(ctx: Context, cams, g: Gaussians, settings: RenderSettings, mask: torch.Tensor, stream=None):
    arr, F = _cams(cams)
    gc = g.to_c()
    prm = settings.to_c()
    st = _lib.load().rtg_unstable_mask(ctx.ptr, arr, F, ctypes.byref(gc), ctypes.byref(prm),
                                       _ptr(mask, torch.uint8, "mask"), _stream(stream))
    _check(st, "rtg_unstable_mask", ctx.ptr)


def render_forward(ctx: Context, cams, g: Gaussians, mask: Optional[torch.Tensor], settings: RenderSettings,
                   color: torch.Tensor, depth: torch.Tensor, alpha: torch.Tensor,
                   index_map: Optional[torch.Tensor] = None, stream=None):
    arr, F = _cams(cams)
    gc = g.to_c()
    prm = settings.to_c()
    st = _lib.load().rtg_render_forward(ctx.ptr, arr, F, ctypes.byref(gc), _ptr(mask, torch.uint8, "mask"),
                                        ctypes.byref(prm), _ptr(color, torch.float32, "color"),
                                        _ptr(depth, torch.float32, "depth"), _ptr(alpha, torch.float32, "alpha"),
                                        _ptr(index_map, torch.int32, "index_map"), _stream(stream))
    _check(st, "rtg_render_forward", ctx.ptr)


def render_forward_l1(ctx: Context, cams, g: Gaussians, mask: Optional[torch.Tensor], settings: RenderSettings,
                      target_color, target_depth, w_color: float, w_depth: float, color, depth, alpha, loss_out,
                      index_map: Optional[torch.Tensor] = None, stream=None):
    arr, F = _cams(cams)
    gc = g.to_c()
    prm = settings.to_c()
    st = _lib.load().rtg_render_forward_l1(
        ctx.ptr, arr, F, ctypes.byref(gc), _ptr(mask, torch.uint8, "mask"), ctypes.byref(prm),
        _ptr(target_color, torch.float32, "target_color"), _ptr(target_depth, torch.float32, "target_depth"),
        float(w_color), float(w_depth), _ptr(color, torch.float32, "color"), _ptr(depth, torch.float32, "depth"),
        _ptr(alpha, torch.float32, "alpha"), _ptr(index_map, torch.int32, "index_map"),
        _ptr(loss_out, torch.float32, "loss_out"), _stream(stream))
    _check(st, "rtg_render_forward_l1", ctx.ptr)


def render_forward_l1_frame(ctx: Context, cams, g: Gaussians, mask: Optional[torch.Tensor], settings: RenderSettings,
                            rgb: torch.Tensor, depth16: torch.Tensor, depth_scale: float, target_color, target_depth,
                            w_color: float, w_depth: float, color, depth, alpha, loss_out,
                            index_map: Optional[torch.Tensor] = None, stream=None):
    """rtg_render_forward_l1_frame: decode the RGB-D sensor frame (rgb uint8 [F,H,W,3], depth16
    uint16 [F,H,W]) into target_color / target_depth, then render_forward_l1 against them."""
    arr, F = _cams(cams)
    gc = g.to_c()
    prm = settings.to_c()
    st = _lib.load().rtg_render_forward_l1_frame(
        ctx.ptr, arr, F, ctypes.byref(gc), _ptr(mask, torch.uint8, "mask"), ctypes.byref(prm),
        _ptr(rgb, torch.uint8, "rgb"), _ptr(depth16, torch.uint16, "depth16"), float(depth_scale),
        _ptr(target_color, torch.float32, "target_color"), _ptr(target_depth, torch.float32, "target_depth"),
        float(w_color), float(w_depth), _ptr(color, torch.float32, "color"), _ptr(depth, torch.float32, "depth"),
        _ptr(alpha, torch.float32, "alpha"), _ptr(index_map, torch.int32, "index_map"),
        _ptr(loss_out, torch.float32, "loss_out"), _stream(stream))
    _check(st, "rtg_render_forward_l1_frame", ctx.ptr)


def render_forward_masked(ctx: Context, cams, g: Gaussians, settings: RenderSettings, mask_out, color, depth, alpha,
                          target_color=None, target_depth=None, w_color: float = 1.0, w_depth: float = 1.0,
                          loss_out=None, index_map: Optional[torch.Tensor] = None, stream=None):
    """Unstable-pixel mask (written to mask_out) and the forward on it, in one pass."""
    arr, F = _cams(cams)
    gc = g.to_c()
    prm = settings.to_c()
    st = _lib.load().rtg_render_forward_masked(
        ctx.ptr, arr, F, ctypes.byref(gc), ctypes.byref(prm), _ptr(mask_out, torch.uint8, "mask_out"),
        _ptr(target_color, torch.float32, "target_color"), _ptr(target_depth, torch.float32, "target_depth"),
        float(w_color), float(w_depth), _ptr(color, torch.float32, "color"), _ptr(depth, torch.float32, "depth"),
        _ptr(alpha, torch.float32, "alpha"), _ptr(index_map, torch.int32, "index_map"),
        _ptr(loss_out, torch.float32, "loss_out"), _stream(stream))
    _check(st, "rtg_render_forward_masked", ctx.ptr)


def render_backward_l1(ctx: Context, g_means, g_scales, g_quats, g_opacity, g_colors, accumulate: bool = False,
                       stream=None):
    st = _lib.load().rtg_render_backward_l1(ctx.ptr, _out_ptr(g_means, "g_means"), _out_ptr(g_scales, "g_scales"),
                                            _out_ptr(g_quats, "g_quats"), _out_ptr(g_opacity, "g_opacity"),
                                            _out_ptr(g_colors, "g_colors"), 1 if accumulate else 0,
                                            _stream(stream))
    _check(st, "rtg_render_backward_l1", ctx.ptr)


def loss_counts(ctx: Context, counts_out: torch.Tensor, stream=None):
    """rtg_loss_counts: (P, P_d, L1 colour sum, L1 depth sum) of the last forward with targets
    into a float64 device tensor of 4."""
    _check(_lib.load().rtg_loss_counts(ctx.ptr, _ptr(counts_out, torch.float64, "counts_out"), _stream(stream)),
           "rtg_loss_counts", ctx.ptr)


def set_loss_scales(ctx: Context, totals: torch.Tensor, w_color: float, w_depth: float, loss_out=None,
                    stream=None):
    """rtg_set_loss_scales: the next backward_l1's gradient scales from batch totals (float64
    device tensor of 4, summed rtg_loss_counts outputs); loss_out (float32 device [3]) gets the
    batch's loss."""
    st = _lib.load().rtg_set_loss_scales(ctx.ptr, _ptr(totals, torch.float64, "totals"), float(w_color),
                                         float(w_depth), _ptr(loss_out, torch.float32, "loss_out"),
                                         _stream(stream))
    _check(st, "rtg_set_loss_scales", ctx.ptr)


def l1_loss(ctx: Context, color, depth, target_color, target_depth, mask, w_color: float, w_depth: float,
            loss_out, dL_dcolor, dL_ddepth, stream=None):
    F, C, H, W = color.shape
    st = _lib.load().rtg_l1_loss(ctx.ptr, F, C, H, W, _ptr(color, torch.float32, "color"),
                                 _ptr(depth, torch.float32, "depth"), _ptr(target_color, torch.float32, "target_color"),
                                 _ptr(target_depth, torch.float32, "target_depth"), _ptr(mask, torch.uint8, "mask"),
                                 float(w_color), float(w_depth), _ptr(loss_out, torch.float32, "loss_out"),
                                 _ptr(dL_dcolor, torch.float32, "dL_dcolor"), _ptr(dL_ddepth, torch.float32, "dL_ddepth"),
                                 _stream(stream))
    _check(st, "rtg_l1_loss", ctx.ptr)


def select_top_error(ctx: Context, color: torch.Tensor, target_color: torch.Tensor, frac: float,
                     mask_out: torch.Tensor, stream=None):
    """Per frame, 1 in mask_out [F,H,W] (uint8) on the floor(frac*H*W) pixels of largest
    colour error |color - target| summed over channels; ties to the lower pixel index."""
    F, C, H, W = color.shape
    if tuple(target_color.shape) != (F, C, H, W) or tuple(mask_out.shape) != (F, H, W):
        raise ValueError("select_top_error: color/target [F,C,H,W] and mask_out [F,H,W] must agree")
    st = _lib.load().rtg_select_top_error(ctx.ptr, F, C, H, W, _ptr(color, torch.float32, "color"),
                                          _ptr(target_color, torch.float32, "target_color"), float(frac),
                                          _ptr(mask_out, torch.uint8, "mask_out"), _stream(stream))
    _check(st, "rtg_select_top_error", ctx.ptr)


def narrow_pixels(ctx: Context, mask: torch.Tensor, target_color: Optional[torch.Tensor] = None,
                  target_depth: Optional[torch.Tensor] = None, w_color: float = 1.0, w_depth: float = 1.0,
                  loss_out: Optional[torch.Tensor] = None, stream=None):
    """Restrict the last forward's pixels to those set in mask [F,H,W] (uint8) for the next
    backward.  With the targets and loss_out it also forms the L1 loss on those pixels, for
    render_backward_l1; without them use l1_loss on the same mask and render_backward."""
    st = _lib.load().rtg_narrow_pixels(ctx.ptr, _ptr(mask, torch.uint8, "mask"),
                                       _ptr(target_color, torch.float32, "target_color"),
                                       _ptr(target_depth, torch.float32, "target_depth"), float(w_color),
                                       float(w_depth), _ptr(loss_out, torch.float32, "loss_out"), _stream(stream))
    _check(st, "rtg_narrow_pixels", ctx.ptr)


def add_candidates(ctx: Context, cams, render_color, render_alpha, render_depth, index_map, color, depth,
                   unstable: torch.Tensor, settings: AddSettings, seed: int, count_out: torch.Tensor,
                   pixel_out: torch.Tensor, kind_out: torch.Tensor, position_out: torch.Tensor,
                   color_out: torch.Tensor, opacity_out: torch.Tensor, stream=None):
    """The new Gaussians of the adding pass (rtg_add_candidates): up to pixel_out.numel() of
    them written in (frame, pixel) order; count_out [1] int64 receives their number."""
    arr, F = _cams(cams)
    C = int(render_color.shape[1])
    cap = int(pixel_out.numel())
    prm = settings.to_c(seed)
    st = _lib.load().rtg_add_candidates(
        ctx.ptr, arr, F, C, _ptr(render_color, torch.float32, "render_color"),
        _ptr(render_alpha, torch.float32, "render_alpha"), _ptr(render_depth, torch.float32, "render_depth"),
        _ptr(index_map, torch.int32, "index_map"), _ptr(color, torch.float32, "color"),
        _ptr(depth, torch.float32, "depth"), _ptr(unstable, torch.uint8, "unstable"), int(unstable.numel()),
        ctypes.byref(prm), cap, _ptr(count_out, torch.int64, "count_out"), _ptr(pixel_out, torch.int32, "pixel_out"),
        _ptr(kind_out, torch.uint8, "kind_out"), _ptr(position_out, torch.float32, "position_out"),
        _ptr(color_out, torch.float32, "color_out"), _ptr(opacity_out, torch.float32, "opacity_out"),
        _stream(stream))
    _check(st, "rtg_add_candidates", ctx.ptr)


@dataclasses.dataclass(frozen=True)
class StateSettings:
    """Thresholds of the state management (Section 3.2): confidence count for stability, error
    count for instability, age (frames) for removal, and the colour / depth error of a pixel.
    delta_e and delta_t are not given in the paper."""
    delta_eta: int = 100
    delta_e: int = 10
    delta_t: int = 200
    delta_c: float = 0.1
    delta_d: float = 0.1

    def to_c(self) -> "_lib.rtg_state_params":
        return _lib.rtg_state_params(int(self.delta_eta), int(self.delta_e), int(self.delta_t), float(self.delta_c),
                                     float(self.delta_d))


@dataclasses.dataclass
class MapArrays:
    """Every per-Gaussian array of the map (rtg_map_arrays)."""
    means: torch.Tensor
    scales: torch.Tensor
    quats: torch.Tensor
    opacity: torch.Tensor
    colors: torch.Tensor
    unstable: torch.Tensor  # u8
    eta: torch.Tensor       # int32 confidence count
    err: torch.Tensor       # int32 error count
    t0: torch.Tensor        # int32 frame of creation

    def to_c(self) -> "_lib.rtg_map_arrays":
        f = lambda t, dt, k: _ptr(t, dt, k)  # noqa: E731
        return _lib.rtg_map_arrays(*[f(getattr(self, k), torch.float32, k) for k in
                                     ("means", "scales", "quats", "opacity", "colors")],
                                   f(self.unstable, torch.uint8, "unstable"), f(self.eta, torch.int32, "eta"),
                                   f(self.err, torch.int32, "err"), f(self.t0, torch.int32, "t0"))

    @staticmethod
    def empty_like(a: "MapArrays") -> "MapArrays":
        return MapArrays(*[torch.empty_like(getattr(a, f.name)) for f in dataclasses.fields(MapArrays)])


def transparent_reg(ctx: Context, compact: Sequence[torch.Tensor], initial: Sequence[torch.Tensor], grads,
                    loss_out: torch.Tensor, w_reg: float = 1000.0, alpha_split: float = 0.5, stream=None):
    """Adds the gradient of w_reg L_reg (transparent Gaussians held to their initial position,
    rotation and scale) to grads (means, scales, quats); loss_out [1] receives w_reg L_reg.
    compact: (means, scales, quats, opacity, ...) [nu, .]; initial: (means0, scales0, quats0)."""
    nu = int(compact[0].shape[0])
    st = _lib.load().rtg_transparent_reg(ctx.ptr, nu, *[_ptr(t, torch.float32, "compact") for t in compact[:4]],
                                         *[_ptr(t, torch.float32, "initial") for t in initial[:3]], float(w_reg),
                                         float(alpha_split), *[_ptr(t, torch.float32, "grad") for t in grads[:3]],
                                         _ptr(loss_out, torch.float32, "loss_out"), _stream(stream))
    _check(st, "rtg_transparent_reg", ctx.ptr)


def confidence_update(ids: torch.Tensor, g_colors: torch.Tensor, eta: torch.Tensor, stream=None):
    """eta[ids[k]] += 1 where the colour gradient row g_colors[k] is non-zero."""
    nu = int(ids.numel())
    if nu == 0:
        return
    C = int(g_colors.numel()) // nu
    st = _lib.load().rtg_confidence_update(nu, C, _ptr(ids, torch.int32, "ids"), _ptr(g_colors, torch.float32, "g_colors"),
                                           _ptr(eta, torch.int32, "eta"), _stream(stream))
    _check(st, "rtg_confidence_update")


def fuse_window(ids: torch.Tensor, eta_start: torch.Tensor, eta_now: torch.Tensor, compact: Sequence[torch.Tensor],
                g: Gaussians, stream=None):
    """Eq. 9: blend the optimised compact rows into the full arrays of g with weights from
    the confidence counts (in place)."""
    nu, C = int(ids.numel()), g.color_width
    if nu == 0:
        return
    st = _lib.load().rtg_fuse_window(nu, C, _ptr(ids, torch.int32, "ids"), _ptr(eta_start, torch.int32, "eta_start"),
                                     _ptr(eta_now, torch.int32, "eta_now"),
                                     *[_ptr(t, torch.float32, "compact") for t in compact],
                                     *[_ptr(getattr(g, k), torch.float32, k) for k in
                                       ("means", "scales", "quats", "opacity", "colors")], _stream(stream))
    _check(st, "rtg_fuse_window")


def error_count(ctx: Context, render_color, render_depth, index_map, color, depth, unstable: torch.Tensor,
                settings: StateSettings, err: torch.Tensor, stream=None):
    """err[i] += the number of frames in which stable Gaussian i is the depth hit of an
    erring pixel."""
    F, C, H, W = render_color.shape
    prm = settings.to_c()
    st = _lib.load().rtg_error_count(ctx.ptr, F, C, H, W, _ptr(render_color, torch.float32, "render_color"),
                                     _ptr(render_depth, torch.float32, "render_depth"),
                                     _ptr(index_map, torch.int32, "index_map"), _ptr(color, torch.float32, "color"),
                                     _ptr(depth, torch.float32, "depth"), _ptr(unstable, torch.uint8, "unstable"),
                                     int(unstable.numel()), ctypes.byref(prm), _ptr(err, torch.int32, "err"),
                                     _stream(stream))
    _check(st, "rtg_error_count", ctx.ptr)


def update_states(frame: int, t0, settings: StateSettings, unstable, eta, err, remove, stream=None):
    prm = settings.to_c()
    st = _lib.load().rtg_update_states(int(unstable.numel()), int(frame), _ptr(t0, torch.int32, "t0"),
                                       ctypes.byref(prm), _ptr(unstable, torch.uint8, "unstable"),
                                       _ptr(eta, torch.int32, "eta"), _ptr(err, torch.int32, "err"),
                                       _ptr(remove, torch.uint8, "remove"), _stream(stream))
    _check(st, "rtg_update_states")


def compact_gaussians(ctx: Context, remove: torch.Tensor, src: MapArrays, dst: MapArrays, count_out: torch.Tensor,
                      stream=None):
    """Copy the rows of src not flagged in remove, in order, to dst; count_out [1] int64."""
    n = int(remove.numel())
    C = _row_width(src.colors)
    a, b = src.to_c(), dst.to_c()
    st = _lib.load().rtg_compact_gaussians(ctx.ptr, n, C, _ptr(remove, torch.uint8, "remove"), ctypes.byref(a),
                                           ctypes.byref(b), _ptr(count_out, torch.int64, "count_out"),
                                           _stream(stream))
    _check(st, "rtg_compact_gaussians", ctx.ptr)


_DUMMY = {}


def _out_ptr(t: torch.Tensor, name: str):
    """Gradient outputs may be empty when no Gaussian is unstable; pass a scratch word."""
    if t.numel() == 0:
        dev = t.device
        if dev not in _DUMMY:
            _DUMMY[dev] = torch.zeros(4, dtype=torch.float32, device=dev)
        return _DUMMY[dev].data_ptr()
    return _ptr(t, torch.float32, name)


def render_backward(ctx: Context, dL_dcolor, dL_ddepth, g_means, g_scales, g_quats, g_opacity, g_colors,
                    accumulate: bool = False, stream=None):
    st = _lib.load().rtg_render_backward(ctx.ptr, _ptr(dL_dcolor, torch.float32, "dL_dcolor"),
                                         _ptr(dL_ddepth, torch.float32, "dL_ddepth"), _out_ptr(g_means, "g_means"),
                                         _out_ptr(g_scales, "g_scales"), _out_ptr(g_quats, "g_quats"),
                                         _out_ptr(g_opacity, "g_opacity"), _out_ptr(g_colors, "g_colors"),
                                         1 if accumulate else 0, _stream(stream))
    _check(st, "rtg_render_backward", ctx.ptr)


def decode_rgbd(rgb: torch.Tensor, depth: torch.Tensor, depth_scale: float, color: torch.Tensor,
                depth_out: torch.Tensor, stream=None):
    """RGB-D sensor frames to the float planes the loss reads (rtg_decode_rgbd): rgb uint8
    [F,H,W,3] (or [H,W,3]), depth uint16 [F,H,W] (or [H,W]) in 1/depth_scale metres; writes
    color [F,3,H,W] = rgb / 255 and depth_out [F,H,W] = depth / depth_scale (0 stays 0)."""
    if rgb.dim() == 3:
        rgb = rgb.unsqueeze(0)
    if depth.dim() == 2:
        depth = depth.unsqueeze(0)
    F, H, W, three = rgb.shape
    if three != 3 or tuple(depth.shape) != (F, H, W):
        raise ValueError("rgb must be [F,H,W,3] and depth [F,H,W]")
    if color.numel() != F * 3 * H * W or depth_out.numel() != F * H * W:
        raise ValueError("color must hold F*3*H*W values and depth_out F*H*W")
    st = _lib.load().rtg_decode_rgbd(F, H, W, _ptr(rgb, torch.uint8, "rgb"), _ptr(depth, torch.uint16, "depth"),
                                     float(depth_scale), _ptr(color, torch.float32, "color"),
                                     _ptr(depth_out, torch.float32, "depth_out"), _stream(stream))
    _check(st, "rtg_decode_rgbd")


def _row_width(colors: torch.Tensor) -> int:
    """Values per Gaussian of a colour array [n, ...], from its shape (so also when n = 0)."""
    return int(math.prod(colors.shape[1:])) if colors.dim() > 1 else 1


def adam_step(params: Sequence[torch.Tensor], grads: Sequence[torch.Tensor], m: torch.Tensor, v: torch.Tensor,
              step: int, hp: AdamSettings = AdamSettings(), stream=None):
    """params/grads: compact (means, scales, quats, opacity, colors); m, v: nu * (11 + C) floats
    each, zero at the start, laid out group by group like the parameters."""
    means, scales, quats, opacity, colors = params
    nu = int(means.shape[0])
    C = _row_width(colors)
    c = hp.to_c()
    ptrs = [_ptr(t, torch.float32, "param") for t in params] + [_ptr(t, torch.float32, "grad") for t in grads]
    st = _lib.load().rtg_adam_step(nu, C, *ptrs, _ptr(m, torch.float32, "m"), _ptr(v, torch.float32, "v"),
                                   int(step), ctypes.byref(c), _stream(stream))
    _check(st, "rtg_adam_step")


def adam_step_counted(params: Sequence[torch.Tensor], grads: Sequence[torch.Tensor], m: torch.Tensor,
                      v: torch.Tensor, step_counter: torch.Tensor, hp: AdamSettings = AdamSettings(), stream=None,
                      after_gradients: bool = False):
    """Adam with the step count in device memory: step_counter is int32 [2] (completed steps,
    and scratch that the call returns to 0); the call increments [0].  after_gradients: the
    kernel just in front on the stream writes none of params, m, v, step_counter
    (rtg_adam_step_counted_after_gradients: the loads start while it finishes)."""
    if step_counter.numel() < 2:
        raise ValueError("step_counter must hold 2 int32 (completed steps, scratch)")
    means, scales, quats, opacity, colors = params
    nu = int(means.shape[0])
    C = _row_width(colors)
    c = hp.to_c()
    ptrs = [_ptr(t, torch.float32, "param") for t in params] + [_ptr(t, torch.float32, "grad") for t in grads]
    lib = _lib.load()
    fn = lib.rtg_adam_step_counted_after_gradients if after_gradients else lib.rtg_adam_step_counted
    st = fn(nu, C, *ptrs, _ptr(m, torch.float32, "m"), _ptr(v, torch.float32, "v"),
            _ptr(step_counter, torch.int32, "step_counter"), ctypes.byref(c), _stream(stream))
    _check(st, "rtg_adam_step_counted")


def unstable_index(ctx: Context, unstable: torch.Tensor, stream=None):
    """Returns (ids int32 [nu] on the device, nu).  Synchronises to read the count."""
    n = int(unstable.shape[0])
    ids = torch.empty(max(n, 1), dtype=torch.int32, device=unstable.device)
    nu_t = torch.zeros(1, dtype=torch.int64, device=unstable.device)
    st = _lib.load().rtg_unstable_index(ctx.ptr, n, _ptr(unstable, torch.uint8, "unstable"),
                                        ids.data_ptr(), nu_t.data_ptr(), _stream(stream))
    _check(st, "rtg_unstable_index", ctx.ptr)
    nu = int(nu_t.item())
    return ids[:nu], nu


def unstable_index_static(unstable: torch.Tensor, ids: torch.Tensor, nu_out: torch.Tensor, stream=None):
    """Allocation-free unstable index (no context): fills ids [>= nu] int32 and nu_out [1]
    int64 on the device.  For callers that must not allocate device memory; limited to
    16,777,216 Gaussians.  Does not synchronise."""
    n = int(unstable.shape[0])
    st = _lib.load().rtg_unstable_index_static(n, _ptr(unstable, torch.uint8, "unstable"),
                                               _ptr(ids, torch.int32, "ids"), _ptr(nu_out, torch.int64, "nu_out"),
                                               _stream(stream))
    _check(st, "rtg_unstable_index_static")


def unstable_rank(ctx: Context, unstable: torch.Tensor, stream=None):
    """(rank int32 [N], ids int32 [nu], nu): the unstable index for rtg_gaussians.rank_map.
    Synchronises to read the count."""
    n = int(unstable.shape[0])
    rank = torch.empty(max(n, 1), dtype=torch.int32, device=unstable.device)
    ids = torch.empty(max(n, 1), dtype=torch.int32, device=unstable.device)
    nu_t = torch.zeros(1, dtype=torch.int64, device=unstable.device)
    st = _lib.load().rtg_unstable_rank(ctx.ptr, n, _ptr(unstable, torch.uint8, "unstable"), rank.data_ptr(),
                                       ids.data_ptr(), nu_t.data_ptr(), _stream(stream))
    _check(st, "rtg_unstable_rank", ctx.ptr)
    nu = int(nu_t.item())
    return rank[:n], ids[:nu], nu


def gather_unstable(ids: torch.Tensor, g: Gaussians, stream=None):
    nu, C = int(ids.shape[0]), g.color_width
    dev = g.means.device
    out = (torch.empty(nu, 3, device=dev), torch.empty(nu, 3, device=dev), torch.empty(nu, 4, device=dev),
           torch.empty(nu, device=dev), torch.empty((nu,) + tuple(g.colors.shape[1:]), device=dev))
    if nu:
        st = _lib.load().rtg_gather_unstable(nu, C, _ptr(ids, torch.int32, "ids"),
                                             *[_ptr(getattr(g, k), torch.float32, k) for k in
                                               ("means", "scales", "quats", "opacity", "colors")],
                                             *[_ptr(t, torch.float32, "out") for t in out], _stream(stream))
        _check(st, "rtg_gather_unstable")
    return out


def scatter_unstable(ids: torch.Tensor, compact: Sequence[torch.Tensor], g: Gaussians, stream=None):
    nu, C = int(ids.shape[0]), g.color_width
    if nu == 0:
        return
    st = _lib.load().rtg_scatter_unstable(nu, C, _ptr(ids, torch.int32, "ids"),
                                          *[_ptr(t, torch.float32, "compact") for t in compact],
                                          *[_ptr(getattr(g, k), torch.float32, k) for k in
                                            ("means", "scales", "quats", "opacity", "colors")], _stream(stream))
    _check(st, "rtg_scatter_unstable")


def get_stats(ctx: Context) -> dict:
    s = rtg_stats()
    _check(_lib.load().rtg_get_stats(ctx.ptr, ctypes.byref(s)), "rtg_get_stats", ctx.ptr)
    return {f[0]: getattr(s, f[0]) for f in rtg_stats._fields_}


def get_status(ctx: Context) -> int:
    return int(_lib.load().rtg_get_status(ctx.ptr))


def reset_status(ctx: Context):
    _lib.load().rtg_reset_status(ctx.ptr)


def last_error(ctx: Context) -> str:
    return _lib.load().rtg_last_error(ctx.ptr).decode()


def debug_binning(ctx: Context, frames: int, width: int, height: int, n: int, stream=None):
    """Copies of the last forward's bucket offsets, sorted ids, per-(frame, Gaussian) tile
    rectangles and depth-key bits (for the exactness tests)."""
    stats = get_stats(ctx)
    tw, th = stats["tile_w"], stats["tile_h"]
    T = ((width + tw - 1) // tw) * ((height + th - 1) // th)
    dev = torch.device("cuda", torch.cuda.current_device())
    offs = torch.empty(frames * T + 1, dtype=torch.int32, device=dev)
    ids = torch.empty(max(stats["pairs"], 1), dtype=torch.int32, device=dev)
    rect = torch.empty(max(frames * n, 1), 4, dtype=torch.int32, device=dev)
    zb = torch.empty(max(frames * n, 1), dtype=torch.int32, device=dev)
    st = _lib.load().rtg_debug_binning(ctx.ptr, offs.data_ptr(), ids.data_ptr(), rect.data_ptr(), zb.data_ptr(),
                                       _stream(stream))
    _check(st, "rtg_debug_binning", ctx.ptr)
    torch.cuda.synchronize()
    u32 = lambda t: t.cpu().numpy().view(np.uint32)  # noqa: E731
    return dict(tile_offsets=u32(offs), sorted_ids=u32(ids[:stats["pairs"]]), rect=rect[:frames * n].cpu().numpy(),
                zbits=u32(zb[:frames * n]), pairs=stats["pairs"])


def profile_enable(ctx: Context, on: bool = True):
    """Per-kernel device timing (CUDA events around each kernel launcher of the context)."""
    _check(_lib.load().rtg_profile_enable(ctx.ptr, 1 if on else 0), "rtg_profile_enable", ctx.ptr)


def profile_read(ctx: Context) -> dict:
    """{kernel kind: (launches, total milliseconds)} since the last read (synchronises)."""
    lib = _lib.load()
    k = int(lib.rtg_profile_kinds())
    launches = (ctypes.c_int64 * k)()
    ms = (ctypes.c_double * k)()
    _check(lib.rtg_profile_read(ctx.ptr, launches, ms, k), "rtg_profile_read", ctx.ptr)
    return {lib.rtg_profile_kind_name(i).decode(): (int(launches[i]), float(ms[i])) for i in range(k)}


def alu_probe(kind: int, iters: int, out: torch.Tensor, stream=None) -> int:
    """Launches the arithmetic-pipe probe (kind 0: FP32 FMA, kind 1: SFU ex2) on the current
    device and returns the operations it performs; `out` is a float32 device scratch of at
    least 2048 x SM-count entries.  The caller times the launch."""
    ops = ctypes.c_int64()
    _check(_lib.load().rtg_alu_probe(int(kind), int(iters), _ptr(out), ctypes.byref(ops), _stream(stream)),
           "rtg_alu_probe")
    return int(ops.value)
