"""Keyframes and global optimisation (Section 3.2, "Keyframes and global optimization").

Whenever a keyframe is added, every Gaussian of the map is optimised over the latest
keyframe and three earlier ones drawn at random, with the loss of the on-the-fly step
(Eq. 8), but only on each keyframe's pixels with the 40% largest colour errors.  Positions
stay fixed and the other parameters use 0.1x the learning rates.  When the scan ends the
map is refined over all keyframes for 10x as many iterations as there are keyframes.

``KeyframeSet`` is the host-side policy (which frames become keyframes, which keyframes a
global step uses); ``GlobalStep`` is one global iteration as C-ABI calls on preallocated
buffers: a full-frame forward of every Gaussian, the top-error selection, the narrowing of
the forward to the selected pixels, the L1 loss on them, the backward and Adam.
"""

from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import api
from .api import AdamSettings, Context, Gaussians, RenderSettings


def rotation_angle_deg(R_a, R_b) -> float:
    """Angle (degrees) of the rotation taking orientation R_a to R_b: acos((tr(R_a^T R_b) - 1) / 2)."""
    Ra = np.asarray(R_a, dtype=np.float64).reshape(3, 3)
    Rb = np.asarray(R_b, dtype=np.float64).reshape(3, 3)
    c = 0.5 * (float(np.sum(Ra * Rb)) - 1.0)  # tr(Ra^T Rb) is the elementwise product sum
    return math.degrees(math.acos(min(1.0, max(-1.0, c))))


class KeyframeSet:
    """The keyframe list: a frame becomes a keyframe when its rotation relative to the last
    keyframe exceeds ``angle_deg`` or its camera moved more than ``move_m`` (30 degrees and
    0.3 m in the paper); the first frame offered is always one."""

    def __init__(self, angle_deg: float = 30.0, move_m: float = 0.3):
        self.angle_deg, self.move_m = float(angle_deg), float(move_m)
        self.frames: List[int] = []   # frame ids of the keyframes, in order
        self.poses: List[tuple] = []  # (R [3,3], t [3]) float64

    def __len__(self) -> int:
        return len(self.frames)

    def is_new(self, R, t) -> bool:
        if not self.poses:
            return True
        R0, t0 = self.poses[-1]
        if rotation_angle_deg(R0, R) > self.angle_deg:
            return True
        return float(np.linalg.norm(np.asarray(t, dtype=np.float64).reshape(3) - t0)) > self.move_m

    def offer(self, frame: int, R, t) -> bool:
        """Add frame ``frame`` with camera-to-world pose (R, t) if the rule takes it."""
        if not self.is_new(R, t):
            return False
        self.frames.append(int(frame))
        self.poses.append((np.asarray(R, dtype=np.float64).reshape(3, 3).copy(),
                           np.asarray(t, dtype=np.float64).reshape(3).copy()))
        return True

    def pick(self, rng: np.random.Generator, n_random: int = 3) -> List[int]:
        """Positions (into this list) of the keyframes of one global step: the latest and
        ``n_random`` distinct earlier ones drawn uniformly (all earlier ones if fewer)."""
        if not self.frames:
            return []
        last = len(self.frames) - 1
        k = min(n_random, last)
        earlier = rng.choice(last, size=k, replace=False) if k > 0 else np.zeros(0, dtype=np.int64)
        return [last] + sorted(int(i) for i in earlier)

    def final_schedule(self, per_keyframe: int = 10) -> List[int]:
        """Keyframe positions of the final refinement, one per iteration: 10x as many
        iterations as keyframes, passing over the list in order."""
        n = len(self.frames)
        return [i % n for i in range(per_keyframe * n)]


def global_adam(base: AdamSettings = AdamSettings(), lr_factor: float = 0.1) -> AdamSettings:
    """Adam settings of the global optimisation: positions fixed (learning rate 0), the other
    groups at lr_factor x their on-the-fly rates."""
    return dataclasses.replace(base, lr_means=0.0, lr_scales=base.lr_scales * lr_factor,
                               lr_quats=base.lr_quats * lr_factor, lr_opacity=base.lr_opacity * lr_factor,
                               lr_colors=base.lr_colors * lr_factor, lr_colors_rest=base.lr_colors_rest * lr_factor)


class GlobalStep:
    """One global iteration per ``step()`` over up to ``max_frames`` keyframes of one size.

    Every Gaussian is optimised: the step flags them all as optimised (the rasterizer's
    "unstable" set is the whole map) and owns Adam moments for all of them.  Per call:
      1. forward of all Gaussians on every pixel of the keyframes;
      2. per keyframe, the ``frac`` pixels of largest colour error (rtg_select_top_error);
      3. the forward narrowed to those pixels, with the L1 colour + depth loss (Eq. 7/8)
         formed on them in the same pass (rtg_narrow_pixels: no second render);
      4. the fused backward to every Gaussian, and Adam with ``global_adam`` settings, in
         place on the full arrays of ``g``.
    The calls allocate nothing and never synchronise; ``capture()`` records one iteration in
    a CUDA graph for a fixed set of cameras and target buffers.
    """

    def __init__(self, ctx: Context, g: Gaussians, width: int, height: int, max_frames: int = 4,
                 settings: RenderSettings = RenderSettings(), adam: AdamSettings = AdamSettings(),
                 frac: float = 0.4, lr_factor: float = 0.1, w_color: float = 1.0, w_depth: float = 1.0):
        if ctx.cap.max_frames < max_frames:
            raise ValueError(f"context holds {ctx.cap.max_frames} frames, the step needs {max_frames}")
        self.ctx, self.settings, self.frac = ctx, settings, float(frac)
        self.hyper = global_adam(adam, lr_factor)
        self.w_color, self.w_depth = w_color, w_depth
        dev = g.means.device
        n, C, Cw = g.n, g.channels, g.color_width
        if g.sh_degree > 0 and self.hyper.colors_dc == 0:  # SH0 rate for the degree-0 terms only
            self.hyper = dataclasses.replace(self.hyper, colors_dc=3)
        self.flags = torch.ones(n, dtype=torch.uint8, device=dev)
        rank, ids, nu = api.unstable_rank(ctx, self.flags)
        self.g = dataclasses.replace(g, unstable=self.flags, rank_map=rank, unstable_ids=ids, n_unstable=nu,
                                     u_means=None, u_scales=None, u_quats=None, u_opacity=None, u_colors=None)
        self.params = (g.means, g.scales, g.quats, g.opacity, g.colors)
        self.grads = [torch.zeros_like(t) for t in self.params]
        self.m = torch.zeros(n * (11 + Cw), device=dev)
        self.v = torch.zeros(n * (11 + Cw), device=dev)
        self.step_counter = torch.zeros(2, dtype=torch.int32, device=dev)
        Fm, H, W = max_frames, height, width
        self.color = torch.zeros(Fm, C, H, W, device=dev)
        self.depth = torch.full((Fm, H, W), -1.0, device=dev)
        self.alpha = torch.zeros(Fm, H, W, device=dev)
        self.selected = torch.zeros(Fm, H, W, dtype=torch.uint8, device=dev)
        self.loss = torch.zeros(3, device=dev)
        self.graph = None

    def _body(self, cams: Sequence, target_color: torch.Tensor, target_depth: torch.Tensor, stream=None):
        F = len(cams)
        color, depth, alpha, sel = self.color[:F], self.depth[:F], self.alpha[:F], self.selected[:F]
        api.render_forward(self.ctx, list(cams), self.g, None, self.settings, color, depth, alpha, None, stream)
        api.select_top_error(self.ctx, color, target_color, self.frac, sel, stream)
        api.narrow_pixels(self.ctx, sel, target_color, target_depth, self.w_color, self.w_depth, self.loss, stream)
        api.render_backward_l1(self.ctx, *self.grads, stream=stream)
        api.adam_step_counted(self.params, self.grads, self.m, self.v, self.step_counter, self.hyper, stream)
        return self.loss

    def step(self, cams: Sequence, target_color: torch.Tensor, target_depth: torch.Tensor, stream=None):
        """One global iteration on keyframes ``cams`` with targets [F,C,H,W] / [F,H,W];
        returns the device loss (L, L_color, L_depth) on the selected pixels."""
        if self.graph is not None:
            self.graph.replay()
            return self.loss
        return self._body(cams, target_color, target_depth, stream)

    def capture(self, cams: Sequence, target_color: torch.Tensor, target_depth: torch.Tensor):
        """Record one iteration for these cameras and target buffers in a CUDA graph; later
        ``step()`` calls replay it (refill the targets in place to change them)."""
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            self._body(cams, target_color, target_depth)
        torch.cuda.synchronize()
        self.graph = graph
        return graph

    def release(self):
        self.graph = None
