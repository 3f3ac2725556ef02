"""The masked on-the-fly optimisation step (Section 3.2, "Gaussian optimization"; Supplement B)
on top of the C ABI: forward over all Gaussians on the unstable pixels, L1 colour and
depth losses, backward to the unstable Gaussians only, Adam on their compact parameters.

Two front ends:
  * ``RTGRasterize``: a torch.autograd.Function whose differentiable inputs are the
    compact unstable parameters [Nu, .]; its backward returns their gradients.
  * ``MaskedStep``: the whole iteration (forward, loss, backward, Adam) as five C-ABI
    calls on preallocated buffers, with no allocation and no host synchronisation.
"""

from __future__ import annotations

import dataclasses
from typing import Optional, Sequence

import torch

from . import api
from .api import AdamSettings, Context, Gaussians, RenderSettings


@dataclasses.dataclass
class RasterState:
    """Non-differentiable inputs of one render: context, full arrays, cameras, mask."""
    ctx: Context
    g: Gaussians
    cams: Sequence
    mask: Optional[torch.Tensor]
    settings: RenderSettings
    color: torch.Tensor = None   # outputs, reused across calls; off-mask pixels keep their fill
    depth: torch.Tensor = None
    alpha: torch.Tensor = None
    index_map: Optional[torch.Tensor] = None

    def __post_init__(self):
        cams = self.cams if isinstance(self.cams, (list, tuple)) else [self.cams]
        F, H, W, C = len(cams), int(cams[0].height), int(cams[0].width), self.g.channels
        dev = self.g.means.device
        if self.color is None:
            self.color = torch.zeros(F, C, H, W, device=dev)
            self.depth = torch.full((F, H, W), -1.0, device=dev)
            self.alpha = torch.zeros(F, H, W, device=dev)
            self.index_map = torch.full((F, H, W), -1, dtype=torch.int32, device=dev)


class RTGRasterize(torch.autograd.Function):
    """(u_means, u_scales, u_quats, u_opacity, u_colors) -> (colour, depth, alpha)."""

    @staticmethod
    def forward(ctx, u_means, u_scales, u_quats, u_opacity, u_colors, state: RasterState):
        g = dataclasses.replace(state.g, u_means=u_means.detach().contiguous(),
                                u_scales=u_scales.detach().contiguous(), u_quats=u_quats.detach().contiguous(),
                                u_opacity=u_opacity.detach().contiguous(), u_colors=u_colors.detach().contiguous())
        api.render_forward(state.ctx, state.cams, g, state.mask, state.settings, state.color, state.depth,
                           state.alpha, state.index_map)
        ctx.state = state
        ctx.shapes = (u_means.shape, u_scales.shape, u_quats.shape, u_opacity.shape, u_colors.shape)
        ctx.mark_non_differentiable(state.alpha)
        return state.color.clone(), state.depth.clone(), state.alpha.clone()

    @staticmethod
    def backward(ctx, d_color, d_depth, d_alpha):
        st: RasterState = ctx.state
        dev = st.color.device
        if d_color is None:
            d_color = torch.zeros_like(st.color)
        if d_depth is None:
            d_depth = torch.zeros_like(st.depth)
        grads = [torch.empty(s, device=dev) for s in ctx.shapes]
        api.render_backward(st.ctx, d_color.contiguous().float(), d_depth.contiguous().float(), *grads)
        return (*grads, None)


def rasterize(u_params: Sequence[torch.Tensor], state: RasterState):
    return RTGRasterize.apply(*u_params, state)


class MaskedStep:
    """One masked optimisation iteration per ``step()`` call, on preallocated buffers.

    With ``recompute_mask`` the unstable-pixel mask (Supplement B) is rebuilt from the
    current unstable parameters at the start of every iteration, so one call runs the whole
    path: mask, forward, L1 loss, backward, Adam.  ``capture()`` records one iteration in a
    CUDA graph; later ``step()`` calls replay it (same cameras and buffers; the Adam step
    count lives on the device).

    The step is one optimisation window (Section 3.2): its cameras and unstable set are
    fixed and only the unstable Gaussians move.  With ``window`` (default) it opens the
    context's window, so the stable Gaussians are projected once here and every iteration
    projects only the unstable ones (results identical; rtg_window_begin).

    With ``frame = (rgb, depth, depth_scale)`` (uint8 [F,H,W,3], uint16 [F,H,W], device) the
    step's input is the sensor frame itself: every iteration first decodes it into
    ``target_color`` / ``target_depth`` (rtg_decode_rgbd), so a frame loop uploads 5 bytes a
    pixel instead of the 16 of the float planes.
    """

    def __init__(self, ctx: Context, g: Gaussians, cams, mask: Optional[torch.Tensor], target_color: torch.Tensor,
                 target_depth: torch.Tensor, settings: RenderSettings = RenderSettings(),
                 adam: AdamSettings = AdamSettings(), w_color: float = 1.0, w_depth: float = 1.0,
                 recompute_mask: bool = False, window: bool = True, scatter_every_step: bool = False,
                 map_state=None, initial: Optional[Sequence[torch.Tensor]] = None, w_reg: float = 1000.0,
                 frame=None):
        if g.sh_degree > 0 and adam.colors_dc == 0:  # Supplement C: SH0 rate for the degree-0 terms
            adam = dataclasses.replace(adam, colors_dc=3)
        self.ctx, self.settings, self.adam = ctx, settings, adam
        self.cams = cams if isinstance(cams, (list, tuple)) else [cams]
        self.mask = mask
        self.recompute_mask = recompute_mask
        if recompute_mask and mask is None:
            raise ValueError("recompute_mask needs a mask buffer")
        self.w_color, self.w_depth = w_color, w_depth
        # the unstable index is fixed for the life of this step object (one window)
        self.rank, self.ids, self.nu = api.unstable_rank(ctx, g.unstable)
        # the optimiser owns compact copies of the unstable parameters, and the renderer reads
        # the unstable Gaussians from them (the u_* overrides); the full arrays are brought up
        # to date by write_back(), or after every step with scatter_every_step
        self.u = api.gather_unstable(self.ids, g)
        self.full = g
        self.scatter_every_step = scatter_every_step
        self.g = dataclasses.replace(g, rank_map=self.rank, unstable_ids=self.ids, n_unstable=self.nu,
                                     u_means=self.u[0], u_scales=self.u[1], u_quats=self.u[2],
                                     u_opacity=self.u[3], u_colors=self.u[4])
        self.state = RasterState(ctx, self.g, self.cams, mask, settings)
        dev = g.means.device
        C = g.color_width
        self.target_color, self.target_depth = target_color, target_depth
        self.frame = frame
        self.loss = torch.zeros(3, device=dev)
        self.grads = [torch.zeros_like(t) for t in self.u]
        self.m = torch.zeros(self.nu * (11 + C), device=dev)
        self.v = torch.zeros(self.nu * (11 + C), device=dev)
        self.step_counter = torch.zeros(2, dtype=torch.int32, device=dev)  # completed steps, scratch
        # transparent-Gaussian regulariser (L_reg of Eq. 8): the unstable Gaussians' values
        # when they were added, given as full arrays (means0, scales0, quats0)
        self.w_reg = w_reg
        self.u0 = None
        self.loss_reg = torch.zeros(1, device=dev)
        if initial is not None:
            m0, s0, q0 = initial
            g0 = Gaussians(m0, s0, q0, g.opacity, g.colors, g.unstable, sh_degree=g.sh_degree)
            self.u0 = api.gather_unstable(self.ids, g0)[:3]
        self.graph = None
        self.window = window
        if window:
            api.window_begin(ctx, self.cams, self.g, settings)
        # with a MapState, every iteration raises the confidence counts of the Gaussians
        # whose colour it updated, and finish() fuses the window's result (Eq. 9)
        self.map_state = map_state
        if map_state is not None:
            map_state.window_start()

    def _body(self, stream=None):
        s = self.state
        if self.frame is not None and not self.recompute_mask and self.g.sh_degree == 0 and self.g.channels == 3:
            # the sensor frame decoded by the forward call itself (its tile-mask pass overlaps
            # the decode), the L1 loss fused in
            api.render_forward_l1_frame(self.ctx, self.cams, self.g, self.mask, self.settings, self.frame[0],
                                        self.frame[1], self.frame[2], self.target_color, self.target_depth,
                                        self.w_color, self.w_depth, s.color, s.depth, s.alpha, self.loss, None,
                                        stream)
            return self._backward_adam(stream)
        if self.frame is not None:
            api.decode_rgbd(self.frame[0], self.frame[1], self.frame[2], self.target_color, self.target_depth, stream)
        if self.recompute_mask:
            # mask, forward and L1 loss in one pass sharing a single projection
            api.render_forward_masked(self.ctx, self.cams, self.g, self.settings, self.mask, s.color, s.depth,
                                      s.alpha, self.target_color, self.target_depth, self.w_color, self.w_depth,
                                      self.loss, None, stream)
        else:
            # forward with the L1 loss fused in (no gradient images)
            api.render_forward_l1(self.ctx, self.cams, self.g, self.mask, self.settings, self.target_color,
                                  self.target_depth, self.w_color, self.w_depth, s.color, s.depth, s.alpha,
                                  self.loss, None, stream)
        return self._backward_adam(stream)

    def _backward_adam(self, stream=None):
        api.render_backward_l1(self.ctx, *self.grads, stream=stream)
        if self.map_state is not None:
            api.confidence_update(self.ids, self.grads[4], self.map_state.eta, stream)
        if self.u0 is not None:
            api.transparent_reg(self.ctx, self.u, self.u0, self.grads, self.loss_reg, self.w_reg, stream=stream)
        # the kernel in front (projection backward, confidence update or regulariser) writes
        # gradients at most, so Adam's parameter and moment loads overlap it
        api.adam_step_counted(self.u, self.grads, self.m, self.v, self.step_counter, self.adam, stream,
                              after_gradients=True)
        if self.scatter_every_step:
            api.scatter_unstable(self.ids, self.u, self.full, stream)
        return self.loss

    def step(self, stream=None):
        """Mask (optional), forward, L1 loss, backward and Adam; returns the device loss (L, Lc, Ld)."""
        if self.graph is not None:
            self.graph.replay()
            return self.loss
        return self._body(stream)

    def capture(self):
        """Record one iteration in a CUDA graph (run at least one eager step() first)."""
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            self._body()
        torch.cuda.synchronize()
        self.graph = graph
        return graph

    def capture_frames(self, frames: Sequence, uploads: Optional[Sequence] = None,
                       loss_host: Optional[Sequence[torch.Tensor]] = None, upload_streams: int = 4):
        """One CUDA graph per sensor-frame buffer set, for a frame loop: ``frames`` holds (rgb,
        depth) device tensors shaped like the step's frame (its depth scale is kept), and
        ``replay(k)`` runs the iteration on set k and returns set k's own loss buffer.

        With ``uploads`` (one pinned host (rgb, depth) pair per set), graph k also copies
        uploads[k] into frame set (k + 1) % len(frames) while it computes (each array in two
        halves over ``upload_streams`` side branches of the graph: one copy alone does not fill
        the host link), so replaying graph i % 2 for frame i moves frame i + 1 in during step
        i.  With ``loss_host`` (one pinned float[3] per set), graph k then copies its loss
        there.  A frame loop is then one launch per frame.  step() keeps its own graph, frame
        and loss buffer."""
        if self.frame is None:
            raise ValueError("capture_frames needs a step built with frame=")
        n = len(frames)
        torch.cuda.synchronize()
        own = (self.frame, self.loss)
        scale = self.frame[2]
        side = [torch.cuda.Stream() for _ in range(upload_streams)] if uploads is not None else []
        self.frame_graphs, self.frame_losses = [], []
        for k, (rgb, dep) in enumerate(frames):
            if rgb.shape != own[0][0].shape or dep.shape != own[0][1].shape:
                raise ValueError("each frame set must match the step's frame shapes")
            self.frame = (rgb, dep, scale)
            self.loss = torch.zeros(3, device=self.loss.device)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                cur = torch.cuda.current_stream()
                if uploads is not None:
                    fork = torch.cuda.Event()
                    fork.record(cur)
                    pieces = []
                    for d, h in zip(frames[(k + 1) % n], uploads[k]):
                        db, hb = d.reshape(-1).view(torch.uint8), h.reshape(-1).view(torch.uint8)
                        half = (db.numel() // 2) & ~15
                        pieces += [(db[:half], hb[:half]), (db[half:], hb[half:])] if half else [(db, hb)]
                    for st in side:
                        st.wait_event(fork)
                    for j, (d, h) in enumerate(pieces):
                        with torch.cuda.stream(side[j % len(side)]):
                            d.copy_(h, non_blocking=True)
                self._body()
                if loss_host is not None:
                    loss_host[k].copy_(self.loss, non_blocking=True)
                for st in side:  # join the upload branches
                    e = torch.cuda.Event()
                    e.record(st)
                    cur.wait_event(e)
            self.frame_graphs.append(graph)
            self.frame_losses.append(self.loss)
        self.frame, self.loss = own
        torch.cuda.synchronize()

    def replay(self, k: int):
        """One iteration on frame set k of capture_frames; returns that set's device loss."""
        self.frame_graphs[k].replay()
        return self.frame_losses[k]

    def write_back(self, stream=None):
        """Scatter the optimised compact parameters into the full arrays."""
        api.scatter_unstable(self.ids, self.u, self.full, stream)

    def finish(self, stream=None):
        """End of the window: with a MapState, fuse the optimised Gaussians into the map with
        the weights of Eq. 9; without one, write them back as they are."""
        if self.map_state is not None:
            api.fuse_window(self.ids, self.map_state.eta_start, self.map_state.eta, self.u, self.full, stream)
        else:
            self.write_back(stream)
