"""One keyframe batch split by frame over several GPUs: one process per GPU, each with its own
context and its own replica of the Gaussians.

The masked iteration over F keyframes (Section 3.2; the batch of one call) is a sum over
frames of per-pixel terms, but the means of Eq. 7 run over every masked pixel of the whole
batch.  So each rank

1. renders its own frames with the fused L1 loss and reports its pixel counts and L1 sums
   (``rtg_loss_counts``);
2. the ranks sum those four numbers (one all-reduce);
3. each rank sets the batch's gradient scales (``rtg_set_loss_scales``) and runs its
   backward, which gives its share of the batch gradient, in the compact unstable order;
4. the ranks sum the compact gradient arrays, N_u x (11 + C) floats (one all-reduce);
5. every rank applies the same Adam step, so the replicas stay equal.

The sum of the shares is the gradient of the batched call over all F frames, up to the
order of floating-point additions.  The collective is passed in (``reduce``), so the same
object serves torch.distributed ranks (NCCL or gloo) and a caller that runs the ranks' shares
itself.
"""

from __future__ import annotations

from typing import Callable, Optional, Sequence

import torch

from . import api
from .api import AdamSettings, Context, Gaussians, RenderSettings
from .optim import MaskedStep


def frame_shard(F: int, rank: int, world: int) -> slice:
    """The frames of rank `rank` among `world`: contiguous, in order, sizes differing by at
    most one (the first F mod world ranks take one more)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError(f"rank {rank} of {world}")
    if F < world:
        raise ValueError(f"{F} frames cannot be split over {world} ranks")
    base, extra = divmod(F, world)
    start = rank * base + min(rank, extra)
    return slice(start, start + base + (1 if rank < extra else 0))


def allreduce_sum(t: torch.Tensor, group=None) -> torch.Tensor:
    """In-place sum over the ranks of `group` (nothing to do without a process group)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def flat_gradients(nu: int, C: int, device) -> tuple:
    """One flat float32 buffer of N_u (11 + C) values and its five views, (means [nu,3],
    scales [nu,3], quats [nu,4], opacity [nu], colours [nu,C]), so that one all-reduce sums
    every gradient group."""
    flat = torch.zeros(nu * (11 + C), device=device)
    sizes = (3, 3, 4, 1, C)
    views, o = [], 0
    for k in sizes:
        v = flat[o:o + nu * k]
        views.append(v.view(nu) if k == 1 else v.view(nu, k))
        o += nu * k
    return flat, views


class FrameShardedStep:
    """The masked iteration of a keyframe batch, this rank's share of it.

    cams, masks [F,H,W], target_color [F,C,H,W] and target_depth [F,H,W] describe the whole
    batch; the rank renders frames ``frame_shard(F, rank, world)``.  ``reduce(t)`` must sum
    `t` in place over the ranks (default: torch.distributed all-reduce on `group`).
    ``step()`` runs the five stages above; ``forward()``, ``backward()`` and ``apply()`` are
    stages 1, 3 and 5, for a caller that performs the sums itself.  ``frame`` optionally gives
    the batch's sensor frames (rgb [F,H,W,3] uint8, depth [F,H,W] uint16, depth_scale), each
    rank decoding its own.
    """

    def __init__(self, ctx: Context, g: Gaussians, cams: Sequence, masks: torch.Tensor,
                 target_color: torch.Tensor, target_depth: torch.Tensor,
                 settings: RenderSettings = RenderSettings(), adam: AdamSettings = AdamSettings(),
                 w_color: float = 1.0, w_depth: float = 1.0, rank: Optional[int] = None,
                 world: Optional[int] = None, group=None,
                 reduce: Optional[Callable[[torch.Tensor], torch.Tensor]] = None, frame=None):
        import torch.distributed as dist
        if rank is None or world is None:
            on = dist.is_available() and dist.is_initialized()
            rank = dist.get_rank(group) if on else 0
            world = dist.get_world_size(group) if on else 1
        self.rank, self.world = rank, world
        self.frames = frame_shard(len(cams), rank, world)
        sl = self.frames
        self.reduce = reduce if reduce is not None else (lambda t: allreduce_sum(t, group))
        local_frame = None
        if frame is not None:
            local_frame = (frame[0][sl], frame[1][sl], frame[2])
        self.inner = MaskedStep(ctx, g, list(cams)[sl], masks[sl], target_color[sl], target_depth[sl], settings,
                                adam, w_color, w_depth, recompute_mask=False, frame=local_frame)
        self.ctx, self.w_color, self.w_depth = ctx, w_color, w_depth
        dev = target_color.device
        self.flat, self.grads = flat_gradients(self.inner.nu, g.color_width, dev)
        self.counts = torch.zeros(4, dtype=torch.float64, device=dev)
        self.loss = torch.zeros(3, device=dev)  # the batch's (L, L_color, L_depth)

    def forward(self, stream=None):
        """Stage 1: this rank's frames with the fused L1 loss, and its counts and sums."""
        s = self.inner
        if s.frame is not None:
            api.decode_rgbd(s.frame[0], s.frame[1], s.frame[2], s.target_color, s.target_depth, stream)
        st = s.state
        api.render_forward_l1(self.ctx, s.cams, s.g, s.mask, s.settings, s.target_color, s.target_depth,
                              self.w_color, self.w_depth, st.color, st.depth, st.alpha, s.loss, None, stream)
        api.loss_counts(self.ctx, self.counts, stream)
        return self.counts

    def backward(self, stream=None):
        """Stage 3 (after self.counts holds the batch totals): this rank's share of the batch
        gradient in self.flat."""
        api.set_loss_scales(self.ctx, self.counts, self.w_color, self.w_depth, self.loss, stream)
        api.render_backward_l1(self.ctx, *self.grads, stream=stream)
        return self.flat

    def apply(self, stream=None):
        """Stage 5 (after self.flat holds the batch gradient): the replicated Adam step."""
        s = self.inner
        api.adam_step_counted(s.u, self.grads, s.m, s.v, s.step_counter, s.adam, stream)

    def step(self):
        """One iteration of the batch; returns the batch's device loss (L, L_color, L_depth)."""
        self.forward()
        self.reduce(self.counts)
        self.backward()
        self.reduce(self.flat)
        self.apply()
        return self.loss

    @property
    def params(self):
        """The compact unstable parameters this rank optimises (equal on every rank)."""
        return self.inner.u
