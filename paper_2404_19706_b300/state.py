"""Fusion and state management of the map (Section 3.2: "Gaussian optimization" with Eq. 9,
and "State management") on top of the C ABI.

``MapState`` owns the per-Gaussian counters: the confidence count eta (raised whenever an
optimisation iteration updates a Gaussian's colour), the error count e and the frame of
creation t0.  It fuses the result of an optimisation window into the map (Eq. 9), counts the
errors of a render of the optimised map against the input frames, converts Gaussians
between stable and unstable, and removes those that stayed unstable too long.
"""

from __future__ import annotations

from typing import Optional, Sequence

import torch

from . import api
from .api import Context, Gaussians, MapArrays, StateSettings


class MapState:
    def __init__(self, ctx: Context, g: Gaussians, t0: Optional[torch.Tensor] = None,
                 settings: StateSettings = StateSettings()):
        self.ctx, self.g, self.settings = ctx, g, settings
        n, dev = g.n, g.means.device
        self.eta = torch.zeros(n, dtype=torch.int32, device=dev)
        self.err = torch.zeros(n, dtype=torch.int32, device=dev)
        self.t0 = t0 if t0 is not None else torch.zeros(n, dtype=torch.int32, device=dev)
        self.eta_start = torch.zeros_like(self.eta)
        self.remove = torch.zeros(n, dtype=torch.uint8, device=dev)
        self.count = torch.zeros(1, dtype=torch.int64, device=dev)

    def arrays(self) -> MapArrays:
        g = self.g
        return MapArrays(g.means, g.scales, g.quats, g.opacity, g.colors, g.unstable, self.eta, self.err, self.t0)

    def window_start(self, stream=None):
        """Remember the confidence counts at the start of an optimisation window."""
        self.eta_start.copy_(self.eta)

    def record_iteration(self, ids: torch.Tensor, g_colors: torch.Tensor, stream=None):
        """After an iteration: eta += 1 for the optimised Gaussians whose colour moved."""
        api.confidence_update(ids, g_colors, self.eta, stream)

    def fuse(self, ids: torch.Tensor, compact: Sequence[torch.Tensor], stream=None):
        """End of the window: Eq. 9 blend of the optimised compact rows into the map."""
        api.fuse_window(ids, self.eta_start, self.eta, compact, self.g, stream)

    def count_errors(self, render_color, render_depth, index_map, color, depth, stream=None):
        """Error counts from a full-frame render of the optimised map and the input frames."""
        api.error_count(self.ctx, render_color, render_depth, index_map, color, depth, self.g.unstable,
                        self.settings, self.err, stream)

    def update(self, frame: int, stream=None) -> torch.Tensor:
        """Stable <-> unstable conversion at frame `frame`; returns the removal flags."""
        api.update_states(frame, self.t0, self.settings, self.g.unstable, self.eta, self.err, self.remove, stream)
        return self.remove

    def prune(self, stream=None) -> int:
        """Drop the Gaussians flagged by update(), keeping the order of the others.  Allocates
        the compacted arrays and synchronises to read their number."""
        src = self.arrays()
        dst = MapArrays.empty_like(src)
        api.compact_gaussians(self.ctx, self.remove, src, dst, self.count, stream)
        n = int(self.count.item())
        g = Gaussians(dst.means[:n], dst.scales[:n], dst.quats[:n], dst.opacity[:n], dst.colors[:n],
                      dst.unstable[:n])
        self.g = g
        self.eta, self.err, self.t0 = dst.eta[:n], dst.err[:n], dst.t0[:n]
        self.eta_start = torch.zeros_like(self.eta)
        self.remove = torch.zeros(n, dtype=torch.uint8, device=self.eta.device)
        return n
