"""Gaussian adding (Section 3.2, "Gaussians adding", Eq. 6) on top of the C ABI.

``AddingPass.run()`` renders the existing map over whole frames (colour, alpha, depth and
the index map of the depth hits) and then finds the pixels that get a new Gaussian: new
geometry (M_s) gets an opaque one, colour errors on geometry that is already right (M_c) a
transparent one unless the Gaussian there is still unstable; a uniform 5% of those pixels
are drawn.  The outputs are the new Gaussians' pixels, kinds, positions (back-projected
input depth), colours (input colour) and opacities, in (frame, pixel) order, on the device.
Two calls on preallocated buffers; nothing is allocated or synchronised.
"""

from __future__ import annotations

from typing import Sequence

import torch

from . import api
from .api import AddSettings, Context, Gaussians, RenderSettings


class AddingPass:
    def __init__(self, ctx: Context, width: int, height: int, channels: int = 3, max_frames: int = 1,
                 capacity: int = 1 << 16, settings: RenderSettings = RenderSettings(),
                 add: AddSettings = AddSettings(), device="cuda"):
        self.ctx, self.settings, self.add = ctx, settings, add
        F, C, H, W = max_frames, channels, height, width
        self.color = torch.zeros(F, C, H, W, device=device)
        self.alpha = torch.zeros(F, H, W, device=device)
        self.depth = torch.full((F, H, W), -1.0, device=device)
        self.index = torch.full((F, H, W), -1, dtype=torch.int32, device=device)
        self.count = torch.zeros(1, dtype=torch.int64, device=device)
        self.pixel = torch.zeros(capacity, dtype=torch.int32, device=device)
        self.kind = torch.zeros(capacity, dtype=torch.uint8, device=device)
        self.position = torch.zeros(capacity, 3, device=device)
        self.new_color = torch.zeros(capacity, C, device=device)
        self.opacity = torch.zeros(capacity, device=device)

    def run(self, cams: Sequence, g: Gaussians, color: torch.Tensor, depth: torch.Tensor, seed: int, stream=None):
        """Render the map on the keyframes ``cams`` and find the new Gaussians against the input
        colour [F,C,H,W] and depth [F,H,W]; returns the device count (may exceed capacity)."""
        cams = list(cams)
        F = len(cams)
        rc, ra, rd, ri = self.color[:F], self.alpha[:F], self.depth[:F], self.index[:F]
        api.render_forward(self.ctx, cams, g, None, self.settings, rc, rd, ra, ri, stream)
        api.add_candidates(self.ctx, cams, rc, ra, rd, ri, color, depth, g.unstable, self.add, seed, self.count,
                           self.pixel, self.kind, self.position, self.new_color, self.opacity, stream)
        return self.count
