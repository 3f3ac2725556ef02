"""Global keyframe optimisation (paper, "Keyframes and global optimization" paragraph of
Section 3): TEST INFRASTRUCTURE ONLY, like the rest of this package.

Whenever a keyframe is added, every Gaussian is optimised over the latest keyframe and
three randomly chosen earlier ones, with the loss of the masked step, but only on the
pixels with the top 40% colour errors of each keyframe; positions are not updated and the
other parameters use 0.1x the learning rates.  A new keyframe is taken when the rotation
relative to the last keyframe exceeds 30 degrees or the translation exceeds 0.3 m.

Readings (the paragraph does not fix them):
  - colour error of a pixel: the L1 distance over channels between render and input,
    summed in float32 in channel order (the rank by sum equals the rank by mean);
  - top 40%: the floor(0.4 * H * W) pixels of largest error in each keyframe, ties broken
    towards the lower pixel index (row-major);
  - rotation angle: the angle of R_last^T R_new; translation: |t_new - t_last|.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

from .adam import AdamHyper


def color_error(color: np.ndarray, target: np.ndarray) -> np.ndarray:
    """Per-pixel colour error [F, H, W] (float32) of colour/target [F, C, H, W] float32:
    |c_0 - t_0| + |c_1 - t_1| + ... accumulated left to right in float32."""
    color = np.asarray(color, dtype=np.float32)
    target = np.asarray(target, dtype=np.float32)
    err = np.zeros(color.shape[:1] + color.shape[2:], dtype=np.float32)
    for c in range(color.shape[1]):
        err = (err + np.abs(color[:, c] - target[:, c])).astype(np.float32)
    return err


def keep_count(frac: float, n_pixels: int) -> int:
    """Pixels kept per keyframe: floor(frac * n) in double precision."""
    return int(math.floor(frac * n_pixels))


def top_error_mask(color: np.ndarray, target: np.ndarray, frac: float = 0.4) -> np.ndarray:
    """[F, H, W] uint8 mask of each keyframe's floor(frac * H * W) largest colour errors;
    among equal errors the lower pixel index is taken first.  Errors are compared as their
    IEEE bit patterns (non-negative floats order like the patterns; NaN ranks highest)."""
    err = color_error(color, target)
    F, H, W = err.shape
    n = H * W
    k = keep_count(frac, n)
    out = np.zeros((F, n), dtype=np.uint8)
    for f in range(F):
        keys = err[f].reshape(-1).view(np.uint32).astype(np.int64)
        order = np.lexsort((np.arange(n), -keys))  # descending key, then ascending index
        out[f, order[:k]] = 1
    return out.reshape(F, H, W)


def global_hyper(base: AdamHyper = AdamHyper(), lr_factor: float = 0.1) -> AdamHyper:
    """Adam settings of the global optimisation: positions frozen, other rates x lr_factor."""
    return dataclasses.replace(base, lr_means=0.0, lr_scales=base.lr_scales * lr_factor,
                               lr_quats=base.lr_quats * lr_factor, lr_opacity=base.lr_opacity * lr_factor,
                               lr_colors=base.lr_colors * lr_factor, lr_colors_rest=base.lr_colors_rest * lr_factor)


def rotation_angle_deg(Ra: np.ndarray, Rb: np.ndarray) -> float:
    """Angle of the relative rotation Ra^T Rb, in degrees."""
    Rrel = np.asarray(Ra, dtype=np.float64).T @ np.asarray(Rb, dtype=np.float64)
    c = (np.trace(Rrel) - 1.0) / 2.0
    return math.degrees(math.acos(max(-1.0, min(1.0, c))))


def is_new_keyframe(R_last, t_last, R_new, t_new, angle_deg: float = 30.0, move_m: float = 0.3) -> bool:
    """The keyframe rule: relative rotation above angle_deg or translation above move_m."""
    if rotation_angle_deg(R_last, R_new) > angle_deg:
        return True
    return float(np.linalg.norm(np.asarray(t_new, np.float64) - np.asarray(t_last, np.float64))) > move_m
