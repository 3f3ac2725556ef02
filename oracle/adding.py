"""Gaussian adding (paper Section 3.2, "Gaussians adding", Eq. 6): TEST INFRASTRUCTURE
ONLY, like the rest of this package.

From a full-frame render of the existing map (colour C_hat, transmission T_hat, depth
D_hat, index map I_hat) and the input frame (colour C, depth D):
  M_s = {T_hat > delta_T or |D_hat - D| > delta_d}           new geometry
  M_c = {|C_hat - C| > delta_c and not in M_s}               colour correction
5% of the pixels of M_s and M_c are drawn uniformly.  A drawn M_s pixel gets an opaque
Gaussian (opacity 0.99).  A drawn M_c pixel looks up the Gaussian of its depth hit in the
index map: if that Gaussian is unstable nothing is added, otherwise a transparent Gaussian
(opacity 0.1).  A new Gaussian sits at the pixel's back-projected input depth with the
pixel's input colour.

Readings (the paragraph leaves them open):
  - T_hat is 1 - alpha of the render; each mask decision is taken in float32 on the
    render's and the frame's float32 values, as the GPU takes it;
  - D_hat = -1 where the render has no depth hit, so such a pixel with valid input depth
    is in M_s; pixels with invalid input depth (D <= 0) are in neither mask (there is no
    position for a new Gaussian);
  - |C_hat - C| is the mean absolute difference over the C channels (as in the colour
    loss), tested as sum_c |C_hat_c - C_c| > C * delta_c, the sum in channel order;
  - the 5% uniform sample: every pixel of M_s or M_c is kept independently with
    probability 5%, from a counter-based draw: SplitMix64 (Steele, Lea and Flood, 2014)
    seeded with `seed`, output number f * H * W + p for pixel p of frame f; the top 24
    bits u are compared with floor(rate * 2^24): kept iff u is below it;
  - an M_c pixel whose index map holds no Gaussian (-1) adds nothing;
  - the position is V(u) = R (D(u) K^-1 (x, y, 1)) + t with the camera-to-world pose (R, t)
    (the vertex map of the input pre-processing, for this pixel only).
Normals, scales and rotations of the new Gaussians (Supplement A) are not computed here.
"""

from __future__ import annotations

import dataclasses

import numpy as np

_M64 = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15


@dataclasses.dataclass(frozen=True)
class AddParams:
    delta_T: float = 0.5
    delta_d: float = 0.1
    delta_c: float = 0.1
    sample_rate: float = 0.05
    opacity_opaque: float = 0.99
    opacity_transparent: float = 0.1
    seed: int = 0


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """Output number `counters` (0-based) of the SplitMix64 stream seeded with `seed`: the
    state advances by the golden-ratio increment before each output, which is mixed by two
    xor-shift-multiply rounds and a final xor-shift."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _M64) + (c + np.uint64(1)) * np.uint64(_GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def sample_threshold(rate: float) -> int:
    """floor(rate * 2^24) in double precision: a pixel is drawn iff its 24-bit draw is below."""
    return int(np.floor(float(rate) * float(1 << 24)))


def sample_keep(seed: int, F: int, H: int, W: int, rate: float) -> np.ndarray:
    """[F, H, W] bool: the uniform draw of each pixel (before any mask)."""
    u = splitmix64(seed, np.arange(F * H * W, dtype=np.uint64)) >> np.uint64(40)
    return (u < np.uint64(sample_threshold(rate))).reshape(F, H, W)


def adding_masks(render_color, render_alpha, render_depth, color, depth, p: AddParams = AddParams()):
    """(M_s, M_c), each [F, H, W] bool, from float32 maps: colours [F, C, H, W], the rest
    [F, H, W]."""
    rc = np.asarray(render_color, np.float32)
    ic = np.asarray(color, np.float32)
    alpha = np.asarray(render_alpha, np.float32)
    Dh = np.asarray(render_depth, np.float32)
    D = np.asarray(depth, np.float32)
    C = rc.shape[1]
    valid = D > np.float32(0)
    T_hat = np.float32(1) - alpha
    m_s = valid & ((T_hat > np.float32(p.delta_T)) | (np.abs(Dh - D) > np.float32(p.delta_d)))
    err = np.zeros(D.shape, np.float32)
    for c in range(C):
        err = (err + np.abs(rc[:, c] - ic[:, c])).astype(np.float32)
    m_c = valid & ~m_s & (err > np.float32(C) * np.float32(p.delta_c))
    return m_s, m_c


def add_candidates(cams, render_color, render_alpha, render_depth, index_map, color, depth, unstable,
                   p: AddParams = AddParams()):
    """The Gaussians to add, in (frame, pixel) order: dict of pixel (f*H*W + y*W + x), kind
    (1 opaque, 2 transparent), position [M, 3] (FP64), colour [M, C], opacity [M]."""
    m_s, m_c = adding_masks(render_color, render_alpha, render_depth, color, depth, p)
    F, H, W = m_s.shape
    keep = sample_keep(p.seed, F, H, W, p.sample_rate)
    idx = np.asarray(index_map, np.int64)
    flags = np.asarray(unstable)
    n = flags.shape[0]
    hit = (idx >= 0) & (idx < n)
    stable_hit = hit & (flags[np.clip(idx, 0, max(n - 1, 0))] == 0) if n else np.zeros_like(hit)
    kind = np.zeros((F, H, W), np.uint8)
    kind[keep & m_c & stable_hit] = 2
    kind[keep & m_s] = 1
    flat = np.flatnonzero(kind.reshape(-1))
    f, rem = np.divmod(flat, H * W)
    y, x = np.divmod(rem, W)
    D = np.asarray(depth, np.float64).reshape(-1)[flat]
    pos = np.zeros((len(flat), 3))
    for i, cam in enumerate(cams):
        sel = f == i
        if not sel.any():
            continue
        v = np.stack([(x[sel] - cam.cx) / cam.fx, (y[sel] - cam.cy) / cam.fy, np.ones(sel.sum())], 1) * D[sel, None]
        pos[sel] = v @ np.asarray(cam.R, np.float64).reshape(3, 3).T + np.asarray(cam.t, np.float64).reshape(3)
    col = np.asarray(color, np.float32)
    C = col.shape[1]
    colors = col.transpose(0, 2, 3, 1).reshape(-1, C)[flat]
    k = kind.reshape(-1)[flat]
    opacity = np.where(k == 1, np.float32(p.opacity_opaque), np.float32(p.opacity_transparent)).astype(np.float32)
    return dict(pixel=flat.astype(np.int64), kind=k, position=pos, color=colors, opacity=opacity,
                m_s=m_s, m_c=m_c)
