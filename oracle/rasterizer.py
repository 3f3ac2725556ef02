"""FP64 brute-force oracle of the depth-split, masked Gaussian rasterizer.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg.  It is a plain per-pixel restatement of the paper's equations and
shares no code with the CUDA path.

What it computes, per pixel u (paper, Section 3.1):
  1. every Gaussian is projected (EWA footprint, Eq. 2) in FP64;
  2. the Gaussians whose footprint value f_i(u) reaches alpha_min are taken front to
     back, ordered by camera-frame depth and then by index;
  3. colour is alpha-composited (Eq. 1) with transmission (Eq. 3), stopping before a
     fragment that would push the transmission below t_eps;
  4. depth comes from the first processed fragment with f > delta_alpha, through the
     ray / disc-plane intersection (Eq. 4) and the three cases of Eq. 5 (-1 if no hit,
     the intersection if the ray and the disc normal are within 60 degrees, else the
     centre's camera depth);
  5. the index map holds that Gaussian's index (Section 3.1, the by-products of the
     depth rendering).

Readings of points the paper leaves open (all carried by ``Settings``):
  * f_i(u) = min(f_max, alpha_i * exp(-0.5 d^T Sigma_2D^-1 d)), d = u - mu, with a
    low-pass dilation Sigma_2D = J W Sigma W^T J^T + lowpass * I (the 3DGS convention
    Eq. 2 cites); a fragment contributes iff f >= alpha_min; no background colour.
  * the hit test of Section 3.1 (the opacity met along the ray above delta_alpha) uses
    that same f value.
  * the 60-degree limit on the angle of normal and ray (Section 3.1) is an angle between
    lines: the plane branch is taken iff |n.r| / |r| >= cos(60 deg) = 0.5 (equality
    included).
  * the disc normal is the axis of the smallest scale, lowest index on ties
    (Section 3.1 takes the eigenvector of the smallest eigenvalue as the normal).
  * a Gaussian is culled if any parameter is not finite, if its camera depth is
    <= near_z, or if |X/Z| > guard_band * (W/2)/fx or |Y/Z| > guard_band * (H/2)/fy.
  * only processed fragments are depth candidates (colour and depth stop together).
"""

from __future__ import annotations

import dataclasses
import math
from typing import Dict, Optional, Sequence, Tuple

import numpy as np
import torch

DT = torch.float64
U32 = 2.0 ** -24  # unit roundoff of IEEE binary32 (the GPU path's arithmetic)


@dataclasses.dataclass(frozen=True)
class Settings:
    """Rendering constants.  Defaults: Section 3.1 (delta_alpha = e^-0.5, the 60 degree
    rule), Supplement B (50% tile rule), and the 3DGS conventions the paper builds on
    for the values it does not state (alpha_min, f_max, t_eps, low-pass, near plane,
    guard band)."""
    near_z: float = 0.2
    alpha_min: float = 1.0 / 255.0
    f_max: float = 0.99
    t_eps: float = 1e-4
    delta_alpha: float = math.exp(-0.5)
    cos_max_angle: float = 0.5
    lowpass: float = 0.3
    guard_band: float = 1.3
    tile_discard_frac: float = 0.5
    mask_tile: int = 16


# ----------------------------------------------------------------------------- geometry

def rotation_from_quaternion(q: torch.Tensor) -> torch.Tensor:
    """R(q) for q = (w, x, y, z), normalised first (Section 3.1: Sigma from s and q)."""
    q = q / torch.linalg.vector_norm(q, dim=-1, keepdim=True)
    w, x, y, z = q.unbind(-1)
    rows = [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
            2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
            2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]
    return torch.stack(rows, -1).reshape(q.shape[:-1] + (3, 3))


def _cam_tensors(cam) -> Tuple[torch.Tensor, torch.Tensor]:
    return (torch.as_tensor(np.asarray(cam.R, dtype=np.float64), dtype=DT),
            torch.as_tensor(np.asarray(cam.t, dtype=np.float64), dtype=DT))


@dataclasses.dataclass
class Projection:
    ids: torch.Tensor        # [V] original index of each candidate, ascending
    visible: torch.Tensor    # [V] bool, passes the culling rules
    marginal: torch.Tensor   # [V] bool, a culling decision is within rounding of flipping
    mu: torch.Tensor         # [V,2] pixel-space centre
    cov2d: torch.Tensor      # [V,3] (a, b, c) of Sigma_2D
    conic: torch.Tensor      # [V,3] (a', b', c') of Sigma_2D^-1
    opacity: torch.Tensor    # [V]
    Z: torch.Tensor          # [V] camera-frame depth of the centre
    means: torch.Tensor      # [V,3] world position
    normal: torch.Tensor     # [V,3] world-space disc normal (unit)
    colors: torch.Tensor     # [V,C]


def project(means: torch.Tensor, scales: torch.Tensor, quats: torch.Tensor, opacity: torch.Tensor,
            colors: torch.Tensor, cam, st: Settings) -> Projection:
    """EWA projection of every Gaussian into the camera (Section 3.1, Eq. 2).

    The pose T_g = [R_g | t_g] maps camera to world (the pixel-ray definition), so a
    world point p has camera coordinates R_g^T (p - t_g).  J is the Jacobian of the
    perspective map (X, Y, Z) -> (fx X/Z + cx, fy Y/Z + cy) at the centre.
    """
    Rg, tg = _cam_tensors(cam)
    fx, fy, cx, cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    if colors.ndim == 3:  # SH coefficients [n, K, 3]: the colour seen from this camera
        from .sh import sh_colors
        colors = sh_colors(colors, means, tg)
    with torch.no_grad():
        finite = (torch.isfinite(means).all(1) & torch.isfinite(scales).all(1) & torch.isfinite(quats).all(1)
                  & torch.isfinite(opacity) & torch.isfinite(colors).all(1)
                  & (torch.linalg.vector_norm(quats, dim=1) > 0))
        pc0 = (torch.nan_to_num(means.detach()) - tg) @ Rg
        X0, Y0, Z0 = pc0.unbind(-1)
        lim_x = st.guard_band * (cam.width / 2.0) / fx
        lim_y = st.guard_band * (cam.height / 2.0) / fy
        Zs = torch.where(Z0 > 0, Z0, torch.ones_like(Z0))
        rx, ry = (X0 / Zs).abs(), (Y0 / Zs).abs()
        visible = finite & (Z0 > st.near_z) & (rx <= lim_x) & (ry <= lim_y)
        m = 1e-6
        marginal = finite & (Z0 > st.near_z * (1 - m)) & (rx <= lim_x * (1 + m)) & (ry <= lim_y * (1 + m)) & (
            ((Z0 - st.near_z).abs() <= m * st.near_z) | ((rx - lim_x).abs() <= m * lim_x)
            | ((ry - lim_y).abs() <= m * lim_y))
        cand = visible | marginal
        ids = torch.nonzero(cand).flatten()
    p = means[ids]
    s = scales[ids]
    R = rotation_from_quaternion(quats[ids])
    Sigma = R @ torch.diag_embed(s * s) @ R.transpose(1, 2)
    pc = (p - tg) @ Rg
    X, Y, Z = pc.unbind(-1)
    zero = torch.zeros_like(Z)
    J = torch.stack([torch.stack([fx / Z, zero, -fx * X / (Z * Z)], -1),
                     torch.stack([zero, fy / Z, -fy * Y / (Z * Z)], -1)], 1)  # [V,2,3]
    W = Rg.T
    cov = J @ W @ Sigma @ W.T @ J.transpose(1, 2)
    a = cov[:, 0, 0] + st.lowpass
    b = cov[:, 0, 1]
    c = cov[:, 1, 1] + st.lowpass
    det = a * c - b * b
    conic = torch.stack([c / det, -b / det, a / det], -1)  # inverse of a symmetric 2x2
    mu = torch.stack([fx * X / Z + cx, fy * Y / Z + cy], -1)
    k = torch.argmin(s.detach(), dim=1)  # smallest axis, first index on ties
    normal = torch.gather(R, 2, k.view(-1, 1, 1).expand(-1, 3, 1)).squeeze(2)
    return Projection(ids=ids, visible=visible[ids], marginal=marginal[ids], mu=mu,
                      cov2d=torch.stack([a, b, c], -1), conic=conic, opacity=opacity[ids], Z=Z,
                      means=p, normal=normal, colors=colors[ids])


# ----------------------------------------------------------------------------- rendering

@dataclasses.dataclass
class RenderResult:
    pixels: torch.Tensor      # [P,2] (x, y)
    color: torch.Tensor       # [P,C]
    depth: torch.Tensor       # [P]
    alpha: torch.Tensor       # [P] 1 - final transmission
    index: torch.Tensor       # [P] index of the depth-hit Gaussian, -1 if none
    n_proc: torch.Tensor      # [P] number of processed (composited) fragments
    borderline: torch.Tensor  # [P] a discrete decision is within FP32 rounding of flipping
    grad_borderline: torch.Tensor  # [P] borderline, or a clamp decision near its switch


def _sorted_projection(pr: Projection) -> Projection:
    """Front-to-back order: camera depth, then index (ids are ascending, sort is stable)."""
    order = torch.sort(pr.Z.detach(), stable=True).indices
    return Projection(**{f.name: getattr(pr, f.name)[order] for f in dataclasses.fields(Projection)})


def _composite(u: torch.Tensor, pr: Projection, cam, st: Settings, need_borderline: bool):
    """Eq. 1-5 for a chunk of pixels u [p,2] against the sorted candidates of ``pr``."""
    Rg, tg = _cam_tensors(cam)
    fx, fy, cx, cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    p_n = u.shape[0]
    if pr.ids.numel() == 0:  # nothing in front of the camera: background everywhere
        C = pr.colors.shape[1]
        zf = torch.zeros(p_n, dtype=DT)
        out = dict(color=torch.zeros(p_n, C, dtype=DT), depth=torch.full((p_n,), -1.0, dtype=DT), alpha=zf,
                   index=torch.full((p_n,), -1, dtype=torch.long), n_proc=torch.zeros(p_n, dtype=torch.long),
                   processed=torch.zeros(p_n, 0, dtype=torch.bool),
                   hit_first=torch.full((p_n,), -1, dtype=torch.long), plane=torch.zeros(p_n, dtype=torch.bool))
        if need_borderline:
            out.update(borderline=torch.zeros(p_n, dtype=torch.bool), grad_borderline=torch.zeros(p_n, dtype=torch.bool))
        return out
    d = u[:, None, :] - pr.mu[None, :, :]
    dx, dy = d[..., 0], d[..., 1]
    ca, cb, cc = pr.conic[:, 0], pr.conic[:, 1], pr.conic[:, 2]
    power = ca * dx * dx + 2 * cb * dx * dy + cc * dy * dy       # Eq. 2 exponent, times -2
    g = torch.exp(-0.5 * power)
    f = torch.clamp(pr.opacity * g, max=st.f_max)                # f_i(u), opacity-clamped
    contrib = (f >= st.alpha_min) & pr.visible[None, :]
    fe = torch.where(contrib, f, torch.zeros_like(f))
    keep = 1 - fe
    T_after = torch.cumprod(keep, dim=1)                          # Eq. 3, running product
    T_before = torch.cat([torch.ones_like(T_after[:, :1]), T_after[:, :-1]], 1)
    processed = contrib & (T_after >= st.t_eps)                   # early stop, before the fragment
    w = torch.where(processed, fe * T_before, torch.zeros_like(fe))
    color = w @ pr.colors                                         # Eq. 1
    T_final = torch.where(processed, keep, torch.ones_like(keep)).prod(1)
    hit = processed & (f > st.delta_alpha)                        # first opaque hit
    has_hit = hit.any(1)
    first = torch.argmax(hit.to(torch.int8), dim=1)
    # Eq. 4 in world coordinates: ray r(theta) = R_g K^-1 u' theta + t_g
    ut = torch.stack([(u[:, 0] - cx) / fx, (u[:, 1] - cy) / fy, torch.ones_like(u[:, 0])], 1)
    ray = ut @ Rg.T
    p_h, n_h, Z_h = pr.means[first], pr.normal[first], pr.Z[first]
    den = (ray * n_h).sum(1)
    cosang = den.abs() / torch.linalg.vector_norm(ray, dim=1)
    plane = cosang >= st.cos_max_angle
    theta = ((p_h - tg) * n_h).sum(1) / torch.where(plane, den, torch.ones_like(den))
    p_int = ray * theta[:, None] + tg
    z_int = ((p_int - tg) @ Rg)[:, 2]                             # (T_g^-1 p)_z, Eq. 5
    depth = torch.where(plane, z_int, Z_h)
    depth = torch.where(has_hit, depth, torch.full_like(depth, -1.0))
    index = torch.where(has_hit, pr.ids[first], torch.full_like(first, -1))
    n_proc = processed.sum(1)
    out = dict(color=color, depth=depth, alpha=1 - T_final, index=index, n_proc=n_proc,
               processed=processed, hit_first=torch.where(has_hit, first, torch.full_like(first, -1)),
               plane=plane & has_hit)
    if not need_borderline:
        return out
    with torch.no_grad():
        out.update(_borderline(dx, dy, power, f, fe, contrib, processed, T_before, T_after, hit, has_hit,
                               cosang, pr, st))
    return out


def _borderline(dx, dy, power, f, fe, contrib, processed, T_before, T_after, hit, has_hit, cosang,
                pr: Projection, st: Settings) -> Dict[str, torch.Tensor]:
    """Flag pixels where a discrete decision lies within the FP32 error of the GPU path.

    The power error bound is 64 u (1 + p)(1 + sqrt(kappa)) + 32 u, with u the binary32
    unit roundoff and kappa = a c / det of Sigma_2D (its correlation conditioning).
    """
    a, b, c = pr.cov2d[:, 0], pr.cov2d[:, 1], pr.cov2d[:, 2]
    kappa = (a * c / (a * c - b * b)).clamp(min=1.0)
    dp = 64 * U32 * (1 + power.abs()) * (1 + kappa.sqrt())[None, :] + 32 * U32
    reached = T_before >= st.t_eps
    alpha = pr.opacity[None, :]
    thr_c = 2 * torch.log(torch.clamp(alpha / st.alpha_min, min=1e-300))
    b_contrib = reached & pr.visible[None, :] & ((power - thr_c).abs() <= dp)
    # hit decisions of processed fragments up to and including the first hit
    before_or_hit = (torch.cumsum(hit.to(torch.int32), 1) - hit.to(torch.int32)) == 0
    thr_h = 2 * torch.log(torch.clamp(alpha / st.delta_alpha, min=1e-300))
    b_hit = processed & before_or_hit & (alpha > st.delta_alpha) & ((power - thr_h).abs() <= dp)
    # early-stop decision: accumulated log-transmission error
    ratio = torch.where(processed, fe / (1 - fe), torch.zeros_like(fe))
    dlnT = torch.cumsum(ratio * (dp / 2 + 8 * U32), 1) + 16 * U32 * (1 + torch.cumsum(processed.to(DT), 1))
    stop_frag = contrib & ~processed & reached
    last_proc = processed & (torch.flip(torch.cumsum(torch.flip(processed.to(torch.int32), [1]), 1), [1]) == 1)
    lnT = torch.log(torch.clamp(T_after, min=1e-300))
    b_stop = (stop_frag | last_proc) & ((lnT - math.log(st.t_eps)).abs() <= dlnT)
    b_cos = has_hit & ((cosang - st.cos_max_angle).abs() <= 1e-5)
    b_cull = reached & pr.marginal[None, :] & (f >= st.alpha_min * (1 - 1e-3))
    border = b_contrib.any(1) | b_hit.any(1) | b_stop.any(1) | b_cos | b_cull.any(1)
    # depth ties: two reached contributors whose depths round to within 4u of each other
    Zs = pr.Z.detach()
    if Zs.numel() > 1:
        gap = Zs[1:] - Zs[:-1]
        tie = gap <= 4 * U32 * Zs[1:].abs()
        if bool(tie.any()):
            grp = torch.cat([torch.zeros(1, dtype=torch.long), torch.cumsum((~tie).to(torch.long), 0)])
            sizes = torch.bincount(grp)
            multi = torch.nonzero(sizes[grp] >= 2).flatten()
            rc = (contrib & reached)[:, multi].to(torch.int32)
            for gidx in torch.unique(grp[multi]).tolist():
                cols = grp[multi] == gidx
                border |= rc[:, cols].sum(1) >= 2
    # clamp switch of f at f_max: the value is continuous, its derivative is not
    b_clamp = processed & ((alpha * torch.exp(-0.5 * power) - st.f_max).abs() <= st.f_max * dp)
    return dict(borderline=border, grad_borderline=border | b_clamp.any(1))


def _params64(scene, requires_grad=False):
    out = []
    for name in ("means", "scales", "quats", "opacity", "colors"):
        arr = getattr(scene, name)
        t = arr.detach().to(DT) if isinstance(arr, torch.Tensor) else torch.as_tensor(
            np.asarray(arr, dtype=np.float64))
        out.append(t)
    return out


def _pixel_list(cam, pixels=None, mask=None) -> torch.Tensor:
    if pixels is not None:
        return torch.as_tensor(np.asarray(pixels), dtype=torch.long).reshape(-1, 2)
    if mask is None:
        mask = np.ones((cam.height, cam.width), dtype=bool)
    ys, xs = np.nonzero(np.asarray(mask).astype(bool))
    return torch.as_tensor(np.stack([xs, ys], 1), dtype=torch.long)


def render(scene, cam, st: Settings = Settings(), pixels=None, mask=None, need_borderline: bool = True,
           chunk_elems: int = 2_000_000) -> RenderResult:
    """Render the requested pixels (default: all, or the True entries of ``mask``)."""
    means, scales, quats, opacity, colors = _params64(scene)
    pix = _pixel_list(cam, pixels, mask)
    with torch.no_grad():
        pr = _sorted_projection(project(means, scales, quats, opacity, colors, cam, st))
        V = max(int(pr.ids.numel()), 1)
        step = max(1, chunk_elems // V)
        parts = []
        for s in range(0, pix.shape[0], step):
            u = pix[s:s + step].to(DT)
            parts.append(_composite(u, pr, cam, st, need_borderline))
    C = 3 if colors.ndim == 3 else colors.shape[1]
    if not parts:
        z = torch.zeros(0, dtype=DT)
        zb = torch.zeros(0, dtype=torch.bool)
        return RenderResult(pix, torch.zeros(0, C, dtype=DT), z, z, torch.zeros(0, dtype=torch.long),
                            torch.zeros(0, dtype=torch.long), zb, zb)

    def cat(k):
        return torch.cat([p[k] for p in parts], 0)
    border = cat("borderline") if need_borderline else torch.zeros(pix.shape[0], dtype=torch.bool)
    gborder = cat("grad_borderline") if need_borderline else border
    return RenderResult(pix, cat("color"), cat("depth"), cat("alpha"), cat("index"), cat("n_proc"),
                        border, gborder)


def render_image(scene, cam, st: Settings = Settings(), mask=None, fill_color: float = 0.0,
                 fill_depth: float = -1.0) -> Dict[str, np.ndarray]:
    """Full images [C,H,W] / [H,W]; pixels outside ``mask`` keep the fill values."""
    res = render(scene, cam, st, mask=mask)
    H, W = cam.height, cam.width
    C = res.color.shape[1]
    color = np.full((C, H, W), fill_color)
    depth = np.full((H, W), fill_depth)
    alpha = np.zeros((H, W))
    index = np.full((H, W), -1, dtype=np.int64)
    n_proc = np.zeros((H, W), dtype=np.int64)
    border = np.zeros((H, W), dtype=bool)
    gborder = np.zeros((H, W), dtype=bool)
    xs, ys = res.pixels[:, 0].numpy(), res.pixels[:, 1].numpy()
    color[:, ys, xs] = res.color.numpy().T
    depth[ys, xs] = res.depth.numpy()
    alpha[ys, xs] = res.alpha.numpy()
    index[ys, xs] = res.index.numpy()
    n_proc[ys, xs] = res.n_proc.numpy()
    border[ys, xs] = res.borderline.numpy()
    gborder[ys, xs] = res.grad_borderline.numpy()
    return dict(color=color, depth=depth, alpha=alpha, index=index, n_proc=n_proc, borderline=border,
                grad_borderline=gborder)


def decision_signature(scene, cam, st: Settings, pixels) -> Tuple[torch.Tensor, ...]:
    """Per-pixel discrete decisions: processed set, hit fragment, depth branch."""
    means, scales, quats, opacity, colors = _params64(scene)
    pix = _pixel_list(cam, pixels)
    with torch.no_grad():
        pr = _sorted_projection(project(means, scales, quats, opacity, colors, cam, st))
        out = _composite(pix.to(DT), pr, cam, st, need_borderline=False)
        ids = pr.ids
        proc_ids = [tuple(ids[row].tolist()) for row in out["processed"]]
        hit = torch.where(out["hit_first"] >= 0, ids[out["hit_first"].clamp(min=0)],
                          torch.full_like(out["hit_first"], -1))
    return (tuple(proc_ids), tuple(hit.tolist()), tuple(out["plane"].tolist()), tuple(pr.ids.tolist()))


# ----------------------------------------------------------------------------- losses

def l1_loss(color, depth, target_color, target_depth, w_c: float = 1.0, w_d: float = 1.0):
    """Eq. 7/8 over a set of rendered pixels (colour [P,C], depth [P]).

    L_color is the mean absolute error over pixels and channels; L_depth is the mean
    absolute error over the pixels with a rendered intersection (depth != -1) and a
    valid input depth (> 0), as Section 3.2 excludes pixels without intersection.
    Returns (L, L_color, L_depth, n_color_pixels, n_depth_pixels).
    """
    color = torch.as_tensor(color, dtype=DT)
    depth = torch.as_tensor(depth, dtype=DT)
    tc = torch.as_tensor(target_color, dtype=DT)
    td = torch.as_tensor(target_depth, dtype=DT)
    P = color.shape[0]
    C = color.shape[1] if color.ndim > 1 else 1
    Lc = (color - tc).abs().sum() / max(P * C, 1)
    valid = (depth.detach() != -1) & (td > 0)
    Pd = int(valid.sum())
    Ld = torch.where(valid, (depth - td).abs(), torch.zeros_like(depth)).sum() / max(Pd, 1)
    return w_c * Lc + w_d * Ld, Lc, Ld, P, Pd


def loss_and_grads(scene, cam, st: Settings, pixels, target_color, target_depth, w_c=1.0, w_d=1.0):
    """Analytic gradient of Eq. 8 (w_reg = 0) w.r.t. the unstable Gaussians' parameters.

    The forward is the same FP64 definition as ``render``; the derivative is taken by
    reverse-mode automatic differentiation of that definition.  Gradients are w.r.t.
    position, linear scale, raw (unnormalised) quaternion, opacity and colour, in
    compact order of ascending index over the unstable Gaussians.
    """
    means, scales, quats, opacity, colors = _params64(scene)
    unstable = torch.as_tensor(np.asarray(scene.unstable)).to(torch.bool)
    leaves = [t.clone().requires_grad_(True) for t in (means, scales, quats, opacity, colors)]
    full = [torch.where(unstable.view(-1, *([1] * (t.ndim - 1))), leaf, t)
            for leaf, t in zip(leaves, (means, scales, quats, opacity, colors))]
    pix = _pixel_list(cam, pixels)
    pr = _sorted_projection(project(*full, cam, st))
    out = _composite(pix.to(DT), pr, cam, st, need_borderline=True)
    tc = torch.as_tensor(np.asarray(target_color), dtype=DT)
    td = torch.as_tensor(np.asarray(target_depth), dtype=DT)
    L, Lc, Ld, P, Pd = l1_loss(out["color"], out["depth"], tc, td, w_c, w_d)
    if L.requires_grad:  # otherwise no unstable Gaussian reaches these pixels: zero gradients
        L.backward()
    sel = torch.nonzero(unstable).flatten()
    grads = {name: (leaf.grad if leaf.grad is not None else torch.zeros_like(leaf))[sel].numpy()
             for name, leaf in zip(("means", "scales", "quats", "opacity", "colors"), leaves)}
    return dict(loss=float(L.detach()), loss_color=float(Lc.detach()), loss_depth=float(Ld.detach()), n_pixels=P, n_depth=Pd,
                grads=grads, color=out["color"].detach().numpy(), depth=out["depth"].detach().numpy(),
                grad_borderline=out["grad_borderline"].numpy(), borderline=out["borderline"].numpy())


def _loss_only(scene_arrays, unstable, cam, st, pix, tc, td, w_c, w_d):
    means, scales, quats, opacity, colors = scene_arrays
    pr = _sorted_projection(project(means, scales, quats, opacity, colors, cam, st))
    out = _composite(pix.to(DT), pr, cam, st, need_borderline=False)
    L = l1_loss(out["color"], out["depth"], tc, td, w_c, w_d)[0]
    return float(L)


def finite_difference_grads(scene, cam, st: Settings, pixels, target_color, target_depth, which,
                            w_c=1.0, w_d=1.0, rel_h: float = 1e-6):
    """Central finite differences of the FP64 loss for the listed (name, gaussian, component).

    Returns (values, stable) where ``stable[k]`` is False if the +h or -h perturbation
    changed any pixel's decision signature (processed set, hit, depth branch), in
    which case the difference quotient does not approximate the derivative.
    """
    arrays = _params64(scene)
    names = ("means", "scales", "quats", "opacity", "colors")
    unstable = np.asarray(scene.unstable)
    pix = _pixel_list(cam, pixels)
    tc = torch.as_tensor(np.asarray(target_color), dtype=DT)
    td = torch.as_tensor(np.asarray(target_depth), dtype=DT)

    class _S:
        pass

    def sig_of(arrs):
        s = _S()
        for nme, a in zip(names, arrs):
            setattr(s, nme, a)
        s.unstable = unstable
        return decision_signature(s, cam, st, pix.numpy())

    base_sig = sig_of(arrays)
    vals, stable = [], []
    for (name, gi, comp) in which:
        k = names.index(name)
        x0 = float(arrays[k][gi].reshape(-1)[comp])
        h = rel_h * max(1.0, abs(x0))
        res = []
        ok = True
        for sgn in (1, -1):
            arrs = [a.clone() for a in arrays]
            flat = arrs[k][gi].reshape(-1)
            flat[comp] = x0 + sgn * h
            arrs[k][gi] = flat.reshape(arrs[k][gi].shape)
            res.append(_loss_only(arrs, unstable, cam, st, pix, tc, td, w_c, w_d))
            ok &= sig_of(arrs) == base_sig
        vals.append((res[0] - res[1]) / (2 * h))
        stable.append(ok)
    return np.array(vals), np.array(stable)


# ----------------------------------------------------------------------------- unstable mask

def unstable_mask(scene, cam, st: Settings = Settings(), chunk_elems: int = 2_000_000):
    """Supplement B: pixels with T_unstable < 1, then the 16x16 tile rule.

    T_unstable is rendered from the unstable Gaussians alone, so it is below one
    exactly where some visible unstable Gaussian has f >= alpha_min (the first
    contributing fragment is always processed).  A 16x16 tile is then cleared when
    fewer than ``tile_discard_frac`` of its in-image pixels are covered (0 = off).
    Returns (mask [H,W] bool, borderline [H,W] bool): a pixel is borderline when an
    unstable Gaussian's coverage decision there is within FP32 rounding; a whole tile
    is borderline when its kept/cleared decision could flip through such pixels.
    """
    means, scales, quats, opacity, colors = _params64(scene)
    uns = torch.as_tensor(np.asarray(scene.unstable)).to(torch.bool)
    sel = torch.nonzero(uns).flatten()
    H, W = cam.height, cam.width
    cover = np.zeros((H, W), dtype=bool)
    border = np.zeros((H, W), dtype=bool)
    with torch.no_grad():
        pr = project(means[sel], scales[sel], quats[sel], opacity[sel], colors[sel], cam, st)
        pix = _pixel_list(cam)
        V = max(int(pr.ids.numel()), 1)
        step = max(1, chunk_elems // V)
        a, b, c = pr.cov2d[:, 0], pr.cov2d[:, 1], pr.cov2d[:, 2]
        kappa = (a * c / (a * c - b * b)).clamp(min=1.0)
        thr = 2 * torch.log(torch.clamp(pr.opacity / st.alpha_min, min=1e-300))
        for s in range(0, pix.shape[0], step):
            u = pix[s:s + step].to(DT)
            d = u[:, None, :] - pr.mu[None]
            power = (pr.conic[:, 0] * d[..., 0] ** 2 + 2 * pr.conic[:, 1] * d[..., 0] * d[..., 1]
                     + pr.conic[:, 2] * d[..., 1] ** 2)
            f = torch.clamp(pr.opacity * torch.exp(-0.5 * power), max=st.f_max)
            cov_px = ((f >= st.alpha_min) & pr.visible[None]).any(1)
            dp = 64 * U32 * (1 + power.abs()) * (1 + kappa.sqrt())[None] + 32 * U32
            b_px = (((power - thr).abs() <= dp) & pr.visible[None]).any(1) | (
                pr.marginal[None] & (f >= st.alpha_min * (1 - 1e-3))).any(1)
            xs, ys = u[:, 0].long().numpy(), u[:, 1].long().numpy()
            cover[ys, xs] = cov_px.numpy()
            border[ys, xs] = b_px.numpy()
    mask, tile_border = apply_tile_rule(cover, border, st.tile_discard_frac, st.mask_tile)
    return mask, border | tile_border


def apply_tile_rule(cover: np.ndarray, border: np.ndarray, frac: float, tile: int = 16):
    """Supplement B: clear each tile x tile block in which fewer than ``frac`` of the
    in-image pixels need rendering (frac = 0 turns the rule off).

    A block is kept iff covered >= frac * in_image.  Returns (mask, tile_borderline):
    a block is borderline when its borderline pixels could move the count across the
    threshold.
    """
    cover = np.asarray(cover, dtype=bool)
    border = np.asarray(border, dtype=bool)
    H, W = cover.shape
    mask = cover.copy()
    tb = np.zeros_like(cover)
    if frac <= 0:
        return mask, tb
    for ty in range(0, H, tile):
        for tx in range(0, W, tile):
            blk = cover[ty:ty + tile, tx:tx + tile]
            n_in = blk.size
            n_cov = int(blk.sum())
            n_b = int(border[ty:ty + tile, tx:tx + tile].sum())
            if not n_cov >= frac * n_in:
                mask[ty:ty + tile, tx:tx + tile] = False
            lo, hi = n_cov - n_b, n_cov + n_b
            if (lo >= frac * n_in) != (hi >= frac * n_in):
                tb[ty:ty + tile, tx:tx + tile] = True
    return mask, tb
