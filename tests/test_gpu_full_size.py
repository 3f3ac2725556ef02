"""Parity at the workloads' full sizes, in the launch configuration the bench runs (window
open with its cached stable lists, the autotuner's typical tuning), on sampled masked
pixels that the FP64 oracle evaluates one by one.

The oracle gets, per sampled pixel set, the Gaussians that can reach those pixels: a
conservative bound on each footprint's screen radius, computed here in FP64 from the scale
and the perspective Jacobian, keeps every Gaussian whose alpha_min support could touch a
sampled pixel (dropping one would fail the comparison, never pass it).  Subsets keep the
index order, so depth ties resolve as in the full set.
"""

import dataclasses

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import COLOR_ATOL, COLOR_RTOL, DEPTH_ATOL, rtg

pytestmark = pytest.mark.gpu
ST = oracle.Settings()


def reach_subset(scene, cam, pix, margin=2.0):
    """Indices of the Gaussians whose support may reach one of the pixels (x, y)."""
    p = scene.means.astype(np.float64)
    R, t = cam.R.astype(np.float64), cam.t.astype(np.float64)
    pc = (p - t) @ R  # camera frame (R maps camera to world)
    X, Y, Z = pc[:, 0], pc[:, 1], pc[:, 2]
    ok = Z > 0.1
    Zs = np.where(ok, Z, 1.0)
    u = cam.fx * X / Zs + cam.cx
    v = cam.fy * Y / Zs + cam.cy
    f = max(cam.fx, cam.fy)
    smax = scene.scales.astype(np.float64).max(axis=1)
    jac = (f / Zs) * np.sqrt(2.0 + (X * X + Y * Y) / (Zs * Zs))  # Frobenius bound of the Jacobian
    sigma = np.sqrt((jac * smax) ** 2 + ST.lowpass)
    r = np.sqrt(2.0 * np.log(255.0)) * sigma + margin  # alpha <= 1: q <= 2 ln(255 alpha)
    keep = np.zeros(scene.n, dtype=bool)
    for x, y in pix:
        keep |= ok & (np.abs(u - x) <= r) & (np.abs(v - y) <= r)
    return np.flatnonzero(keep)


def check_pixels(scene, cam, color, depth, alpha, index, pix, max_border=2):
    """color [C,H,W], depth/alpha/index [H,W] (numpy) against the oracle at pix."""
    sub = reach_subset(scene, cam, pix)
    ref = oracle.render(scene.subset(sub), cam, ST, pixels=pix)
    ok = ~ref.borderline.numpy()
    assert (~ok).sum() <= max_border
    xs, ys = pix[:, 0], pix[:, 1]
    gc = color[:, ys, xs].T.astype(np.float64)
    rc = ref.color.numpy()
    assert (np.abs(gc - rc)[ok] <= COLOR_ATOL + COLOR_RTOL * np.abs(rc[ok])).all(), np.abs(gc - rc)[ok].max()
    assert (np.abs(alpha[ys, xs] - ref.alpha.numpy())[ok] <= COLOR_ATOL + COLOR_RTOL).all()
    assert (np.abs(depth[ys, xs] - ref.depth.numpy())[ok] <= DEPTH_ATOL).all()
    ri = ref.index.numpy()
    want = np.where(ri >= 0, sub[np.maximum(ri, 0)], -1)
    np.testing.assert_array_equal(index[ys, xs][ok], want[ok])
    return int(ok.sum())


def masked_forward(scene, cams, tuning, max_pairs, seed):
    """The bench's path: precomputed unstable index, window open, fused mask + forward."""
    m = rtg()
    F, H, W, C = len(cams), cams[0].height, cams[0].width, scene.colors.shape[1]
    ctx = m.Context(max_gaussians=scene.n, max_frames=F, max_width=W, max_height=H, max_channels=C,
                    max_pairs=max_pairs)
    ctx.set_tuning(tuning)
    g = m.Gaussians.from_scene(scene)
    rank, ids, nu = m.unstable_rank(ctx, g.unstable)
    g = dataclasses.replace(g, rank_map=rank, unstable_ids=ids, n_unstable=nu)
    m.window_begin(ctx, cams, g, m.RenderSettings())
    assert m.window_is_open(ctx)
    mask = torch.zeros(F, H, W, dtype=torch.uint8, device="cuda")
    color = torch.zeros(F, C, H, W, device="cuda")
    depth = torch.full((F, H, W), -1.0, device="cuda")
    alpha = torch.zeros(F, H, W, device="cuda")
    index = torch.full((F, H, W), -1, dtype=torch.int32, device="cuda")
    m.render_forward_masked(ctx, cams, g, m.RenderSettings(), mask, color, depth, alpha, index_map=index)
    torch.cuda.synchronize()
    st = m.get_stats(ctx)
    assert st["status"] == 0 and m.window_is_open(ctx)
    out = dict(mask=mask.cpu().numpy(), color=color.cpu().numpy(), depth=depth.cpu().numpy(),
               alpha=alpha.cpu().numpy(), index=index.cpu().numpy(), stats=st)
    del ctx
    torch.cuda.empty_cache()
    return out


def sample_masked(mask, k, rng):
    ys, xs = np.nonzero(mask)
    assert len(xs) >= k
    sel = rng.choice(len(xs), size=k, replace=False)
    return np.stack([xs[sel], ys[sel]], 1)


def test_masked_step_1M_sampled():
    """1M Gaussians, 20% unstable in 3 blobs, 640x480, mask with the tile rule (the bench's
    camera candidate), the bench's tuning: 8x8 / batch 64 / persistent at 2 CTAs per SM /
    ranking sort <= 512."""
    m = rtg()
    scene, layout = synth.room_scene(3000, 1_000_000)
    cams = synth.room_camera_candidates(3001, layout, 640, 480, 600.0)
    for _ in range(8):
        cam = next(cams)  # candidate 7
    scene.unstable = synth.flag_blobs(scene, [cam], 200_000, 3, seed=3000 + 100 + 7, n_in_view=1)
    out = masked_forward(scene, [cam], m.Tuning(8, 8, 64, 1, 2, 8, 512), 24_000_000, 3)
    cov = out["mask"][0].mean()
    assert 0.25 <= cov <= 0.40, cov
    pix = sample_masked(out["mask"][0], 48, np.random.default_rng(31))
    n = check_pixels(scene, cam, out["color"][0], out["depth"][0], out["alpha"][0], out["index"][0], pix)
    assert n >= 46


def test_batched_keyframes_2M_sampled():
    """2M Gaussians on a 2x2 grid of rooms, 10% unstable in 8 blobs, 8 keyframes at
    1200x680 in one call, the bench's tuning: 8x16 / batch 32 / CTA per tile / ranking sort
    <= 512."""
    m = rtg()
    scene, layout = synth.multiroom_scene(4000, 2_000_000)
    scene.unstable = synth.flag_blobs(scene, [], 200_000, 8, seed=4100, n_in_view=0)
    cams = [c for _, c in zip(range(8), synth.room_camera_candidates(4001, layout, 1200, 680, 600.0))]
    out = masked_forward(scene, cams, m.Tuning(8, 16, 32, 0, 4, 8, 512), 48 << 20, 4)
    rng = np.random.default_rng(41)
    frames = [f for f in range(8) if out["mask"][f].sum() >= 16]
    assert len(frames) >= 3
    for f in frames[:3]:
        pix = sample_masked(out["mask"][f], 16, rng)
        n = check_pixels(scene, cams[f], out["color"][f], out["depth"][f], out["alpha"][f], out["index"][f], pix)
        assert n >= 14


def test_large_floor_5M_32_keyframes_8_channels_sampled():
    """5M Gaussians on a 30x20x3 m floor (5x4 rooms), 90% opaque, 8 colour channels, 10%
    unstable, 32 keyframes at 1200x680 in one call, the bench's tuning: 8x8 / batch 32 /
    persistent at 2 CTAs per SM / ranking sort <= 512."""
    m = rtg()
    scene, layout = synth.room_scene(5000, 5_000_000, channels=8, opaque_frac=0.9, size=(30.0, 20.0, 3.0),
                                     grid=(5, 4), n_boxes=60)
    scene.unstable = synth.flag_blobs(scene, [], 500_000, 24, seed=5100, n_in_view=0)
    cams = [c for _, c in zip(range(32), synth.room_camera_candidates(5001, layout, 1200, 680, 600.0))]
    out = masked_forward(scene, cams, m.Tuning(8, 8, 32, 1, 2, 8, 512), 128 << 20, 5)
    assert out["stats"]["masked_pixels"] > 0
    rng = np.random.default_rng(51)
    frames = [f for f in range(32) if out["mask"][f].sum() >= 8]
    assert len(frames) >= 3
    for f in frames[:3]:
        pix = sample_masked(out["mask"][f], 8, rng)
        n = check_pixels(scene, cams[f], out["color"][f], out["depth"][f], out["alpha"][f], out["index"][f], pix)
        assert n >= 7


GROUPS = ("means", "scales", "quats", "opacity", "colors")


def test_masked_step_1M_gradients_sampled_pixels():
    """The backward at full size, in the bench's tuning: the 1M-Gaussian masked-step scene with
    the loss restricted to sampled masked pixels, against the FP64 oracle's analytic
    gradient on the Gaussians that can reach those pixels; every other unstable Gaussian
    must get exactly zero."""
    m = rtg()
    scene, layout = synth.room_scene(3000, 1_000_000)
    cams = synth.room_camera_candidates(3001, layout, 640, 480, 600.0)
    for _ in range(8):
        cam = next(cams)  # candidate 7
    scene.unstable = synth.flag_blobs(scene, [cam], 200_000, 3, seed=3000 + 100 + 7, n_in_view=1)
    H, W = cam.height, cam.width
    ctx = m.Context(max_gaussians=scene.n, max_width=W, max_height=H, max_pairs=24_000_000)
    ctx.set_tuning(m.Tuning(8, 8, 64, 1, 2, 8, 512))
    g = m.Gaussians.from_scene(scene)
    mask = torch.zeros(1, H, W, dtype=torch.uint8, device="cuda")
    m.unstable_mask(ctx, cam, g, m.RenderSettings(), mask)
    rng = np.random.default_rng(77)
    pix = sample_masked(mask[0].cpu().numpy(), 64, rng)
    sub_idx = reach_subset(scene, cam, pix)
    sub = scene.subset(sub_idx)
    tc = rng.uniform(0.0, 1.0, (len(pix), 3))
    td = rng.uniform(1.0, 5.0, len(pix))
    # pixels whose gradient sits on a threshold (alpha_min, f_max, the hit test) are left out
    pre = oracle.loss_and_grads(sub, cam, ST, pix, tc, td)
    keep = ~pre["grad_borderline"]
    assert keep.sum() >= 56
    pix, tc, td = pix[keep], tc[keep], td[keep]
    ref = oracle.loss_and_grads(sub, cam, ST, pix, tc, td)
    # the GPU step on exactly those pixels
    ms = torch.zeros(1, H, W, dtype=torch.uint8, device="cuda")
    tcol = torch.zeros(1, 3, H, W, device="cuda")
    tdep = torch.zeros(1, H, W, device="cuda")
    xs, ys = torch.as_tensor(pix[:, 0]).cuda(), torch.as_tensor(pix[:, 1]).cuda()
    ms[0, ys, xs] = 1
    tcol[0, :, ys, xs] = torch.as_tensor(tc.T, dtype=torch.float32).cuda()
    tdep[0, ys, xs] = torch.as_tensor(td, dtype=torch.float32).cuda()
    color = torch.zeros(1, 3, H, W, device="cuda")
    depth = torch.full((1, H, W), -1.0, device="cuda")
    alpha = torch.zeros(1, H, W, device="cuda")
    m.render_forward(ctx, cam, g, ms, m.RenderSettings(), color, depth, alpha)
    loss = torch.zeros(3, device="cuda")
    dc, dd = torch.zeros_like(color), torch.zeros_like(depth)
    m.l1_loss(ctx, color, depth, tcol, tdep, ms, 1.0, 1.0, loss, dc, dd)
    nu = int(scene.unstable.sum())
    grads = [torch.zeros(nu, 3, device="cuda"), torch.zeros(nu, 3, device="cuda"), torch.zeros(nu, 4, device="cuda"),
             torch.zeros(nu, device="cuda"), torch.zeros(nu, 3, device="cuda")]
    m.render_backward(ctx, dc, dd, *grads)
    torch.cuda.synchronize()
    assert m.get_status(ctx) == 0
    assert float(loss[0]) == pytest.approx(ref["loss"], rel=1e-4)
    got = {k: t.cpu().numpy().astype(np.float64) for k, t in zip(GROUPS, grads)}
    # compact rank of every unstable Gaussian of the full scene; the subset's, in its order
    rank = np.cumsum(scene.unstable.astype(np.int64)) - 1
    sub_unstable = sub_idx[scene.unstable[sub_idx] != 0]
    rows = rank[sub_unstable]
    others = np.ones(nu, dtype=bool)
    others[rows] = False
    for k in GROUPS:
        r = ref["grads"][k].reshape(len(rows), -1)
        gg = got[k].reshape(nu, -1)[rows]
        scale = np.abs(r).max()
        assert scale > 0, k
        assert np.linalg.norm(gg - r) <= 1e-3 * np.linalg.norm(r), (k, np.linalg.norm(gg - r) / np.linalg.norm(r))
        assert (np.abs(gg - r) <= 1e-3 * np.abs(r) + 1e-3 * scale).all(), (k, np.abs(gg - r).max(), scale)
        assert not got[k].reshape(nu, -1)[others].any(), k  # no influence on these pixels


def test_target_300k_fused_step_sampled_pixels():
    """The 300k masked step in the launch configuration the bench times: precomputed unstable
    index, window open (cached stable lists), the fused L1 forward and its backward, 8x8
    tiles, 32-record batches, the persistent schedule at 2 CTAs per SM, 8-bit digits,
    ranking sort up to 256 keys.  The unstable mask's coverage, then on sampled masked pixels
    the render, the loss and every gradient against the FP64 oracle; the unstable Gaussians
    that cannot reach those pixels get exactly zero."""
    m = rtg()
    scene, layout = synth.room_scene(2000, 300_000)
    cams = synth.room_camera_candidates(2001, layout, 640, 480, 600.0)
    for _ in range(11):
        cam = next(cams)  # candidate 10
    scene.unstable = synth.flag_blobs(scene, [cam], 60_000, 3, seed=2000 + 100 + 10, n_in_view=1)
    H, W = cam.height, cam.width
    ctx = m.Context(max_gaussians=scene.n, max_width=W, max_height=H)
    ctx.set_tuning(m.Tuning(8, 8, 32, 1, 2, 8, 256))
    g = m.Gaussians.from_scene(scene)
    rank, ids, nu = m.unstable_rank(ctx, g.unstable)
    g = dataclasses.replace(g, rank_map=rank, unstable_ids=ids, n_unstable=nu)
    mask = torch.zeros(1, H, W, dtype=torch.uint8, device="cuda")
    m.unstable_mask(ctx, cam, g, m.RenderSettings(), mask)
    cov = float(mask.float().mean())
    assert 0.25 <= cov <= 0.40, cov
    m.window_begin(ctx, [cam], g, m.RenderSettings())
    rng = np.random.default_rng(2010)
    pix = sample_masked(mask[0].cpu().numpy(), 64, rng)
    sub_idx = reach_subset(scene, cam, pix)
    sub = scene.subset(sub_idx)
    tc = rng.uniform(0.0, 1.0, (len(pix), 3))
    td = rng.uniform(1.0, 5.0, len(pix))
    pre = oracle.loss_and_grads(sub, cam, ST, pix, tc, td)
    keep = ~pre["grad_borderline"]
    assert keep.sum() >= 56
    pix, tc, td = pix[keep], tc[keep], td[keep]
    ref = oracle.loss_and_grads(sub, cam, ST, pix, tc, td)
    ms = torch.zeros(1, H, W, dtype=torch.uint8, device="cuda")
    tcol = torch.zeros(1, 3, H, W, device="cuda")
    tdep = torch.zeros(1, H, W, device="cuda")
    xs, ys = torch.as_tensor(pix[:, 0]).cuda(), torch.as_tensor(pix[:, 1]).cuda()
    ms[0, ys, xs] = 1
    tcol[0, :, ys, xs] = torch.as_tensor(tc.T, dtype=torch.float32).cuda()
    tdep[0, ys, xs] = torch.as_tensor(td, dtype=torch.float32).cuda()
    color = torch.zeros(1, 3, H, W, device="cuda")
    depth = torch.full((1, H, W), -1.0, device="cuda")
    alpha = torch.zeros(1, H, W, device="cuda")
    index = torch.full((1, H, W), -1, dtype=torch.int32, device="cuda")
    loss = torch.zeros(3, device="cuda")
    m.render_forward_l1(ctx, [cam], g, ms, m.RenderSettings(), tcol, tdep, 1.0, 1.0, color, depth, alpha, loss,
                        index)
    grads = [torch.zeros(nu, 3, device="cuda"), torch.zeros(nu, 3, device="cuda"), torch.zeros(nu, 4, device="cuda"),
             torch.zeros(nu, device="cuda"), torch.zeros(nu, 3, device="cuda")]
    m.render_backward_l1(ctx, *grads)
    torch.cuda.synchronize()
    assert m.get_status(ctx) == 0 and m.window_is_open(ctx)
    n = check_pixels(scene, cam, color[0].cpu().numpy(), depth[0].cpu().numpy(), alpha[0].cpu().numpy(),
                     index[0].cpu().numpy(), pix)
    assert n >= len(pix) - 2
    assert float(loss[0]) == pytest.approx(ref["loss"], rel=1e-4)
    got = {k: t.cpu().numpy().astype(np.float64) for k, t in zip(GROUPS, grads)}
    rank_np = np.cumsum(scene.unstable.astype(np.int64)) - 1
    rows = rank_np[sub_idx[scene.unstable[sub_idx] != 0]]
    others = np.ones(nu, dtype=bool)
    others[rows] = False
    for k in GROUPS:
        r = ref["grads"][k].reshape(len(rows), -1)
        gg = got[k].reshape(nu, -1)[rows]
        scale = np.abs(r).max()
        assert scale > 0, k
        assert np.linalg.norm(gg - r) <= 1e-3 * np.linalg.norm(r), (k, np.linalg.norm(gg - r) / np.linalg.norm(r))
        assert (np.abs(gg - r) <= 1e-3 * np.abs(r) + 1e-3 * scale).all(), (k, np.abs(gg - r).max(), scale)
        assert not got[k].reshape(nu, -1)[others].any(), k
    ctx.close()
