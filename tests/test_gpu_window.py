"""Optimisation window (Section 3.2: only the unstable Gaussians move within a window):
forwards that reuse the stable Gaussians' records give exactly what full forwards give."""

import numpy as np
import pytest
import torch

import synth
from gpu_util import ctx_for, gpu_forward, rtg

pytestmark = pytest.mark.gpu

W, H, F = 120, 88, 2


def setup(seed, channels=3):
    m = rtg()
    scene, layout = synth.room_scene(seed, 30000, channels=channels)
    cams = [c for _, c in zip(range(F), synth.room_camera_candidates(seed + 1, layout, W, H, 100.0))]
    scene.unstable = synth.flag_blobs(scene, cams, 5000, 3, seed=seed + 2)
    ref = gpu_forward(synth.jitter_scene(scene, seed + 3), cams)
    tc = torch.tensor(ref["color"]).cuda()
    td = torch.tensor(np.where(ref["depth"] > 0, ref["depth"], 0)).cuda()
    ctx = ctx_for(scene.n, cams, channels)
    g = m.Gaussians.from_scene(scene)
    rank, ids, nu = m.unstable_rank(ctx, g.unstable)
    import dataclasses
    g = dataclasses.replace(g, rank_map=rank, unstable_ids=ids, n_unstable=nu)
    masks = torch.as_tensor(synth.random_masks(seed + 4, F, H, W, 0.2, 0.6)).cuda()
    return ctx, g, cams, tc, td, masks, nu


def render(ctx, g, cams, tc, td, masks, nu, fused, C=3):
    m = rtg()
    out = dict(mask=torch.zeros(F, H, W, dtype=torch.uint8, device="cuda"),
               color=torch.zeros(F, C, H, W, device="cuda"), depth=torch.zeros(F, H, W, device="cuda"),
               alpha=torch.zeros(F, H, W, device="cuda"), index=torch.zeros(F, H, W, dtype=torch.int32, device="cuda"),
               loss=torch.zeros(3, device="cuda"))
    if fused:
        m.render_forward_masked(ctx, cams, g, m.RenderSettings(), out["mask"], out["color"], out["depth"],
                                out["alpha"], tc, td, 1.0, 1.0, out["loss"], out["index"])
    else:
        m.render_forward_l1(ctx, cams, g, masks, m.RenderSettings(), tc, td, 1.0, 1.0, out["color"], out["depth"],
                            out["alpha"], out["loss"], out["index"])
    grads = [torch.zeros(nu, k, device="cuda") for k in (3, 3, 4)] + [torch.zeros(nu, device="cuda"),
                                                                      torch.zeros(nu, C, device="cuda")]
    m.render_backward_l1(ctx, *grads)
    torch.cuda.synchronize()
    out["grads"] = grads
    out["stats"] = m.get_stats(ctx)
    assert out["stats"]["status"] == 0
    return out


def same(a, b):
    """b (a window forward) equals a (a full forward).  With the window's cached lists only
    the unstable projections count as visible."""
    for k in ("mask", "color", "depth", "alpha", "index"):
        assert torch.equal(a[k], b[k]), k
    np.testing.assert_allclose(a["loss"].cpu().numpy(), b["loss"].cpu().numpy(), rtol=1e-6)
    for k in ("pairs", "fragments", "masked_pixels", "max_tile_pairs"):
        assert a["stats"][k] == b["stats"][k], k
    assert 0 < b["stats"]["visible"] <= a["stats"]["visible"]
    for x, y in zip(a["grads"], b["grads"]):
        x, y = x.cpu().numpy(), y.cpu().numpy()
        assert np.abs(x - y).max(initial=0) <= 2e-5 * max(np.abs(x).max(initial=0), 1e-30)


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("tile", [(16, 16), (8, 16)])
def test_window_forward_equals_full_forward(fused, tile):
    m = rtg()
    ctx, g, cams, tc, td, masks, nu = setup(5100)
    ctx.set_tuning(m.Tuning(tile[0], tile[1], schedule=1))
    full = render(ctx, g, cams, tc, td, masks, nu, fused)
    m.window_begin(ctx, cams, g, m.RenderSettings())
    assert m.window_is_open(ctx)
    for _ in range(2):  # the window serves repeated iterations
        win = render(ctx, g, cams, tc, td, masks, nu, fused)
        assert m.window_is_open(ctx)
        same(full, win)


def test_window_follows_the_unstable_gaussians_as_they_move():
    """Moving the unstable Gaussians (as the optimiser does) inside the window: each render
    equals a full render of the same parameters."""
    m = rtg()
    ctx, g, cams, tc, td, masks, nu = setup(5200)
    ctx_full = ctx_for(g.n, cams)
    m.window_begin(ctx, cams, g, m.RenderSettings())
    u = g.unstable.bool()
    rng = torch.Generator(device="cuda").manual_seed(5)
    for it in range(3):
        g.means[u] += 0.01 * torch.randn(int(u.sum()), 3, device="cuda", generator=rng)
        g.colors[u] = torch.rand(int(u.sum()), 3, device="cuda", generator=rng)
        win = render(ctx, g, cams, tc, td, masks, nu, fused=True)
        full = render(ctx_full, g, cams, tc, td, masks, nu, fused=True)
        assert m.window_is_open(ctx)
        same(full, win)


def test_mismatching_forward_closes_the_window():
    m = rtg()
    ctx, g, cams, tc, td, masks, nu = setup(5300)
    m.window_begin(ctx, cams, g, m.RenderSettings())
    # a different camera set: rendered without the window (and correctly), window closed
    other = [cams[1], cams[0]]
    got = render(ctx, g, other, tc, td, masks, nu, fused=False)
    assert not m.window_is_open(ctx)
    ref = render(ctx_for(g.n, other), g, other, tc, td, masks, nu, fused=False)
    same(ref, got)
    # reopened and ended explicitly
    m.window_begin(ctx, cams, g, m.RenderSettings())
    assert m.window_is_open(ctx)
    m.window_end(ctx)
    assert not m.window_is_open(ctx)
    # the mask pass writes unstable records only, so it leaves the window open
    m.window_begin(ctx, cams, g, m.RenderSettings())
    m.unstable_mask(ctx, cams, g, m.RenderSettings(), torch.zeros(F, H, W, dtype=torch.uint8, device="cuda"))
    assert m.window_is_open(ctx)
    full = render(ctx_for(g.n, cams), g, cams, tc, td, masks, nu, fused=True)
    same(full, render(ctx, g, cams, tc, td, masks, nu, fused=True))


def test_window_needs_the_unstable_index():
    m = rtg()
    ctx, g, cams, tc, td, masks, nu = setup(5400)
    import dataclasses
    bare = dataclasses.replace(g, rank_map=None, unstable_ids=None, n_unstable=0)
    with pytest.raises(ValueError):
        m.window_begin(ctx, cams, bare, m.RenderSettings())


def test_masked_step_with_and_without_window_agree():
    m = rtg()
    scene, layout = synth.room_scene(5500, 30000)
    cams = [c for _, c in zip(range(F), synth.room_camera_candidates(5501, layout, W, H, 100.0))]
    scene.unstable = synth.flag_blobs(scene, cams, 5000, 3, seed=5502)
    ref = gpu_forward(synth.jitter_scene(scene, 5503), cams)
    tc = torch.tensor(ref["color"]).cuda()
    td = torch.tensor(np.where(ref["depth"] > 0, ref["depth"], 0)).cuda()
    out = []
    for window in (False, True):
        ctx = ctx_for(scene.n, cams)
        g = m.Gaussians.from_scene(scene)
        mask = torch.zeros(F, H, W, dtype=torch.uint8, device="cuda")
        step = m.MaskedStep(ctx, g, cams, mask, tc, td, recompute_mask=True, window=window)
        losses = [step.step().clone() for _ in range(3)]
        step.capture()
        losses += [step.step().clone() for _ in range(3)]
        step.write_back()
        torch.cuda.synchronize()
        assert m.window_is_open(ctx) == window
        out.append((torch.stack(losses).cpu().numpy(), g.means.cpu().numpy(), mask.clone()))
    np.testing.assert_allclose(out[1][0], out[0][0], rtol=1e-4)
    # gradients agree to rounding (atomic order), but Adam normalises each update, so an
    # element whose gradient is ~0 can step by +-lr either way: bound the bulk, not the max
    d = np.abs(out[1][1] - out[0][1])
    assert np.mean(d > 1e-6) < 0.01 and d.max() <= 6 * 2 * 1e-3 + 1e-6
    assert out[0][0][-1, 0] < out[0][0][0, 0]  # the loss goes down


def test_window_lists_follow_the_render_tile():
    """Changing the render tile rebuilds the window's cached stable lists for the new grid."""
    m = rtg()
    ctx, g, cams, tc, td, masks, nu = setup(5600)
    ref_ctx = ctx_for(g.n, cams)
    m.window_begin(ctx, cams, g, m.RenderSettings())
    for t in (m.Tuning(8, 16, schedule=1), m.Tuning(32, 8, 64), m.Tuning(16, 16, sort_rank_max=512)):
        ctx.set_tuning(t)
        ref_ctx.set_tuning(t)
        assert m.window_is_open(ctx)
        for fused in (False, True):
            same(render(ref_ctx, g, cams, tc, td, masks, nu, fused), render(ctx, g, cams, tc, td, masks, nu, fused))


def test_window_too_large_for_lists_keeps_projections_only():
    """A pair capacity that holds a masked forward but not the stable Gaussians' whole-frame
    lists: the window keeps its projections only, and forwards stay exact."""
    m = rtg()
    ctx0, g, cams, tc, td, _, nu = setup(5700)
    small = torch.as_tensor(synth.random_masks(5710, F, H, W, 0.03, 0.08)).cuda()
    full = render(ctx0, g, cams, tc, td, small, nu, fused=False)
    probe = ctx_for(g.n, cams)
    c = torch.zeros(F, 3, H, W, device="cuda")
    d = torch.zeros(F, H, W, device="cuda")
    a = torch.zeros(F, H, W, device="cuda")
    m.render_forward(probe, cams, g, None, m.RenderSettings(), c, d, a)  # whole frames
    ids = m.debug_binning(probe, F, W, H, g.n)["sorted_ids"]
    stable_whole = int((g.unstable.cpu().numpy()[ids.astype(np.int64)] == 0).sum())
    masked = full["stats"]["pairs"]
    assert stable_whole > masked + 2, (stable_whole, masked)
    ctx = ctx_for(g.n, cams, max_pairs=(stable_whole + masked) // 2)
    m.window_begin(ctx, cams, g, m.RenderSettings())
    assert m.window_is_open(ctx) and m.get_status(ctx) == 0
    win = render(ctx, g, cams, tc, td, small, nu, fused=False)
    same(full, win)
