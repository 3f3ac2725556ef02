"""Launch configurations and keyframe batching.

The render tile, the per-warp record batch, the schedule (CTA per tile, or persistent
warps over the cost-ordered item queue) and the sort's digit width / ranking cutoff are
free choices of the implementation: rendered values must be bit-identical under every
one of them, and the loss and gradients equal to float32 rounding.  Rendering F keyframes
in one call must give each frame exactly what a call with that frame alone gives, and the
gradients must be the sum of the per-frame gradients.
"""

import numpy as np
import pytest
import torch

import synth
from gpu_util import ctx_for, gpu_forward, rtg

pytestmark = pytest.mark.gpu

W, H, F = 136, 100, 3  # ragged against every tile width and height


def tunings():
    T = rtg().Tuning
    return [
        T(8, 8), T(8, 16), T(16, 8), T(32, 8), T(batch=64), T(schedule=1),
        T(schedule=1, batch=64, persist_ctas_per_sm=1), T(16, 8, schedule=1, persist_ctas_per_sm=8),
        T(8, 8, 64, 1, 2, 4, 0), T(sort_digit_bits=4), T(sort_rank_max=256), T(sort_rank_max=2048),
        T(32, 8, 64, 1, 4, 4, 512),
    ]


def scene_and_cams(channels=3, seed=3100):
    scene, layout = synth.room_scene(seed, 20000, channels=channels)
    cams = [c for _, c in zip(range(F), synth.room_camera_candidates(seed + 1, layout, W, H, 110.0))]
    scene.unstable = synth.flag_blobs(scene, cams, 4000, 3, seed=seed + 2)
    masks = synth.random_masks(seed + 3, F, H, W, 0.15, 0.7)
    return scene, cams, masks


def targets(scene, cams, seed):
    ref = gpu_forward(synth.jitter_scene(scene, seed), cams)
    tc = torch.tensor(ref["color"]).cuda()
    td = torch.tensor(np.where(ref["depth"] > 0, ref["depth"], 0)).cuda()
    return tc, td


def run_step(ctx, scene, cams, mask, tc, td, tuning=None, accumulate=False, grads=None, masked=False):
    """Forward with the fused L1 loss, then its backward; returns images, loss, gradients."""
    m = rtg()
    if tuning is not None:
        ctx.set_tuning(tuning)
    g = m.Gaussians.from_scene(scene)
    nF, C = len(cams), scene.colors.shape[1]
    nu = int(scene.unstable.astype(bool).sum())
    color = torch.zeros(nF, C, H, W, device="cuda")
    depth = torch.full((nF, H, W), -1.0, device="cuda")
    alpha = torch.zeros(nF, H, W, device="cuda")
    index = torch.full((nF, H, W), -1, dtype=torch.int32, device="cuda")
    loss = torch.zeros(3, device="cuda")
    if grads is None:
        grads = [torch.zeros(nu, k, device="cuda") for k in (3, 3, 4)] + \
                [torch.zeros(nu, device="cuda"), torch.zeros(nu, C, device="cuda")]
    mk = mask
    if masked:
        mk = torch.zeros(nF, H, W, dtype=torch.uint8, device="cuda")
        m.render_forward_masked(ctx, cams, g, m.RenderSettings(), mk, color, depth, alpha, tc, td, 1.0, 1.0, loss,
                                index)
    else:
        m.render_forward_l1(ctx, cams, g, mask, m.RenderSettings(), tc, td, 1.0, 1.0, color, depth, alpha, loss,
                            index)
    m.render_backward_l1(ctx, *grads, accumulate=accumulate)
    torch.cuda.synchronize()
    st = m.get_stats(ctx)
    assert st["status"] == 0
    # g is returned too: a later backward of this forward reads the Gaussian arrays again
    return dict(color=color, depth=depth, alpha=alpha, index=index, loss=loss, grads=grads, stats=st, mask=mk, g=g)


def assert_grads_close(a, b, rel=2e-5):
    for x, y in zip(a, b):
        x, y = x.cpu().numpy().astype(np.float64), y.cpu().numpy().astype(np.float64)
        scale = max(np.abs(x).max(initial=0.0), 1e-30)
        assert np.abs(x - y).max(initial=0.0) <= rel * scale, (np.abs(x - y).max(), scale)


@pytest.mark.parametrize("channels", [3, 8])
def test_every_tuning_renders_bit_identical_images(channels):
    scene, cams, masks = scene_and_cams(channels, seed=3100 + channels)
    tc, td = targets(scene, cams, 3150)
    mask = torch.as_tensor(masks).reshape(F, H, W).cuda()
    ctx = ctx_for(scene.n, cams, channels)
    ref = run_step(ctx, scene, cams, mask, tc, td, rtg().Tuning())
    assert ref["stats"]["masked_pixels"] > 1000 and ref["stats"]["pairs"] > 1000
    for t in tunings():
        got = run_step(ctx, scene, cams, mask, tc, td, t)
        for k in ("color", "depth", "alpha", "index"):
            assert torch.equal(got[k], ref[k]), (t, k)
        assert got["stats"]["fragments"] == ref["stats"]["fragments"], t
        assert got["stats"]["masked_pixels"] == ref["stats"]["masked_pixels"], t
        np.testing.assert_allclose(got["loss"].cpu().numpy(), ref["loss"].cpu().numpy(), rtol=1e-5)
        assert_grads_close(got["grads"], ref["grads"])


def test_fused_mask_under_every_tile_matches_default():
    """rtg_render_forward_masked keeps the tile rule on its 16 x 16 grid whatever the render
    tile: the mask and the images are bit-identical to the default tiling's."""
    scene, cams, _ = scene_and_cams(3, seed=3200)
    tc, td = targets(scene, cams, 3250)
    ctx = ctx_for(scene.n, cams)
    ref = run_step(ctx, scene, cams, None, tc, td, rtg().Tuning(), masked=True)
    assert 0 < int(ref["mask"].sum()) < F * H * W
    for t in tunings()[:8]:
        got = run_step(ctx, scene, cams, None, tc, td, t, masked=True)
        for k in ("mask", "color", "depth", "alpha", "index"):
            assert torch.equal(got[k], ref[k]), (t, k)
        assert_grads_close(got["grads"], ref["grads"])


@pytest.mark.parametrize("empty_frame", [None, 1])
@pytest.mark.parametrize("schedule", [0, 1])
def test_batched_keyframes_equal_per_frame_calls(schedule, empty_frame):
    """One call over F keyframes renders each frame bit for bit like a call with that frame
    alone; its gradients (explicit per-pixel dL images, so no loss normalisation couples
    the frames) equal the per-frame gradients summed with accumulate.  empty_frame: that
    keyframe's mask is empty (it adds no work item; its outputs keep their contents)."""
    m = rtg()
    scene, cams, masks = scene_and_cams(3, seed=3300)
    mask = torch.as_tensor(masks).reshape(F, H, W).cuda()
    if empty_frame is not None:
        mask[empty_frame] = 0
    assert int(mask.sum()) > 0
    g = m.Gaussians.from_scene(scene)
    nu = int(scene.unstable.astype(bool).sum())
    rng = np.random.default_rng(3301)
    dc = torch.tensor(rng.normal(size=(F, 3, H, W)).astype(np.float32)).cuda()
    dd = torch.tensor(rng.normal(size=(F, H, W)).astype(np.float32)).cuda()
    tune = m.Tuning(16, 8, 64, schedule, 4, 8, 256)

    def grads0():
        return [torch.zeros(nu, k, device="cuda") for k in (3, 3, 4)] + \
               [torch.zeros(nu, device="cuda"), torch.zeros(nu, 3, device="cuda")]

    def bufs(nf):
        return (torch.zeros(nf, 3, H, W, device="cuda"), torch.full((nf, H, W), -1.0, device="cuda"),
                torch.zeros(nf, H, W, device="cuda"), torch.full((nf, H, W), -1, dtype=torch.int32, device="cuda"))

    ctx = ctx_for(scene.n, cams)
    ctx.set_tuning(tune)
    cb, db, ab, ib = bufs(F)
    gb = grads0()
    m.render_forward(ctx, cams, g, mask, m.RenderSettings(), cb, db, ab, ib)
    m.render_backward(ctx, dc, dd, *gb)
    ctx1 = ctx_for(scene.n, cams[:1])
    ctx1.set_tuning(tune)
    gs = grads0()
    for f in range(F):
        c1, d1, a1, i1 = bufs(1)
        m.render_forward(ctx1, [cams[f]], g, mask[f:f + 1].contiguous(), m.RenderSettings(), c1, d1, a1, i1)
        m.render_backward(ctx1, dc[f:f + 1].contiguous(), dd[f:f + 1].contiguous(), *gs, accumulate=f > 0)
        torch.cuda.synchronize()
        assert torch.equal(c1[0], cb[f]) and torch.equal(d1[0], db[f])
        assert torch.equal(a1[0], ab[f]) and torch.equal(i1[0], ib[f])
    assert_grads_close(gs, gb, rel=5e-5)
    assert max(float(x.abs().max()) for x in gb) > 0


def test_repeated_backward_after_one_forward():
    """The persistent backward's queue is refilled for a second backward of the same forward."""
    scene, cams, masks = scene_and_cams(3, seed=3400)
    tc, td = targets(scene, cams, 3450)
    mask = torch.as_tensor(masks).reshape(F, H, W).cuda()
    ctx = ctx_for(scene.n, cams)
    a = run_step(ctx, scene, cams, mask, tc, td, rtg().Tuning(schedule=1))
    g2 = [torch.zeros_like(x) for x in a["grads"]]
    rtg().render_backward_l1(ctx, *g2)
    torch.cuda.synchronize()
    assert_grads_close(g2, a["grads"])
    # accumulate adds a third copy on top of the second
    rtg().render_backward_l1(ctx, *g2, accumulate=True)
    torch.cuda.synchronize()
    assert_grads_close(g2, [2 * x for x in a["grads"]])


def test_tuning_validation_and_readback():
    m = rtg()
    ctx = m.Context(max_gaussians=100)
    assert ctx.get_tuning() == m.Tuning()
    for bad in (m.Tuning(4, 8), m.Tuning(16, 32), m.Tuning(32, 16), m.Tuning(12, 8), m.Tuning(batch=48),
                m.Tuning(schedule=2), m.Tuning(persist_ctas_per_sm=0), m.Tuning(persist_ctas_per_sm=9),
                m.Tuning(sort_digit_bits=6), m.Tuning(sort_rank_max=4096), m.Tuning(sort_rank_max=-1)):
        with pytest.raises(m.RTGError):
            ctx.set_tuning(bad)
        assert ctx.get_tuning() == m.Tuning()
    t = m.Tuning(32, 8, 64, 1, 2, 4, 128)
    ctx.set_tuning(t)
    assert ctx.get_tuning() == t


def test_small_tiles_overflow_reports_status():
    """8 x 8 tiles make more pairs than 16 x 16 ones: a capacity that holds one tiling and
    not the other reports RTG_ERR_WORKSPACE for the finer one only."""
    m = rtg()
    scene, cams, masks = scene_and_cams(3, seed=3500)
    mask = torch.as_tensor(masks).reshape(F, H, W).cuda()
    probe = gpu_forward(scene, cams, mask=masks)
    p16 = probe["stats"]["pairs"]
    c8 = ctx_for(scene.n, cams)
    c8.set_tuning(m.Tuning(8, 8))
    p8 = gpu_forward(scene, cams, mask=masks, ctx=c8)["stats"]["pairs"]
    assert p8 > p16
    ctx = ctx_for(scene.n, cams, max_pairs=(p16 + p8) // 2)
    gpu_forward(scene, cams, mask=masks, ctx=ctx)
    assert m.get_status(ctx) == 0
    ctx.set_tuning(m.Tuning(8, 8, schedule=1))
    color = torch.zeros(F, 3, H, W, device="cuda")
    depth = torch.zeros(F, H, W, device="cuda")
    alpha = torch.zeros(F, H, W, device="cuda")
    m.render_forward(ctx, cams, m.Gaussians.from_scene(scene), mask, m.RenderSettings(), color, depth, alpha)
    torch.cuda.synchronize()
    assert m.get_status(ctx) == m._lib.RTG_ERR_WORKSPACE
    assert float(color.abs().sum()) == 0.0  # the render kernels skipped their work


def test_autotuner_picks_a_timed_candidate_and_checks_renders():
    m = rtg()
    from paper_2404_19706_b300.tune import autotune
    scene, cams, _ = scene_and_cams(3, seed=3600)
    tc, td = targets(scene, cams, 3650)
    ctx = ctx_for(scene.n, cams)
    g = m.Gaussians.from_scene(scene)
    mask = torch.zeros(F, H, W, dtype=torch.uint8, device="cuda")
    step = m.MaskedStep(ctx, g, cams, mask, tc, td, recompute_mask=True)
    keep = [t.clone() for t in (g.means, g.scales, g.quats, g.opacity, g.colors)]
    ck = [torch.zeros(F, H, W, dtype=torch.uint8, device="cuda"), torch.zeros(F, 3, H, W, device="cuda"),
          torch.zeros(F, H, W, device="cuda"), torch.zeros(F, H, W, device="cuda")]

    def check():
        m.render_forward_masked(ctx, cams, step.g, m.RenderSettings(), *ck)
        return ck

    def restore():
        for t, k in zip((g.means, g.scales, g.quats, g.opacity, g.colors), keep):
            t.copy_(k)
        for t in (step.m, step.v, step.step_counter):
            t.zero_()
        for t, k in zip(step.u, m.api.gather_unstable(step.ids, step.g)):
            t.copy_(k)

    res = autotune(ctx, step._body, check, restore, warmup=1, iters=3, repeats=1)
    assert ctx.get_tuning() == res.best
    timed = [r for r in res.table if r["ms"] is not None]
    assert len(res.table) == 1 + 40 + 5 and len(timed) == len(res.table)
    assert res.best_ms == min(r["ms"] for r in timed if r["tuning"] == res.best.as_dict())
    assert res.best_ms <= res.default_ms * 1.0001 or res.best.as_dict() == res.table[0]["tuning"]


def test_many_tile_call_backward_matches_per_tile_schedule():
    """A call of more than 8,192 render tiles (four 480x360 keyframes in 8x8 tiles) takes the
    segmented backward with ten warps a CTA: its renders equal the per-tile schedule's bit
    for bit, its gradients those of the per-tile whole-list replay to float32 rounding."""
    m = rtg()
    nF, hh, ww = 4, 360, 480
    scene, layout = synth.room_scene(3500, 60000)
    cams = [c for _, c in zip(range(nF), synth.room_camera_candidates(3501, layout, ww, hh, 360.0))]
    scene.unstable = synth.flag_blobs(scene, cams, 12000, 4, seed=3502)
    mask = torch.as_tensor(synth.random_masks(3503, nF, hh, ww, 0.3, 0.8)).reshape(nF, hh, ww).cuda()
    ref = gpu_forward(synth.jitter_scene(scene, 3504), cams)
    tc = torch.tensor(ref["color"]).cuda()
    td = torch.tensor(np.where(ref["depth"] > 0, ref["depth"], 0)).cuda()
    ref["ctx"].close()
    g = m.Gaussians.from_scene(scene)
    nu = int(scene.unstable.astype(bool).sum())
    outs = []
    for tune in (m.Tuning(8, 8, 32, 1, 2, 8, 512), m.Tuning(8, 8, 32, 0, 4, 8, 512)):
        ctx = ctx_for(scene.n, cams)
        ctx.set_tuning(tune)
        img = [torch.zeros(nF, 3, hh, ww, device="cuda"), torch.full((nF, hh, ww), -1.0, device="cuda"),
               torch.zeros(nF, hh, ww, device="cuda"), torch.full((nF, hh, ww), -1, dtype=torch.int32, device="cuda")]
        loss = torch.zeros(3, device="cuda")
        grads = [torch.zeros(nu, k, device="cuda") for k in (3, 3, 4)] + \
                [torch.zeros(nu, device="cuda"), torch.zeros(nu, 3, device="cuda")]
        m.render_forward_l1(ctx, cams, g, mask, m.RenderSettings(), tc, td, 1.0, 1.0, img[0], img[1], img[2], loss,
                            img[3])
        m.render_backward_l1(ctx, *grads)
        torch.cuda.synchronize()
        st = m.get_stats(ctx)
        assert st["status"] == 0
        outs.append((img, loss, grads, st))
        ctx.close()
    (ia, la, ga, sa), (ib, lb, gb, sb) = outs
    assert sa["pairs"] > 0 and sa["fragments"] == sb["fragments"]
    for x, y in zip(ia, ib):
        assert torch.equal(x, y)
    np.testing.assert_allclose(la.cpu().numpy(), lb.cpu().numpy(), rtol=1e-5)
    for x, y in zip(ga, gb):
        x, y = x.cpu().numpy(), y.cpu().numpy()
        scale = max(np.abs(x).max(), np.abs(y).max())
        assert scale > 0 and np.abs(x - y).max() <= 1e-4 * scale, (np.abs(x - y).max(), scale)
