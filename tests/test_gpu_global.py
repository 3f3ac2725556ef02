"""Global keyframe optimisation on the GPU (Section 3.2, "Keyframes and global
optimization"): the top-error pixel selection bit-exact against the oracle, the narrowed
backward against a forward rendered on the narrowed mask, the global step's gradients
against the FP64 oracle with every Gaussian optimised, and the step's Adam settings
(positions fixed, 0.1x rates) against the oracle's Adam."""

import dataclasses

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import ctx_for, rtg
from oracle import global_opt as go
from test_gpu_backward import GROUPS, compare_groups, crop_problem

pytestmark = pytest.mark.gpu
ST = oracle.Settings()


def gpu_select(color, target, frac, ctx=None):
    m = rtg()
    F, C, H, W = color.shape
    if ctx is None:
        ctx = m.Context(max_gaussians=1, max_frames=F, max_width=W, max_height=H, max_channels=3, max_pairs=1 << 10)
    c = torch.as_tensor(np.ascontiguousarray(color, np.float32)).cuda()
    t = torch.as_tensor(np.ascontiguousarray(target, np.float32)).cuda()
    out = torch.full((F, H, W), 7, dtype=torch.uint8, device="cuda")
    m.select_top_error(ctx, c, t, frac, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def tie_heavy(seed, F, C, H, W, levels):
    """Colours on a grid of `levels` values against a zero target: many equal errors."""
    rng = np.random.default_rng(seed)
    color = (rng.integers(0, levels, (F, C, H, W)) / levels).astype(np.float32)
    return color, np.zeros_like(color)


@pytest.mark.parametrize("F,C,H,W,levels", [(1, 3, 7, 5, 3), (3, 3, 37, 53, 4), (2, 8, 100, 130, 6),
                                            (2, 3, 64, 64, 0), (1, 1, 1, 1, 2)])
@pytest.mark.parametrize("frac", [0.4, 0.0, 1.0, 0.25, 0.999])
def test_select_matches_oracle(F, C, H, W, levels, frac):
    if levels:
        color, target = tie_heavy(F * 1000 + H, F, C, H, W, levels)
    else:  # continuous errors: no ties
        rng = np.random.default_rng(5)
        color = rng.uniform(0, 1, (F, C, H, W)).astype(np.float32)
        target = rng.uniform(0, 1, (F, C, H, W)).astype(np.float32)
    got = gpu_select(color, target, frac)
    want = go.top_error_mask(color, target, frac)
    np.testing.assert_array_equal(got, want)


def test_select_all_equal_and_mostly_zero():
    """All errors equal: the first k pixels.  70% zero errors: the threshold is 0 and the
    zero-error pixels taken are the lowest-indexed ones (spanning several blocks)."""
    H, W = 90, 200
    color = np.full((2, 3, H, W), 0.5, np.float32)
    target = np.zeros_like(color)
    got = gpu_select(color, target, 0.4)
    k = go.keep_count(0.4, H * W)
    flat = got.reshape(2, -1)
    assert (flat[:, :k] == 1).all() and (flat[:, k:] == 0).all()
    rng = np.random.default_rng(8)
    color = np.where(rng.random((2, 3, H, W)) < 0.3, rng.uniform(0, 1, (2, 3, H, W)), 0).astype(np.float32)
    color[:, :, rng.random((H, W)) < 0.7] = 0.0
    got = gpu_select(color, target, 0.4)
    np.testing.assert_array_equal(got, go.top_error_mask(color, target, 0.4))


def test_select_full_size_four_keyframes():
    """Four 1200x680 keyframes (816k pixels each, 200 blocks per frame), errors quantised to
    256 levels so ties straddle many blocks."""
    color, target = tie_heavy(77, 4, 3, 680, 1200, 256)
    got = gpu_select(color, target, 0.4)
    np.testing.assert_array_equal(got, go.top_error_mask(color, target, 0.4))


def test_select_argument_errors():
    m = rtg()
    ctx = m.Context(max_gaussians=1, max_frames=2, max_width=16, max_height=16, max_pairs=1 << 10)
    c = torch.zeros(1, 3, 8, 8, device="cuda")
    out = torch.zeros(1, 8, 8, dtype=torch.uint8, device="cuda")
    for frac in (-0.1, 1.5, float("nan")):
        with pytest.raises(m.RTGError):
            m.select_top_error(ctx, c, c, frac, out)
    big = torch.zeros(3, 3, 8, 8, device="cuda")
    with pytest.raises(m.RTGError):  # more frames than the capacity
        m.select_top_error(ctx, big, big, 0.4, torch.zeros(3, 8, 8, dtype=torch.uint8, device="cuda"))
    with pytest.raises(m.RTGError):  # no forward to narrow
        m.narrow_pixels(ctx, out)


def _render(m, ctx, cams, g, mask, C, H, W):
    F = len(cams)
    color = torch.zeros(F, C, H, W, device="cuda")
    depth = torch.full((F, H, W), -1.0, device="cuda")
    alpha = torch.zeros(F, H, W, device="cuda")
    m.render_forward(ctx, cams, g, mask, m.RenderSettings(), color, depth, alpha)
    return color, depth, alpha


def _loss_backward(m, ctx, color, depth, tc, td, mask, n, C):
    loss = torch.zeros(3, device="cuda")
    dc, dd = torch.zeros_like(color), torch.zeros_like(depth)
    m.l1_loss(ctx, color, depth, tc, td, mask, 1.0, 1.0, loss, dc, dd)
    grads = [torch.zeros(n, 3, device="cuda"), torch.zeros(n, 3, device="cuda"), torch.zeros(n, 4, device="cuda"),
             torch.zeros(n, device="cuda"), torch.zeros(n, C, device="cuda")]
    m.render_backward(ctx, dc, dd, *grads)
    torch.cuda.synchronize()
    assert m.get_status(ctx) == 0
    return loss.cpu().numpy(), {k: t.cpu().numpy().astype(np.float64) for k, t in zip(GROUPS, grads)}


@pytest.mark.parametrize("tuning", [(16, 16, 32, 0, 4, 8, 0), (8, 16, 32, 1, 4, 8, 256)])
def test_narrowed_backward_equals_masked_forward(tuning):
    """Full-frame forward narrowed to the top-40% pixels == a forward rendered on that mask,
    for the loss (to float32 rounding) and the gradients of every Gaussian; two keyframes."""
    m = rtg()
    scene, layout = synth.room_scene(6100, 40_000)
    scene.unstable = np.ones(scene.n, np.uint8)
    cams = [c for _, c in zip(range(2), synth.room_camera_candidates(6101, layout, 160, 120, 150.0))]
    target = synth.jitter_scene(scene, 6102)
    F, C, H, W = 2, 3, 120, 160
    tgt = m.Gaussians.from_scene(target)
    ctx = ctx_for(scene.n, cams)
    ctx.set_tuning(m.Tuning(*tuning))
    tc, td, _ = _render(m, ctx, cams, tgt, None, C, H, W)
    td = torch.where(td > 0, td, torch.zeros_like(td))
    g = m.Gaussians.from_scene(scene)
    color, depth, _ = _render(m, ctx, cams, g, None, C, H, W)
    sel = torch.zeros(F, H, W, dtype=torch.uint8, device="cuda")
    m.select_top_error(ctx, color, tc, 0.4, sel)
    m.narrow_pixels(ctx, sel)
    loss_a, grads_a = _loss_backward(m, ctx, color, depth, tc, td, sel, scene.n, C)
    assert sel.sum().item() == 2 * go.keep_count(0.4, H * W)
    color_b, depth_b, _ = _render(m, ctx, cams, g, sel, C, H, W)
    loss_b, grads_b = _loss_backward(m, ctx, color_b, depth_b, tc, td, sel, scene.n, C)
    np.testing.assert_allclose(loss_a, loss_b, rtol=1e-6)
    for k in GROUPS:
        a, b = grads_a[k], grads_b[k]
        assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b) + 1e-12, k
    # fused: narrowing with the targets forms the loss for render_backward_l1, and equals a
    # forward_l1 rendered on the mask
    grads_c, loss_c = _fused(m, ctx, cams, g, None, sel, tc, td, scene.n, C)
    grads_d, loss_d = _fused(m, ctx, cams, g, sel, None, tc, td, scene.n, C)
    np.testing.assert_allclose(loss_c, loss_d, rtol=1e-6)
    np.testing.assert_allclose(loss_c, loss_b, rtol=1e-6)
    assert m.get_stats(ctx)["masked_pixels"] == 2 * go.keep_count(0.4, H * W)
    for k in GROUPS:
        assert np.linalg.norm(grads_c[k] - grads_d[k]) <= 1e-5 * np.linalg.norm(grads_d[k]) + 1e-12, k
        assert np.linalg.norm(grads_c[k] - grads_b[k]) <= 1e-5 * np.linalg.norm(grads_b[k]) + 1e-12, k
    # narrowing without targets refuses the fused backward
    _render(m, ctx, cams, g, None, C, H, W)
    m.narrow_pixels(ctx, sel)
    with pytest.raises(m.RTGError):
        m.render_backward_l1(ctx, *[torch.zeros(scene.n, k, device="cuda") for k in (3, 3, 4, 1, 3)])
    with pytest.raises(m.RTGError):  # one target without the other
        m.narrow_pixels(ctx, sel, tc, None, 1.0, 1.0, torch.zeros(3, device="cuda"))


def _fused(m, ctx, cams, g, render_mask, narrow_mask, tc, td, n, C):
    """forward_l1 on render_mask (None: every pixel), then (narrow_mask) narrowing with the
    targets, then backward_l1; returns (gradients, loss)."""
    F, _, H, W = tc.shape
    loss = torch.zeros(3, device="cuda")
    color = torch.zeros(F, C, H, W, device="cuda")
    depth = torch.full((F, H, W), -1.0, device="cuda")
    m.render_forward_l1(ctx, cams, g, render_mask, m.RenderSettings(), tc, td, 1.0, 1.0, color, depth,
                        torch.zeros(F, H, W, device="cuda"), loss)
    if narrow_mask is not None:
        m.narrow_pixels(ctx, narrow_mask, tc, td, 1.0, 1.0, loss)
    grads = [torch.zeros(n, 3, device="cuda"), torch.zeros(n, 3, device="cuda"), torch.zeros(n, 4, device="cuda"),
             torch.zeros(n, device="cuda"), torch.zeros(n, C, device="cuda")]
    m.render_backward_l1(ctx, *grads)
    torch.cuda.synchronize()
    assert m.get_status(ctx) == 0
    return {k: t.cpu().numpy().astype(np.float64) for k, t in zip(GROUPS, grads)}, loss.cpu().numpy()


@pytest.mark.parametrize("seed", [3000, 3100])
def test_global_gradients_match_oracle(seed):
    """Every Gaussian optimised; the GPU picks the top-40% pixels of its own render (checked
    bit-exact against the oracle's selection on the same colours), the forward is narrowed
    to them (less the oracle's borderline pixels) and the gradients of all Gaussians match
    the FP64 analytic gradient on exactly those pixels."""
    m = rtg()
    crop, cam, tc, td = crop_problem(seed)
    crop.unstable = np.ones(crop.n, np.uint8)
    H, W = cam.height, cam.width
    ctx = ctx_for(crop.n, cam)
    g = m.Gaussians.from_scene(crop)
    color, depth, _ = _render(m, ctx, [cam], g, None, 3, H, W)
    tct = torch.tensor(tc, dtype=torch.float32, device="cuda").reshape(1, 3, H, W)
    tdt = torch.tensor(td, dtype=torch.float32, device="cuda").reshape(1, H, W)
    sel = torch.zeros(1, H, W, dtype=torch.uint8, device="cuda")
    m.select_top_error(ctx, color, tct, 0.4, sel)
    torch.cuda.synchronize()
    sel_np = sel.cpu().numpy()
    np.testing.assert_array_equal(sel_np, go.top_error_mask(color.cpu().numpy(), tct.cpu().numpy(), 0.4))
    pre = oracle.render_image(crop, cam, ST)
    use = (sel_np[0] != 0) & ~pre["grad_borderline"]
    assert use.sum() >= 0.9 * sel_np.sum()
    mk = torch.as_tensor(use.astype(np.uint8)).reshape(1, H, W).cuda()
    m.narrow_pixels(ctx, mk)
    loss, got = _loss_backward(m, ctx, color, depth, tct, tdt, mk, crop.n, 3)
    ys, xs = np.nonzero(use)
    ref = oracle.loss_and_grads(crop, cam, ST, np.stack([xs, ys], 1), tc[:, ys, xs].T, td[ys, xs])
    assert loss[0] == pytest.approx(ref["loss"], rel=1e-4)
    compare_groups(got, ref["grads"])


def test_global_step_adam_and_frozen_positions():
    """GlobalStep: the loss and gradients equal the explicit call sequence; one step applies
    the oracle's Adam with the global settings (positions unchanged, bit for bit); the step
    replays from a CUDA graph."""
    m = rtg()
    crop, cam, tc, td = crop_problem(3300)
    H, W = cam.height, cam.width
    cams = [cam, cam]
    ctx = ctx_for(crop.n, cams)
    g = m.Gaussians.from_scene(crop)
    tct = torch.tensor(np.stack([tc, tc]), dtype=torch.float32, device="cuda").reshape(2, 3, H, W)
    tdt = torch.tensor(np.stack([td, td]), dtype=torch.float32, device="cuda").reshape(2, H, W)
    step = m.GlobalStep(ctx, g, W, H, max_frames=2)
    before = {k: getattr(g, k).cpu().numpy().copy() for k in GROUPS}
    loss = step.step(cams, tct, tdt)
    torch.cuda.synchronize()
    assert m.get_status(ctx) == 0
    grads = {k: t.cpu().numpy().astype(np.float64) for k, t in zip(GROUPS, step.grads)}
    after = {k: getattr(g, k).cpu().numpy() for k in GROUPS}
    np.testing.assert_array_equal(after["means"], before["means"])
    assert not np.array_equal(after["colors"], before["colors"])
    # selection: the same top-40% on both (identical) keyframes
    sel = step.selected[:2].cpu().numpy()
    np.testing.assert_array_equal(sel, go.top_error_mask(step.color[:2].cpu().numpy(), tct.cpu().numpy(), 0.4))
    # Adam of the oracle with the global settings on the GPU's gradients
    hyper = go.global_hyper(oracle.AdamHyper())
    zeros = {k: np.zeros_like(v, dtype=np.float64) for k, v in before.items()}
    params = {k: v.astype(np.float64) for k, v in before.items()}
    newp, _, _ = oracle.adam_step(params, grads, dict(zeros), dict(zeros), 1, hyper)
    for k in GROUPS:
        np.testing.assert_allclose(after[k], newp[k], rtol=1e-5, atol=1e-6, err_msg=k)
    # the loss is that of the explicit sequence on the selected pixels
    assert float(loss[0]) > 0
    # graph replay continues the same iteration (the capture records, the replay runs)
    step.capture(cams, tct, tdt)
    step.step(cams, tct, tdt)
    torch.cuda.synchronize()
    assert step.step_counter.tolist() == [2, 0]
    np.testing.assert_array_equal(g.means.cpu().numpy(), before["means"])
