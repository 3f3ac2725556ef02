"""The whole masked iteration (forward, fused L1 loss, backward, Adam) in its degenerate cases,
under both schedules and under graph replay:

- an empty mask: no pixel is optimised, so the loss is zero, every gradient is exactly zero
  and Adam, starting from zero moments, leaves every parameter bit for bit as it was
  (Section 3.2: the loss runs over the masked pixels only);
- no unstable Gaussian: nothing is optimised (the compact arrays are empty and the counted
  Adam step does nothing), while the forward still renders the stable Gaussians under the
  mask, equal bit for bit to a plain masked forward of the same scene.
"""

import numpy as np
import pytest
import torch

import synth
from gpu_util import rtg

pytestmark = pytest.mark.gpu

SCHEDULES = {"per-tile": (8, 8, 32, 0, 2, 8, 512, 1), "persistent": (8, 8, 32, 1, 2, 8, 512, 1)}


def scene_and_targets(seed, n, nu):
    m = rtg()
    scene, layout = synth.room_scene(seed, n)
    cam = next(synth.room_camera_candidates(seed + 1, layout, 320, 240, 240.0))
    scene.unstable = synth.flag_blobs(scene, [cam], nu, 3, seed=seed + 2) if nu else np.zeros(scene.n, np.uint8)
    H, W = cam.height, cam.width
    ctx = m.Context(max_gaussians=scene.n, max_width=W, max_height=H)
    tc = torch.zeros(1, 3, H, W, device="cuda")
    td = torch.full((1, H, W), -1.0, device="cuda")
    ref = m.Gaussians.from_scene(synth.jitter_scene(scene, seed + 3))
    m.render_forward(ctx, cam, ref, None, m.RenderSettings(), tc, td, torch.zeros(1, H, W, device="cuda"))
    td.clamp_(min=0)
    ctx.close()
    return scene, cam, tc, td


@pytest.mark.parametrize("schedule", sorted(SCHEDULES))
@pytest.mark.parametrize("graph", [False, True])
def test_empty_mask_changes_nothing(schedule, graph):
    m = rtg()
    scene, cam, tc, td = scene_and_targets(8300, 20000, 4000)
    H, W = cam.height, cam.width
    ctx = m.Context(max_gaussians=scene.n, max_width=W, max_height=H)
    ctx.set_tuning(m.Tuning(*SCHEDULES[schedule]))
    g = m.Gaussians.from_scene(scene)
    mask = torch.zeros(1, H, W, dtype=torch.uint8, device="cuda")
    step = m.MaskedStep(ctx, g, [cam], mask, tc, td)
    before = [t.clone() for t in step.u]
    assert step.nu == 4000
    step.step()
    if graph:
        step.capture()
        for _ in range(2):
            step.step()
    torch.cuda.synchronize()
    assert m.get_status(ctx) == 0
    assert step.loss.tolist() == [0.0, 0.0, 0.0]
    for t in step.grads:
        assert int(torch.count_nonzero(t)) == 0
    for a, b in zip(step.u, before):
        assert torch.equal(a, b)
    assert int(torch.count_nonzero(step.m)) == 0 and int(torch.count_nonzero(step.v)) == 0
    assert step.step_counter.tolist() == [3 if graph else 1, 0]
    ctx.close()


@pytest.mark.parametrize("schedule", sorted(SCHEDULES))
def test_no_unstable_gaussian_optimises_nothing_and_still_renders(schedule):
    m = rtg()
    scene, cam, tc, td = scene_and_targets(8400, 20000, 0)
    H, W = cam.height, cam.width
    rng = np.random.default_rng(8401)
    mask_np = np.zeros((1, H, W), np.uint8)  # a 96 x 64 rectangle plus scattered pixels
    mask_np[0, 40:104, 100:196] = 1
    mask_np[0][rng.random((H, W)) < 0.05] = 1
    mask = torch.from_numpy(mask_np).cuda()
    ctx = m.Context(max_gaussians=scene.n, max_width=W, max_height=H)
    ctx.set_tuning(m.Tuning(*SCHEDULES[schedule]))
    g = m.Gaussians.from_scene(scene)
    step = m.MaskedStep(ctx, g, [cam], mask, tc, td)
    assert step.nu == 0 and all(t.shape[0] == 0 for t in step.u)
    loss = step.step().clone()
    step.step()
    torch.cuda.synchronize()
    assert m.get_status(ctx) == 0
    assert step.step_counter.tolist() == [0, 0]  # the counted Adam step over no parameter does nothing
    assert torch.isfinite(loss).all() and float(loss[0]) > 0.0
    assert torch.equal(step.loss, loss)  # nothing moved, so the second iteration repeats the first
    ctx2 = m.Context(max_gaussians=scene.n, max_width=W, max_height=H)
    ctx2.set_tuning(m.Tuning(*SCHEDULES[schedule]))
    color = torch.zeros(1, 3, H, W, device="cuda")
    depth = torch.zeros(1, H, W, device="cuda")
    alpha = torch.zeros(1, H, W, device="cuda")
    m.render_forward(ctx2, cam, m.Gaussians.from_scene(scene), mask, m.RenderSettings(), color, depth, alpha)
    torch.cuda.synchronize()
    sel = mask.bool()
    assert int(sel.sum()) > 0
    assert torch.equal(step.state.color[sel.unsqueeze(1).expand_as(color)], color[sel.unsqueeze(1).expand_as(color)])
    assert torch.equal(step.state.depth[sel], depth[sel])
    assert torch.equal(step.state.alpha[sel], alpha[sel])
    ctx2.close()
    ctx.close()
