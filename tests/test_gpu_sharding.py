"""A keyframe batch split by frame (paper_2404_19706_b300.sharding) on one GPU.

The ranks' contexts are run one after the other in this process, with the two sums the
ranks' all-reduces would form taken by the test: the shares must add up to the gradient,
the loss and the Adam update of the batched call over all the frames (gradients to float32
atomic-order rounding), and one rank alone must equal MaskedStep.
"""

import dataclasses

import numpy as np
import pytest
import torch

import synth
from gpu_util import ctx_for, gpu_forward, rtg

pytestmark = pytest.mark.gpu

W, H, F = 136, 100, 4


def problem(seed=3300):
    scene, layout = synth.room_scene(seed, 20000)
    cams = [c for _, c in zip(range(F), synth.room_camera_candidates(seed + 1, layout, W, H, 110.0))]
    scene.unstable = synth.flag_blobs(scene, cams, 4000, 3, seed=seed + 2)
    m = rtg()
    g = m.Gaussians.from_scene(scene)
    ctx = ctx_for(scene.n, cams)
    masks = torch.zeros(F, H, W, dtype=torch.uint8, device="cuda")
    m.unstable_mask(ctx, cams, g, m.RenderSettings(), masks)
    ctx.close()
    ref = gpu_forward(synth.jitter_scene(scene, seed + 4), cams)
    tc = torch.tensor(ref["color"]).cuda()
    td = torch.tensor(np.where(ref["depth"] > 0, ref["depth"], 0)).cuda()
    ref["ctx"].close()
    assert int(masks.sum()) > 0
    return scene, cams, masks, tc, td


def group_close(a, b, rel=2e-5):
    """Equal to float32 summation-order rounding, relative to the group's largest value."""
    a, b = a.detach().cpu().numpy(), b.detach().cpu().numpy()
    scale = max(np.abs(a).max(initial=0), np.abs(b).max(initial=0), 1e-30)
    assert np.abs(a - b).max(initial=0) <= rel * scale, f"max diff {np.abs(a - b).max():.3e} of {scale:.3e}"


def batched_reference(scene, cams, masks, tc, td):
    """MaskedStep over all frames: one forward/backward call, one Adam step."""
    m = rtg()
    ctx = ctx_for(scene.n, cams)
    step = m.MaskedStep(ctx, m.Gaussians.from_scene(scene), cams, masks, tc, td)
    step.step()
    torch.cuda.synchronize()
    out = dict(loss=step.loss.clone(), grads=[t.clone() for t in step.grads], params=[t.clone() for t in step.u])
    ctx.close()
    return out


def test_one_rank_equals_masked_step():
    m = rtg()
    from paper_2404_19706_b300.sharding import FrameShardedStep
    scene, cams, masks, tc, td = problem()
    ref = batched_reference(scene, cams, masks, tc, td)
    ctx = ctx_for(scene.n, cams)
    sh = FrameShardedStep(ctx, m.Gaussians.from_scene(scene), cams, masks, tc, td, rank=0, world=1)
    sh.step()
    torch.cuda.synchronize()
    assert m.get_status(ctx) == 0
    # the same kernels on the same inputs, but the gradient rows are float32 atomic sums whose
    # order changes from run to run, so two runs agree to that rounding only
    for a, b in zip(sh.grads, ref["grads"]):
        group_close(a, b)
    for a, b in zip(sh.params, ref["params"]):
        group_close(a, b, rel=1e-5)
    np.testing.assert_allclose(sh.loss.cpu().numpy(), ref["loss"].cpu().numpy(), rtol=1e-6)
    ctx.close()


@pytest.mark.parametrize("world", [2, 3])
def test_rank_shares_sum_to_the_batched_call(world):
    m = rtg()
    from paper_2404_19706_b300.sharding import FrameShardedStep
    scene, cams, masks, tc, td = problem()
    ref = batched_reference(scene, cams, masks, tc, td)
    ranks = []
    for r in range(world):
        ctx = ctx_for(scene.n, cams)
        ranks.append(FrameShardedStep(ctx, m.Gaussians.from_scene(scene), cams, masks, tc, td, rank=r, world=world))
    # the iteration's five stages, with the two all-reduces formed here
    for s in ranks:
        s.forward()
    total = sum(s.counts for s in ranks)
    for s in ranks:
        s.counts.copy_(total)
        s.backward()
    grad = sum(s.flat for s in ranks)
    for s in ranks:
        s.flat.copy_(grad)
        s.apply()
    torch.cuda.synchronize()
    for s in ranks:
        assert m.get_status(s.ctx) == 0
    assert [len(range(F)[s.frames]) for s in ranks] == [len(x) for x in np.array_split(np.arange(F), world)]
    np.testing.assert_allclose(ranks[0].loss.cpu().numpy(), ref["loss"].cpu().numpy(), rtol=2e-5)
    for a, b in zip(ranks[0].grads, ref["grads"]):
        group_close(a, b)
    # replicated Adam: every rank holds the same parameters, equal to the batched step's
    for s in ranks[1:]:
        for a, b in zip(s.params, ranks[0].params):
            assert torch.equal(a, b)
    for a, b in zip(ranks[0].params, ref["params"]):
        group_close(a, b, rel=1e-5)
    for s in ranks:
        s.ctx.close()


def test_rank_share_needs_a_forward_with_targets():
    m = rtg()
    scene, cams, masks, tc, td = problem()
    ctx = ctx_for(scene.n, cams)
    counts = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(m.RTGError):
        m.loss_counts(ctx, counts)
    with pytest.raises(m.RTGError):
        m.set_loss_scales(ctx, counts, 1.0, 1.0)
    ctx.close()
