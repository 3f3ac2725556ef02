"""RGB-D frame decode (rtg_decode_rgbd) against the same conversion on the host, and a
masked step fed the sensor frame against one fed the decoded float planes."""

import numpy as np
import pytest
import torch

from gpu_util import rtg

pytestmark = pytest.mark.gpu


def host_decode(rgb, depth, scale):
    color = (rgb.astype(np.float32) / np.float32(255)).transpose(0, 3, 1, 2)
    return np.ascontiguousarray(color), depth.astype(np.float32) / np.float32(scale)


@pytest.mark.parametrize("F,H,W,scale", [(1, 7, 5, 5000.0), (1, 4, 6, 5000.0), (3, 33, 65, 1000.0),
                                         (2, 480, 640, 6553.5)])
def test_decode_matches_host_bit_for_bit(F, H, W, scale):
    m = rtg()
    rng = np.random.default_rng(F * H + W)
    rgb = rng.integers(0, 256, (F, H, W, 3), dtype=np.uint8)
    depth = rng.integers(0, 65536, (F, H, W), dtype=np.uint16)
    rgb[0, 0, 0] = (0, 255, 128)
    depth[0, 0, :2] = (0, 65535)
    color = torch.full((F, 3, H, W), -1.0, device="cuda")
    dout = torch.full((F, H, W), -1.0, device="cuda")
    m.decode_rgbd(torch.from_numpy(rgb).cuda(), torch.from_numpy(depth).cuda(), scale, color, dout)
    torch.cuda.synchronize()
    ref_c, ref_d = host_decode(rgb, depth, scale)
    assert np.array_equal(color.cpu().numpy(), ref_c)
    assert np.array_equal(dout.cpu().numpy(), ref_d)
    assert float(dout[0, 0, 0]) == 0.0


def test_decode_rejects_bad_shapes_and_types():
    m = rtg()
    rgb = torch.zeros(1, 4, 4, 3, dtype=torch.uint8, device="cuda")
    depth = torch.zeros(1, 4, 4, dtype=torch.uint16, device="cuda")
    color, dout = torch.zeros(1, 3, 4, 4, device="cuda"), torch.zeros(1, 4, 4, device="cuda")
    with pytest.raises(ValueError):
        m.decode_rgbd(rgb, torch.zeros(1, 4, 5, dtype=torch.uint16, device="cuda"), 1000.0, color, dout)
    with pytest.raises(TypeError):
        m.decode_rgbd(rgb, depth.to(torch.int32), 1000.0, color, dout)
    with pytest.raises(RuntimeError):
        m.decode_rgbd(rgb, depth, 0.0, color, dout)


def test_masked_step_from_sensor_frame_equals_decoded_targets():
    import synth
    m = rtg()
    scene, layout = synth.room_scene(515, 20000)
    cam = next(synth.room_camera_candidates(516, layout, 96, 72, 90.0))
    scene.unstable = synth.flag_blobs(scene, [cam], 3000, 2, seed=3)
    H, W = cam.height, cam.width
    ref = m.Gaussians.from_scene(synth.jitter_scene(scene, 9))
    ctx0 = m.Context(max_gaussians=scene.n, max_width=W, max_height=H)
    c = torch.zeros(1, 3, H, W, device="cuda")
    d = torch.full((1, H, W), -1.0, device="cuda")
    a = torch.zeros(1, H, W, device="cuda")
    m.render_forward(ctx0, cam, ref, None, m.RenderSettings(), c, d, a)
    rgb = (c[0].clamp(0, 1) * 255).round().to(torch.uint8).permute(1, 2, 0).contiguous().unsqueeze(0)
    dep = torch.where(d > 0, (d * 5000).round(), torch.zeros_like(d)).clamp(0, 65535).to(torch.int32)
    dep = dep.to(torch.uint16)
    out = []
    for use_frame in (False, True):
        ctx = m.Context(max_gaussians=scene.n, max_width=W, max_height=H)
        g = m.Gaussians.from_scene(scene)
        tc, td = torch.zeros(1, 3, H, W, device="cuda"), torch.zeros(1, H, W, device="cuda")
        if not use_frame:
            m.decode_rgbd(rgb, dep, 5000.0, tc, td)
        mask = torch.zeros(1, H, W, dtype=torch.uint8, device="cuda")
        step = m.MaskedStep(ctx, g, [cam], mask, tc, td, recompute_mask=True,
                            frame=(rgb, dep, 5000.0) if use_frame else None)
        loss = step.step().cpu().numpy().copy()  # the first loss: the forward of identical targets
        for _ in range(2):
            step.step()
        torch.cuda.synchronize()
        out.append((loss, tc.cpu().numpy(), td.cpu().numpy(), [t.cpu().numpy().copy() for t in step.u]))
    assert out[0][0][0] > 0
    np.testing.assert_array_equal(out[0][1], out[1][1])  # the step decoded the same planes
    np.testing.assert_array_equal(out[0][2], out[1][2])
    np.testing.assert_allclose(out[1][0], out[0][0], rtol=1e-6)
    # the parameters after three steps: the gradient rows are float32 atomics whose order
    # varies between runs
    for a_, b_ in zip(out[0][3], out[1][3]):
        np.testing.assert_allclose(b_, a_, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("uploads", [False, True])
def test_graphs_per_frame_set_equal_eager_steps(uploads):
    """MaskedStep.capture_frames: one graph per sensor-frame buffer set; replay(k) runs the
    iteration on set k and returns that set's loss.  Alternating two sets holding frames A and
    B gives the losses and parameters of eager steps on A, B, A, B; step() keeps its own
    graph and loss buffer.  With uploads, set 1 starts empty: graph 0 uploads B into it from
    pinned host memory while it computes on A, graph 1 uploads A back into set 0, and each
    graph copies its loss to its pinned host slot."""
    import synth
    m = rtg()
    scene, layout = synth.room_scene(535, 20000)
    cam = next(synth.room_camera_candidates(536, layout, 96, 72, 90.0))
    scene.unstable = synth.flag_blobs(scene, [cam], 3000, 2, seed=7)
    H, W = cam.height, cam.width
    rng = np.random.default_rng(537)
    frames = []
    for _ in range(2):
        rgb = torch.from_numpy(rng.integers(0, 256, (1, H, W, 3), dtype=np.uint8)).cuda()
        dep = torch.from_numpy(rng.integers(4000, 20000, (1, H, W)).astype(np.uint16)).cuda()
        frames.append((rgb, dep))
    runs = []
    for graphed in (False, True):
        ctx = m.Context(max_gaussians=scene.n, max_width=W, max_height=H)
        g = m.Gaussians.from_scene(scene)
        mask = torch.zeros(1, H, W, dtype=torch.uint8, device="cuda")
        m.unstable_mask(ctx, cam, g, m.RenderSettings(), mask)
        tc, td = torch.zeros(1, 3, H, W, device="cuda"), torch.zeros(1, H, W, device="cuda")
        own = (frames[0][0].clone(), frames[0][1].clone())
        step = m.MaskedStep(ctx, g, [cam], mask, tc, td, frame=(own[0], own[1], 5000.0))
        losses = []
        if graphed:
            sets = [[torch.zeros_like(f[0]), torch.zeros_like(f[1])] for f in frames]
            sets[0][0].copy_(frames[0][0])
            sets[0][1].copy_(frames[0][1])
            if uploads:
                hosts = [[frames[1][0].cpu().pin_memory(), frames[1][1].cpu().pin_memory()],
                         [frames[0][0].cpu().pin_memory(), frames[0][1].cpu().pin_memory()]]
                lh = [torch.full((3,), -1.0).pin_memory() for _ in range(2)]
                step.capture_frames(sets, uploads=hosts, loss_host=lh)
            else:
                sets[1][0].copy_(frames[1][0])
                sets[1][1].copy_(frames[1][1])
                step.capture_frames(sets)
            for k in (0, 1, 0, 1):
                out = step.replay(k)
                torch.cuda.synchronize()
                losses.append(out.cpu().numpy().copy())
                if uploads:
                    assert np.array_equal(lh[k].numpy(), losses[-1])
            if uploads:
                assert torch.equal(sets[1][0], frames[1][0]) and torch.equal(sets[0][1], frames[0][1])
            assert step.loss.data_ptr() not in [x.data_ptr() for x in step.frame_losses]
        else:
            for k in (0, 1, 0, 1):
                own[0].copy_(frames[k][0])
                own[1].copy_(frames[k][1])
                losses.append(step.step().cpu().numpy().copy())
        torch.cuda.synchronize()
        runs.append((losses, [t.cpu().numpy().copy() for t in step.u]))
        ctx.close()
    np.testing.assert_array_equal(runs[0][0][0], runs[1][0][0])  # the first forward: same parameters
    for a_, b_ in zip(runs[0][0][1:], runs[1][0][1:]):
        np.testing.assert_allclose(b_, a_, rtol=1e-5)
    for a_, b_ in zip(runs[0][1], runs[1][1]):  # float32 atomics order the gradient sums differently
        np.testing.assert_allclose(b_, a_, rtol=1e-4, atol=1e-6)


@pytest.mark.parametrize("tuning", [None, (8, 8, 32, 1, 2, 8, 512)])
def test_forward_l1_frame_equals_decode_then_forward(tuning):
    """rtg_render_forward_l1_frame (decode inside the forward call, the tile-mask pass
    running beside it) gives the targets of rtg_decode_rgbd and the render and loss of
    rtg_render_forward_l1 on them, bit for bit; two frames, a mask."""
    import synth
    m = rtg()
    scene, layout = synth.room_scene(616, 20000)
    cams = [c for _, c in zip(range(2), synth.room_camera_candidates(617, layout, 112, 80, 100.0))]
    scene.unstable = synth.flag_blobs(scene, cams, 3000, 3, seed=618)
    F, H, W = 2, 80, 112
    rng = np.random.default_rng(619)
    rgb = torch.from_numpy(rng.integers(0, 256, (F, H, W, 3), dtype=np.uint8)).cuda()
    dep = torch.from_numpy(rng.integers(0, 40000, (F, H, W), dtype=np.uint16)).cuda()
    g = m.Gaussians.from_scene(scene)
    outs = []
    for fused in (False, True):
        ctx = m.Context(max_gaussians=scene.n, max_frames=F, max_width=W, max_height=H)
        if tuning is not None:
            ctx.set_tuning(m.Tuning(*tuning))
        mask = torch.zeros(F, H, W, dtype=torch.uint8, device="cuda")
        m.unstable_mask(ctx, cams, g, m.RenderSettings(), mask)
        tc, td = torch.full((F, 3, H, W), -5.0, device="cuda"), torch.full((F, H, W), -5.0, device="cuda")
        c, d, a = torch.zeros(F, 3, H, W, device="cuda"), torch.zeros(F, H, W, device="cuda"), torch.zeros(F, H, W,
                                                                                                        device="cuda")
        idx = torch.full((F, H, W), -7, dtype=torch.int32, device="cuda")
        loss = torch.zeros(3, device="cuda")
        if fused:
            m.render_forward_l1_frame(ctx, cams, g, mask, m.RenderSettings(), rgb, dep, 5000.0, tc, td, 1.0, 0.5, c, d,
                                      a, loss, idx)
        else:
            m.decode_rgbd(rgb, dep, 5000.0, tc, td)
            m.render_forward_l1(ctx, cams, g, mask, m.RenderSettings(), tc, td, 1.0, 0.5, c, d, a, loss, idx)
        torch.cuda.synchronize()
        assert m.get_status(ctx) == 0 and int(mask.sum()) > 0
        outs.append([mask, tc, td, c, d, a, idx, loss])
        ctx.close()
    for x, y in zip(*outs):
        assert torch.equal(x, y)
    ref_c, ref_d = host_decode(rgb.cpu().numpy(), dep.cpu().numpy(), 5000.0)
    assert np.array_equal(outs[1][1].cpu().numpy(), ref_c) and np.array_equal(outs[1][2].cpu().numpy(), ref_d)


def test_forward_l1_frame_rejects_bad_frames():
    import synth
    m = rtg()
    cam = synth.identity_camera(32, 24, 30.0, 16.0, 12.0)
    scene, _ = synth.room_scene(620, 500)
    g = m.Gaussians.from_scene(scene)
    ctx = m.Context(max_gaussians=scene.n, max_width=32, max_height=24)
    rgb = torch.zeros(1, 24, 32, 3, dtype=torch.uint8, device="cuda")
    dep = torch.zeros(1, 24, 32, dtype=torch.uint16, device="cuda")
    planes = [torch.zeros(1, 3, 24, 32, device="cuda"), torch.zeros(1, 24, 32, device="cuda")]
    outs = [torch.zeros(1, 3, 24, 32, device="cuda"), torch.zeros(1, 24, 32, device="cuda"),
            torch.zeros(1, 24, 32, device="cuda"), torch.zeros(3, device="cuda")]
    with pytest.raises(m.RTGError):
        m.render_forward_l1_frame(ctx, cam, g, None, m.RenderSettings(), rgb, dep, 0.0, *planes, 1.0, 1.0, *outs)
    with pytest.raises(m.RTGError):
        m.render_forward_l1_frame(ctx, cam, g, None, m.RenderSettings(), rgb, dep, float("nan"), *planes, 1.0, 1.0,
                                  *outs)
    ctx.close()
