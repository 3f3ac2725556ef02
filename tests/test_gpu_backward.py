"""GPU backward (rtg_l1_loss + rtg_render_backward) vs the oracle's analytic FP64 gradient
and its central finite differences, on a 200-Gaussian crop of the room workload."""

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import ctx_for, rtg

pytestmark = pytest.mark.gpu
ST = oracle.Settings()
GROUPS = ("means", "scales", "quats", "opacity", "colors")


def crop_problem(seed, n_keep=200, win=48, frac_unstable=0.5):
    """200 surfels nearest to a visible surface point, seen by a win x win camera at the
    640x480 camera's position aimed at that point (focal length 600 kept)."""
    import math
    scene, layout = synth.room_scene(seed, 60000)
    cams = synth.room_camera_candidates(seed + 1, layout)
    rng = np.random.default_rng(seed)
    p = scene.means.astype(np.float64)
    while True:
        cam = next(cams)
        pc = (p - cam.t.astype(np.float64)) @ cam.R.astype(np.float64)
        with np.errstate(divide="ignore", invalid="ignore"):
            u = cam.fx * pc[:, 0] / pc[:, 2] + cam.cx
            v = cam.fy * pc[:, 1] / pc[:, 2] + cam.cy
        vis = (pc[:, 2] > 0.8) & (np.abs(u - 320) < 150) & (np.abs(v - 240) < 100) & (scene.opacity > 0.5)
        if vis.sum() > 100:
            break
    c = rng.choice(np.flatnonzero(vis))
    d = np.linalg.norm(p - p[c], axis=1)
    keep = np.sort(np.argpartition(d, n_keep)[:n_keep])
    crop = scene.subset(keep)
    crop.unstable = (rng.random(n_keep) < frac_unstable).astype(np.uint8)
    ray = p[c] - cam.t.astype(np.float64)
    ray /= np.linalg.norm(ray)
    wcam = synth.look_at_camera(cam.t, math.atan2(ray[1], ray[0]), math.asin(ray[2]), win, win, cam.fx)
    target = synth.jitter_scene(crop, seed + 2)
    tref = oracle.render_image(target, wcam, ST)
    tc = tref["color"]
    td = np.where(tref["depth"] > 0, tref["depth"], 0.0)
    return crop, wcam, tc, td


def gpu_grads(scene, cam, mask, tc, td, w_c=1.0, w_d=1.0, tuning=None, stats=None):
    m = rtg()
    H, W = cam.height, cam.width
    ctx = ctx_for(scene.n, cam)
    if tuning is not None:
        ctx.set_tuning(tuning)
    g = m.Gaussians.from_scene(scene)
    color = torch.zeros(1, 3, H, W, device="cuda")
    depth = torch.full((1, H, W), -1.0, device="cuda")
    alpha = torch.zeros(1, H, W, device="cuda")
    mk = torch.as_tensor(mask.astype(np.uint8)).reshape(1, H, W).cuda()
    m.render_forward(ctx, cam, g, mk, m.RenderSettings(), color, depth, alpha)
    tct = torch.tensor(tc, dtype=torch.float32, device="cuda").reshape(1, 3, H, W)
    tdt = torch.tensor(td, dtype=torch.float32, device="cuda").reshape(1, H, W)
    loss = torch.zeros(3, device="cuda")
    dc, dd = torch.zeros_like(color), torch.zeros_like(depth)
    m.l1_loss(ctx, color, depth, tct, tdt, mk, w_c, w_d, loss, dc, dd)
    nu = int(scene.unstable.sum())
    grads = [torch.zeros(nu, 3, device="cuda"), torch.zeros(nu, 3, device="cuda"), torch.zeros(nu, 4, device="cuda"),
             torch.zeros(nu, device="cuda"), torch.zeros(nu, 3, device="cuda")]
    m.render_backward(ctx, dc, dd, *grads)
    torch.cuda.synchronize()
    assert m.get_status(ctx) == 0
    if stats is not None:
        stats.update(m.get_stats(ctx))
    return {k: t.cpu().numpy().astype(np.float64) for k, t in zip(GROUPS, grads)}, loss.cpu().numpy()


def compare_groups(got, ref, rel=1e-3):
    for k in GROUPS:
        r, gg = ref[k].reshape(len(ref[k]), -1), got[k].reshape(len(got[k]), -1)
        scale = np.abs(r).max()
        if scale == 0:
            assert np.abs(gg).max() == 0, k
            continue
        assert np.linalg.norm(gg - r) <= rel * np.linalg.norm(r), (k, np.linalg.norm(gg - r) / np.linalg.norm(r))
        assert (np.abs(gg - r) <= rel * np.abs(r) + rel * scale).all(), (k, np.abs(gg - r).max(), scale)


@pytest.mark.parametrize("seed", [3000, 3100])
def test_gradients_match_oracle_analytic(seed):
    crop, cam, tc, td = crop_problem(seed)
    H, W = cam.height, cam.width
    pre = oracle.render_image(crop, cam, ST)
    mask = ~pre["grad_borderline"] & (pre["alpha"] > 0)
    ys, xs = np.nonzero(mask)
    pix = np.stack([xs, ys], 1)
    ref = oracle.loss_and_grads(crop, cam, ST, pix, tc[:, ys, xs].T, td[ys, xs])
    got, loss = gpu_grads(crop, cam, mask, tc, td)
    assert loss[0] == pytest.approx(ref["loss"], rel=1e-4)
    compare_groups(got, ref["grads"])


@pytest.mark.parametrize("batch", [32, 64])
def test_long_lists_replayed_in_segments_match_oracle(batch):
    """The persistent backward takes each 32-pixel group's list in segments of 64 entries
    (the eighth running to the end of the list), each started from the forward's checkpoint
    of the transmission and of the colour in front of it.  On a deep stack of faint
    Gaussians, where pixels walk 500-900 list entries before their transmission runs out,
    its gradients match the FP64 oracle's, and those of the whole-list replay of the
    per-tile schedule to float32 rounding."""
    m = rtg()
    scene, cam = synth.stack_scene(4100)
    H, W = cam.height, cam.width
    pre = oracle.render_image(scene, cam, ST)
    assert pre["n_proc"].max() > 8 * 64  # fragments reach the open-ended last segment
    mask = ~pre["grad_borderline"] & (pre["alpha"] > 0)
    rng = np.random.default_rng(4101)
    tc = rng.uniform(0, 1, (3, H, W))
    td = rng.uniform(1.5, 3.0, (H, W))
    ys, xs = np.nonzero(mask)
    ref = oracle.loss_and_grads(scene, cam, ST, np.stack([xs, ys], 1), tc[:, ys, xs].T, td[ys, xs])
    st = {}
    seg, loss = gpu_grads(scene, cam, mask, tc, td, tuning=m.Tuning(8, 8, batch, 1, 2, 8, 512), stats=st)
    assert st["max_tile_pairs"] > 8 * 64
    assert loss[0] == pytest.approx(ref["loss"], rel=1e-4)
    compare_groups(seg, ref["grads"])
    whole, _ = gpu_grads(scene, cam, mask, tc, td, tuning=m.Tuning(8, 8, batch, 0, 4, 8, 512))
    for k in GROUPS:
        scale = np.abs(whole[k]).max()
        assert scale > 0
        assert np.abs(seg[k] - whole[k]).max() <= 1e-4 * scale, (k, np.abs(seg[k] - whole[k]).max(), scale)


def test_gradients_match_finite_differences():
    """The 200-Gaussian crop (48 x 48 pixels): every parameter of 12 unstable Gaussians per
    group, drawn among those that reach a compared pixel, against FP64 central differences
    of the oracle's loss (parameters whose +-h perturbation changes a pixel's decision
    signature are left out)."""
    crop, cam, tc, td = crop_problem(3000)
    pre = oracle.render_image(crop, cam, ST)
    mask = ~pre["grad_borderline"] & (pre["alpha"] > 0)
    ys, xs = np.nonzero(mask)
    pix = np.stack([xs, ys], 1)
    got, _ = gpu_grads(crop, cam, mask, tc, td)
    uns = np.flatnonzero(crop.unstable)
    ref = oracle.loss_and_grads(crop, cam, ST, pix, tc[:, ys, xs].T, td[ys, xs])
    reach = np.flatnonzero(np.any(np.concatenate(
        [ref["grads"][k].reshape(len(uns), -1) for k in GROUPS], 1) != 0, axis=1))
    assert len(reach) >= 24, len(reach)
    rng = np.random.default_rng(0)
    which, gvals = [], []
    for name, width in (("means", 3), ("scales", 3), ("quats", 4), ("opacity", 1), ("colors", 3)):
        gmat = got[name].reshape(len(uns), -1)
        for k in rng.choice(reach, size=12, replace=False):
            for comp in range(width):
                which.append((name, uns[k], comp))
                gvals.append(gmat[k, comp])
    fd, stable = oracle.finite_difference_grads(crop, cam, ST, pix, tc[:, ys, xs].T, td[ys, xs], which)
    gvals = np.array(gvals)
    assert stable.mean() > 0.8
    assert (np.abs(fd[stable]) > 0).mean() > 0.8  # the drawn parameters do move the loss
    scale = np.abs(fd[stable]).max()
    err = np.abs(gvals - fd)[stable]
    assert (err <= 1e-3 * np.abs(fd[stable]) + 1e-3 * scale).all(), err.max() / scale


def test_gradient_special_cases_on_gpu():
    """Peak pixel: dL/dc = alpha / 3 and dL/dalpha = sum(c) / 3 under L = mean_c |C - 0|;
    fronto-parallel opaque disc under a depth-only loss: dL/dz = 1, dL/dx = dL/dy = 0."""
    cam = synth.identity_camera(33, 33, 40.0, 16.0, 16.0)
    c = np.array([0.2, 0.5, 0.9], np.float32)
    one = synth.Scene(means=np.array([[0, 0, 2.0]], np.float32), scales=np.array([[0.05, 0.03, 0.01]], np.float32),
                      quats=np.array([[1, 0, 0, 0]], np.float32), opacity=np.array([0.5], np.float32),
                      colors=c[None], unstable=np.ones(1, np.uint8))
    mask = np.zeros((33, 33), bool)
    mask[16, 16] = True
    got, _ = gpu_grads(one, cam, mask, np.zeros((3, 33, 33)), np.zeros((33, 33)), w_c=1.0, w_d=0.0)
    np.testing.assert_allclose(got["colors"][0], np.full(3, 0.5 / 3), rtol=1e-5)
    assert got["opacity"][0] == pytest.approx(float(c.sum()) / 3, rel=1e-5)
    disc = synth.disc_gaussian([0, 0, 2.0], [0, 0, 1], 0.1, 0.001, 0.99, [1, 1, 1])
    mask = np.zeros((33, 33), bool)
    mask[15:18, 15:18] = True
    got, _ = gpu_grads(disc, cam, mask, np.zeros((3, 33, 33)), np.ones((33, 33)), w_c=0.0, w_d=1.0)
    np.testing.assert_allclose(got["means"][0], [0.0, 0.0, 1.0], atol=1e-5)


def test_autograd_function_matches_direct_backward():
    m = rtg()
    crop, cam, tc, td = crop_problem(3300)
    g = m.Gaussians.from_scene(crop)
    ctx = ctx_for(crop.n, cam)
    ids, nu = m.unstable_index(ctx, g.unstable)
    leaves = [t.clone().requires_grad_(True) for t in m.gather_unstable(ids, g)]
    state = m.RasterState(ctx, g, [cam], None, m.RenderSettings())
    color, depth, alpha = m.rasterize(leaves, state)
    tct = torch.tensor(tc, dtype=torch.float32, device="cuda")[None]
    tdt = torch.tensor(td, dtype=torch.float32, device="cuda")[None]
    valid = (depth.detach() != -1) & (tdt > 0)
    loss = (color - tct).abs().mean() + ((depth - tdt).abs() * valid).sum() / valid.sum()
    loss.backward()
    pre = oracle.render_image(crop, cam, ST)
    ys, xs = np.nonzero(np.ones((cam.height, cam.width), bool))
    ref = oracle.loss_and_grads(crop, cam, ST, np.stack([xs, ys], 1), tc[:, ys, xs].T, td[ys, xs])
    if pre["grad_borderline"].any():
        pytest.skip("crop has borderline pixels; covered by the masked analytic test")
    compare_groups({k: leaf.grad.cpu().numpy().astype(np.float64) for k, leaf in zip(GROUPS, leaves)},
                   ref["grads"])
