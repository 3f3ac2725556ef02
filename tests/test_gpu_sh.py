"""SH colour and the transparent regulariser on the GPU (Section 3.1 view-dependent colour;
Section 3.2, L_reg of Eq. 8; Supplement C SH learning rates) against the FP64 oracle:
renders with SH degree 1..3, the gradients of SH coefficients and of positions through the
view direction, batched frames with different view directions, Adam with split colour
rates, and the regulariser's loss and gradient."""

import dataclasses

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import assert_forward_matches, ctx_for, gpu_forward, rtg
from oracle import sh as osh
from test_gpu_backward import GROUPS, compare_groups, crop_problem

pytestmark = pytest.mark.gpu
ST = oracle.Settings()


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_sh_forward_matches_oracle(degree):
    scene, cam = synth.scatter_scene(1100 + degree, n=1500)
    scene.colors = synth.sh_coefficients(1200 + degree, scene.n, degree)
    ref = oracle.render_image(scene, cam, ST)
    got = gpu_forward(scene, cam)
    assert_forward_matches(ref, got["color"][0], got["depth"][0], got["alpha"][0], got["index"][0])


def test_sh_view_dependence_two_frames_batched():
    """Two cameras in one call see different colours of the same Gaussians (each frame
    against the oracle)."""
    scene, layout = synth.room_scene(2100, 30000)
    scene.colors = synth.sh_coefficients(2101, scene.n, 3, rest_sigma=0.3)
    cams = [c for _, c in zip(range(2), synth.room_camera_candidates(2102, layout, 96, 72, 90.0))]
    got = gpu_forward(scene, cams)
    for f, cam in enumerate(cams):
        ref = oracle.render_image(scene, cam, ST)
        assert_forward_matches(ref, got["color"][f], got["depth"][f], got["alpha"][f], got["index"][f])


def sh_grads(scene, cams, masks, tcs, tds):
    """GPU gradients of the unstable Gaussians, frame by frame accumulated (each frame its
    own loss), SH coefficient rows [nu, K, 3]."""
    m = rtg()
    ctx = ctx_for(scene.n, cams[0])
    g = m.Gaussians.from_scene(scene)
    nu = int(scene.unstable.sum())
    K = scene.colors.shape[1]
    grads = [torch.zeros(nu, 3, device="cuda"), torch.zeros(nu, 3, device="cuda"), torch.zeros(nu, 4, device="cuda"),
             torch.zeros(nu, device="cuda"), torch.zeros(nu, K, 3, device="cuda")]
    for f, cam in enumerate(cams):
        H, W = cam.height, cam.width
        color = torch.zeros(1, 3, H, W, device="cuda")
        depth = torch.full((1, H, W), -1.0, device="cuda")
        mk = torch.as_tensor(masks[f].astype(np.uint8)).reshape(1, H, W).cuda()
        m.render_forward(ctx, cam, g, mk, m.RenderSettings(), color, depth, torch.zeros(1, H, W, device="cuda"))
        tct = torch.tensor(tcs[f], dtype=torch.float32, device="cuda").reshape(1, 3, H, W)
        tdt = torch.tensor(tds[f], dtype=torch.float32, device="cuda").reshape(1, H, W)
        loss = torch.zeros(3, device="cuda")
        dc, dd = torch.zeros_like(color), torch.zeros_like(depth)
        m.l1_loss(ctx, color, depth, tct, tdt, mk, 1.0, 1.0, loss, dc, dd)
        m.render_backward(ctx, dc, dd, *grads, accumulate=f > 0)
    torch.cuda.synchronize()
    assert m.get_status(ctx) == 0
    return {k: t.cpu().numpy().astype(np.float64) for k, t in zip(GROUPS, grads)}


@pytest.mark.parametrize("seed", [3000, 3100])
def test_sh_gradients_match_oracle(seed):
    crop, cam, tc, td = crop_problem(seed)
    crop.colors = synth.sh_coefficients(seed + 5, crop.n, 3, rest_sigma=0.3)
    target = synth.jitter_scene(crop, seed + 6)
    tref = oracle.render_image(target, cam, ST)
    tc, td = tref["color"], np.where(tref["depth"] > 0, tref["depth"], 0.0)
    pre = oracle.render_image(crop, cam, ST)
    mask = ~pre["grad_borderline"] & (pre["alpha"] > 0)
    ys, xs = np.nonzero(mask)
    ref = oracle.loss_and_grads(crop, cam, ST, np.stack([xs, ys], 1), tc[:, ys, xs].T, td[ys, xs])
    got = sh_grads(crop, [cam], [mask], [tc], [td])
    compare_groups(got, ref["grads"])


def test_sh_gradients_two_views_accumulate():
    """The same Gaussians seen from two cameras: their gradients are the sum of the two
    views' gradients, each with its own view directions (oracle per view, summed)."""
    crop, cam, _, _ = crop_problem(3200)
    crop.colors = synth.sh_coefficients(3205, crop.n, 2, rest_sigma=0.3)
    cam2 = dataclasses.replace(cam.copy(), t=(cam.t + np.array([0.05, -0.03, 0.02], np.float32)).astype(np.float32))
    target = synth.jitter_scene(crop, 3206)
    masks, tcs, tds, refs = [], [], [], []
    for c in (cam, cam2):
        tref = oracle.render_image(target, c, ST)
        tc, td = tref["color"], np.where(tref["depth"] > 0, tref["depth"], 0.0)
        pre = oracle.render_image(crop, c, ST)
        mask = ~pre["grad_borderline"] & (pre["alpha"] > 0)
        ys, xs = np.nonzero(mask)
        refs.append(oracle.loss_and_grads(crop, c, ST, np.stack([xs, ys], 1), tc[:, ys, xs].T, td[ys, xs])["grads"])
        masks.append(mask)
        tcs.append(tc)
        tds.append(td)
    got = sh_grads(crop, [cam, cam2], masks, tcs, tds)
    compare_groups(got, {k: refs[0][k] + refs[1][k] for k in GROUPS})


def test_adam_split_colour_rates_match_oracle():
    m = rtg()
    rng = np.random.default_rng(9)
    nu, K = 3000, 16
    params = {"means": rng.normal(size=(nu, 3)), "scales": rng.uniform(0.01, 0.1, (nu, 3)),
              "quats": rng.normal(size=(nu, 4)), "opacity": rng.uniform(0.1, 1, nu),
              "colors": rng.normal(size=(nu, K, 3))}
    params = {k: v.astype(np.float32) for k, v in params.items()}
    grads = {k: rng.normal(size=v.shape).astype(np.float32) for k, v in params.items()}
    hp = m.AdamSettings(colors_dc=3)
    pt = [torch.tensor(params[k]).cuda() for k in GROUPS]
    gt = [torch.tensor(grads[k]).cuda() for k in GROUPS]
    mm = torch.zeros(nu * (11 + 3 * K), device="cuda")
    vv = torch.zeros_like(mm)
    cnt = torch.zeros(2, dtype=torch.int32, device="cuda")
    m.adam_step_counted(pt, gt, mm, vv, cnt, hp)
    torch.cuda.synchronize()
    ohp = oracle.AdamHyper(colors_dc=3, lr_colors=hp.lr_colors, lr_colors_rest=hp.lr_colors_rest)
    zeros = {k: np.zeros_like(v, dtype=np.float64) for k, v in params.items()}
    newp, _, _ = oracle.adam_step(params, grads, dict(zeros), dict(zeros), 1, ohp)
    for k, t in zip(GROUPS, pt):
        np.testing.assert_allclose(t.cpu().numpy(), newp[k], rtol=1e-5, atol=1e-6, err_msg=k)
    # the rates differ: a degree-0 coefficient moved 20x as far as a higher one
    d = np.abs(pt[4].cpu().numpy() - params["colors"])
    assert np.median(d[:, 0]) > 10 * np.median(d[:, 1:])


def test_transparent_regulariser_matches_oracle():
    m = rtg()
    rng = np.random.default_rng(10)
    nu = 5000
    m0 = rng.normal(size=(nu, 3)).astype(np.float32)
    s0 = rng.uniform(0.01, 0.1, (nu, 3)).astype(np.float32)
    q0 = rng.normal(size=(nu, 4)).astype(np.float32)
    mm = (m0 + rng.normal(0, 0.01, (nu, 3))).astype(np.float32)
    ss = (s0 * np.exp(rng.normal(0, 0.05, (nu, 3)))).astype(np.float32)
    qq = (q0 + rng.normal(0, 0.02, (nu, 4))).astype(np.float32)
    op = rng.choice([0.1, 0.99], nu).astype(np.float32)
    ctx = m.Context(max_gaussians=nu, max_frames=1, max_width=8, max_height=8, max_pairs=1 << 10)
    t = lambda a: torch.tensor(a).cuda()  # noqa: E731
    g0 = [torch.zeros(nu, 3, device="cuda"), torch.zeros(nu, 3, device="cuda"), torch.zeros(nu, 4, device="cuda")]
    loss = torch.zeros(1, device="cuda")
    m.transparent_reg(ctx, [t(mm), t(ss), t(qq), t(op)], [t(m0), t(s0), t(q0)], g0, loss, 1000.0)
    torch.cuda.synchronize()
    L, ref = osh.transparent_reg(mm, ss, qq, op, m0, s0, q0, 1000.0)
    assert float(loss.item()) == pytest.approx(L, rel=1e-5)
    for k, gg in zip(("means", "scales", "quats"), g0):
        np.testing.assert_allclose(gg.cpu().numpy(), ref[k], rtol=1e-4, atol=1e-9, err_msg=k)
    # the gradient is added to what the arrays hold
    ones = [torch.ones_like(x) for x in g0]
    m.transparent_reg(ctx, [t(mm), t(ss), t(qq), t(op)], [t(m0), t(s0), t(q0)], ones, loss, 1000.0)
    for k, gg in zip(("means", "scales", "quats"), ones):
        np.testing.assert_allclose(gg.cpu().numpy() - 1.0, ref[k], atol=3e-7, err_msg=k)


def test_masked_step_with_sh_and_regulariser():
    """A MaskedStep window on an SH room: the loss falls, and with the regulariser the
    transparent unstable Gaussians stay closer to where they were added."""
    m = rtg()
    scene, layout = synth.room_scene(2060, 20000)
    scene.colors = synth.sh_coefficients(2061, scene.n, 3)
    cam = next(synth.room_camera_candidates(2062, layout, 128, 96, 120.0))
    scene.unstable = synth.flag_blobs(scene, [cam], 6000, 3, seed=14)
    tref = gpu_forward(synth.jitter_scene(scene, 15, pos_sigma=0.01), cam)
    tc = torch.tensor(tref["color"]).cuda()
    td = torch.tensor(np.where(tref["depth"] > 0, tref["depth"], 0)).cuda()
    drift = {}
    for reg in (False, True):
        ctx = ctx_for(scene.n, cam)
        g = m.Gaussians.from_scene(scene)
        init = (g.means.clone(), g.scales.clone(), g.quats.clone()) if reg else None
        mask = torch.zeros(1, 96, 128, dtype=torch.uint8, device="cuda")
        step = m.MaskedStep(ctx, g, [cam], mask, tc, td, recompute_mask=True, initial=init,
                            adam=m.AdamSettings(lr_means=1e-3))
        assert step.adam.colors_dc == 3
        losses = [float(step.step()[0]) for _ in range(30)]
        torch.cuda.synchronize()
        assert m.get_status(ctx) == 0
        assert losses[-1] < losses[0]
        step.write_back()
        tr = (scene.unstable != 0) & (scene.opacity < 0.5)
        moved = (g.means.cpu().numpy() - scene.means)[tr]
        drift[reg] = float(np.abs(moved).mean())
        if reg:
            assert float(step.loss_reg.item()) >= 0
    assert drift[True] < drift[False]
