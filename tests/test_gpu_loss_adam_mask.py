"""GPU L1 loss, Adam and unstable-pixel mask vs the oracle; the full MaskedStep; device-side
capacity overflow reported without a hang."""

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import ctx_for, gpu_forward, rtg

pytestmark = pytest.mark.gpu
ST = oracle.Settings()


def test_l1_loss_matches_oracle():
    m = rtg()
    rng = np.random.default_rng(1)
    F, C, H, W = 2, 3, 37, 53
    color = rng.uniform(0, 1, (F, C, H, W)).astype(np.float32)
    depth = np.where(rng.random((F, H, W)) < 0.2, -1.0, rng.uniform(1, 5, (F, H, W))).astype(np.float32)
    tcol = rng.uniform(0, 1, (F, C, H, W)).astype(np.float32)
    tdep = np.where(rng.random((F, H, W)) < 0.1, 0.0, rng.uniform(1, 5, (F, H, W))).astype(np.float32)
    mask = (rng.random((F, H, W)) < 0.6).astype(np.uint8)
    ctx = ctx_for(10, synth.identity_camera(W, H, 50, 10, 10), channels=3)
    t = lambda a: torch.tensor(a).cuda()  # noqa: E731
    loss = torch.zeros(3, device="cuda")
    dc, dd = torch.zeros(F, C, H, W, device="cuda"), torch.zeros(F, H, W, device="cuda")
    m.l1_loss(ctx, t(color), t(depth), t(tcol), t(tdep), t(mask), 1.0, 1.0, loss, dc, dd)
    sel = mask.astype(bool)
    L, Lc, Ld, P, Pd = oracle.l1_loss(np.moveaxis(color, 1, -1)[sel], depth[sel], np.moveaxis(tcol, 1, -1)[sel],
                                      tdep[sel])
    got = loss.cpu().numpy()
    assert got == pytest.approx([float(L), float(Lc), float(Ld)], rel=1e-5)
    # gradient images: sign / count on the masked (and depth-valid) pixels, zero elsewhere
    sgn = np.sign(color - tcol) * sel[:, None]
    np.testing.assert_allclose(dc.cpu().numpy(), sgn / (P * C), rtol=1e-6)
    vd = sel & (depth != -1) & (tdep > 0)
    np.testing.assert_allclose(dd.cpu().numpy(), np.sign(depth - tdep) * vd / Pd, rtol=1e-6)


def test_adam_matches_oracle_three_steps():
    """Three Adam steps on 1,000 compact Gaussians; the oracle runs Algorithm 1 in FP64 on the
    same gradients (scale in log space)."""
    m = rtg()
    rng = np.random.default_rng(2)
    nu, C = 1000, 3
    p = dict(means=rng.normal(size=(nu, 3)), scales=np.exp(rng.normal(-4, 0.5, (nu, 3))),
             quats=rng.normal(size=(nu, 4)), opacity=rng.uniform(0, 1, nu), colors=rng.uniform(0, 1, (nu, 3)))
    p = {k: v.astype(np.float32) for k, v in p.items()}
    tp = [torch.tensor(p[k]).cuda() for k in oracle.adam.GROUPS]
    mm = torch.zeros(nu, 11 + C, device="cuda")
    vv = torch.zeros(nu, 11 + C, device="cuda")
    hp = oracle.AdamHyper()
    cur = {k: v.astype(np.float64) for k, v in p.items()}
    om = {k: np.zeros_like(v) for k, v in cur.items()}
    ov = {k: np.zeros_like(v) for k, v in cur.items()}
    for step in range(1, 4):
        gr = {k: rng.normal(size=v.shape).astype(np.float32) for k, v in p.items()}
        m.adam_step(tp, [torch.tensor(gr[k]).cuda() for k in oracle.adam.GROUPS], mm, vv, step)
        cur, om, ov = oracle.adam_step(cur, gr, om, ov, step, hp)
        torch.cuda.synchronize()
        for k, t in zip(oracle.adam.GROUPS, tp):
            np.testing.assert_allclose(t.cpu().numpy(), cur[k], rtol=1e-5, atol=1e-6, err_msg=f"{k} step {step}")


def test_unstable_mask_matches_oracle():
    m = rtg()
    scene, layout = synth.room_scene(2020, 20000)
    cam = next(synth.room_camera_candidates(2021, layout, 120, 90, 110.0))
    scene.unstable = synth.flag_blobs(scene, [cam], 4000, 3, seed=5)
    for frac in (0.0, 0.5):
        st = oracle.Settings(tile_discard_frac=frac)
        ref, border = oracle.unstable_mask(scene, cam, st)
        ctx = ctx_for(scene.n, cam)
        out = torch.zeros(1, cam.height, cam.width, dtype=torch.uint8, device="cuda")
        m.unstable_mask(ctx, cam, m.Gaussians.from_scene(scene), m.RenderSettings(tile_discard_frac=frac), out)
        got = out[0].cpu().numpy().astype(bool)
        assert border.mean() < 0.01
        np.testing.assert_array_equal(got[~border], ref[~border])
        assert 0.05 < ref.mean() < 0.95


def test_masked_step_reduces_loss_and_keeps_stable_fixed():
    m = rtg()
    scene, layout = synth.room_scene(2030, 20000)
    cam = next(synth.room_camera_candidates(2031, layout, 128, 96, 120.0))
    scene.unstable = synth.flag_blobs(scene, [cam], 4000, 3, seed=6)
    target = synth.jitter_scene(scene, 7)
    tref = gpu_forward(target, cam)  # a fixed target input for the loss (not a compared value)
    ctx = ctx_for(scene.n, cam)
    g = m.Gaussians.from_scene(scene)
    mask = torch.zeros(1, 96, 128, dtype=torch.uint8, device="cuda")
    m.unstable_mask(ctx, cam, g, m.RenderSettings(), mask)
    tc = torch.tensor(tref["color"]).cuda()
    td = torch.tensor(np.where(tref["depth"] > 0, tref["depth"], 0)).cuda()
    stable_before = g.means[g.unstable == 0].clone()
    step = m.MaskedStep(ctx, g, [cam], mask, tc, td)
    losses = [float(step.step()[0]) for _ in range(30)]
    assert losses[-1] < losses[0]
    step.write_back()
    torch.cuda.synchronize()
    assert torch.equal(g.means[g.unstable == 0], stable_before)
    assert m.get_status(ctx) == 0


def test_pair_overflow_is_reported_and_outputs_untouched():
    m = rtg()
    scene, cam = synth.scatter_scene(1000, n=2000)
    ctx = ctx_for(scene.n, cam, max_pairs=100)
    g = m.Gaussians.from_scene(scene)
    color = torch.full((1, 3, cam.height, cam.width), 7.0, device="cuda")
    depth = torch.full((1, cam.height, cam.width), 7.0, device="cuda")
    alpha = torch.full((1, cam.height, cam.width), 7.0, device="cuda")
    m.render_forward(ctx, cam, g, None, m.RenderSettings(), color, depth, alpha)
    torch.cuda.synchronize()
    assert m.get_status(ctx) == m._lib.RTG_ERR_WORKSPACE
    assert (color == 7.0).all() and (depth == 7.0).all()
    m.reset_status(ctx)
    assert m.get_status(ctx) == 0


def test_argument_errors_raise():
    m = rtg()
    scene, cam = synth.scatter_scene(1000, n=100)
    ctx = ctx_for(scene.n, cam)
    g = m.Gaussians.from_scene(scene)
    out = [torch.zeros(1, 3, 120, 160, device="cuda"), torch.zeros(1, 120, 160, device="cuda"),
           torch.zeros(1, 120, 160, device="cuda")]
    big = synth.identity_camera(4000, 120, 150, 79.5, 59.5)
    with pytest.raises(m.RTGError):
        m.render_forward(ctx, big, g, None, m.RenderSettings(), *out)
    with pytest.raises(m.RTGError):
        m.render_forward(ctx, cam, g, None, m.RenderSettings(alpha_min=0.0), *out)
    fresh = ctx_for(scene.n, cam)
    with pytest.raises(m.RTGError):  # backward before any forward
        m.render_backward(fresh, out[0], out[1], *[torch.zeros(1, device="cuda")] * 5)


def test_masked_step_graph_replay_matches_eager():
    """A captured iteration (mask, forward, loss, backward, counted Adam) replayed from a CUDA
    graph follows the same trajectory as eager iterations."""
    m = rtg()
    scene, layout = synth.room_scene(2040, 20000)
    cam = next(synth.room_camera_candidates(2041, layout, 128, 96, 120.0))
    scene.unstable = synth.flag_blobs(scene, [cam], 4000, 3, seed=8)
    tref = gpu_forward(synth.jitter_scene(scene, 9), cam)
    tc = torch.tensor(tref["color"]).cuda()
    td = torch.tensor(np.where(tref["depth"] > 0, tref["depth"], 0)).cuda()

    def make():
        ctx = ctx_for(scene.n, cam)
        g = m.Gaussians.from_scene(scene)
        mask = torch.zeros(1, 96, 128, dtype=torch.uint8, device="cuda")
        return m.MaskedStep(ctx, g, [cam], mask, tc, td, recompute_mask=True)

    eager, graphed = make(), make()
    la = [float(eager.step()[0]) for _ in range(6)]
    lb = [float(graphed.step()[0])]
    graphed.capture()
    lb += [float(graphed.step()[0]) for _ in range(5)]
    torch.cuda.synchronize()
    np.testing.assert_allclose(lb, la, rtol=1e-4)
    # the gradient rows are float32 atomic sums whose order differs between runs, and Adam
    # divides each gradient by its own running RMS: where a gradient is near zero, that order
    # decides the sign of a full step.  So almost every element must agree closely and the
    # whole arrays to 1e-4 of their norm.
    for a, b in zip(eager.u, graphed.u):
        a, b = a.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)
        assert (~np.isclose(b, a, rtol=1e-4, atol=1e-6)).mean() <= 1e-3
        assert np.linalg.norm(b - a) <= 1e-4 * np.linalg.norm(a)
    assert graphed.step_counter.tolist() == [6, 0] and eager.step_counter.tolist() == [6, 0]


def test_adam_after_gradients_equals_adam_step_counted():
    """rtg_adam_step_counted_after_gradients (parameter and moment loads issued before the
    wait on the kernel in front, which here writes the gradients) gives
    rtg_adam_step_counted's result bit for bit, ragged group ends and several rounds of the
    grid included."""
    m = rtg()
    rng = np.random.default_rng(7)
    for nu, C in ((1, 3), (1237, 3), (333_331, 3), (50_001, 8)):
        p = [torch.tensor(rng.normal(size=s).astype(np.float32)).cuda()
             for s in ((nu, 3), (nu, 3), (nu, 4), (nu,), (nu, C))]
        p[1] = p[1].abs() + 0.01
        mm = torch.tensor(rng.normal(size=nu * (11 + C)).astype(np.float32)).cuda() * 1e-3
        vv = torch.tensor(rng.uniform(0, 1e-4, nu * (11 + C)).astype(np.float32)).cuda()
        grads = [torch.zeros_like(t) for t in p]
        out = []
        for after in (False, True):
            q, a_m, a_v = [t.clone() for t in p], mm.clone(), vv.clone()
            cnt = torch.tensor([4, 0], dtype=torch.int32, device="cuda")
            for step in range(2):
                # the kernel in front writes the gradients (a fill per group)
                for k, g in enumerate(grads):
                    g.copy_(torch.sin(torch.arange(g.numel(), device="cuda", dtype=torch.float32) * (k + 1 + step))
                            .reshape(g.shape))
                m.adam_step_counted(q, grads, a_m, a_v, cnt, after_gradients=after)
            torch.cuda.synchronize()
            out.append((q, a_m, a_v, cnt.tolist()))
        for a, b in zip(out[0][0] + [out[0][1], out[0][2]], out[1][0] + [out[1][1], out[1][2]]):
            assert torch.equal(a, b)
        assert out[0][3] == out[1][3] == [6, 0]


def test_masked_step_scatter_every_step_keeps_full_arrays_current():
    """The renderer reads the unstable Gaussians from the optimiser's compact arrays; with
    scatter_every_step the full arrays follow them after every step, otherwise write_back()
    brings them up to date, and the stable rows never change."""
    m = rtg()
    scene, layout = synth.room_scene(2045, 20000)
    cam = next(synth.room_camera_candidates(2046, layout, 128, 96, 120.0))
    scene.unstable = synth.flag_blobs(scene, [cam], 4000, 3, seed=10)
    tref = gpu_forward(synth.jitter_scene(scene, 11), cam)
    tc = torch.tensor(tref["color"]).cuda()
    td = torch.tensor(np.where(tref["depth"] > 0, tref["depth"], 0)).cuda()
    for every in (True, False):
        ctx = ctx_for(scene.n, cam)
        g = m.Gaussians.from_scene(scene)
        before = g.means.clone()
        mask = torch.zeros(1, 96, 128, dtype=torch.uint8, device="cuda")
        step = m.MaskedStep(ctx, g, [cam], mask, tc, td, recompute_mask=True, scatter_every_step=every)
        for _ in range(3):
            step.step()
        torch.cuda.synchronize()
        u = g.unstable.bool()
        if not every:
            assert torch.equal(g.means, before)  # untouched until write_back
            step.write_back()
            torch.cuda.synchronize()
        assert torch.equal(g.means[u], step.u[0]) and not torch.equal(g.means[u], before[u])
        assert torch.equal(g.means[~u], before[~u])


def test_precomputed_unstable_index_is_bitwise_identical():
    import dataclasses
    m = rtg()
    scene, layout = synth.room_scene(2050, 20000)
    cam = next(synth.room_camera_candidates(2051, layout, 112, 80, 100.0))
    scene.unstable = synth.flag_blobs(scene, [cam], 3000, 3, seed=10)
    ctx = ctx_for(scene.n, cam)
    g = m.Gaussians.from_scene(scene)
    rank, ids, nu = m.unstable_rank(ctx, g.unstable)
    assert nu == int(scene.unstable.sum())
    np.testing.assert_array_equal(ids.cpu().numpy(), np.flatnonzero(scene.unstable))
    flags = scene.unstable.astype(np.int64)
    exp_rank = np.where(flags > 0, np.cumsum(flags) - 1, -1)
    np.testing.assert_array_equal(rank.cpu().numpy(), exp_rank)
    g2 = dataclasses.replace(g, rank_map=rank, unstable_ids=ids, n_unstable=nu)
    outs = []
    for gg in (g, g2):
        mask = torch.zeros(1, 80, 112, dtype=torch.uint8, device="cuda")
        m.unstable_mask(ctx, cam, gg, m.RenderSettings(), mask)
        col = torch.zeros(1, 3, 80, 112, device="cuda")
        dep = torch.full((1, 80, 112), -1.0, device="cuda")
        alp = torch.zeros(1, 80, 112, device="cuda")
        m.render_forward(ctx, cam, gg, mask, m.RenderSettings(), col, dep, alp)
        dc = torch.sign(col - 0.5) / 1000.0
        dd = torch.where(dep > 0, torch.ones_like(dep), torch.zeros_like(dep)) / 1000.0
        grads = [torch.zeros(nu, 3, device="cuda"), torch.zeros(nu, 3, device="cuda"), torch.zeros(nu, 4, device="cuda"),
                 torch.zeros(nu, device="cuda"), torch.zeros(nu, 3, device="cuda")]
        m.render_backward(ctx, dc, dd, *grads)
        torch.cuda.synchronize()
        outs.append([mask.cpu(), col.cpu(), dep.cpu()] + [t.cpu() for t in grads])
    for a, b in zip(outs[0][:3], outs[1][:3]):
        assert torch.equal(a, b)
    assert outs[0][0].float().mean() > 0.05
    # the gradient rows are float32 atomic sums whose order differs between the two runs; an
    # element whose contributions cancel can differ relatively more, so the bound is relative
    # to each group's largest magnitude
    for a, b in zip(outs[0][3:], outs[1][3:]):
        a, b = a.numpy().astype(np.float64), b.numpy().astype(np.float64)
        assert np.abs(b - a).max() <= 1e-5 * np.abs(a).max()


def test_fused_l1_forward_backward_match_separate_calls():
    """rtg_render_forward_l1 + rtg_render_backward_l1 give the loss and gradients of
    rtg_render_forward + rtg_l1_loss + rtg_render_backward."""
    m = rtg()
    scene, layout = synth.room_scene(2060, 20000)
    cam = next(synth.room_camera_candidates(2061, layout, 112, 80, 100.0))
    scene.unstable = synth.flag_blobs(scene, [cam], 3000, 3, seed=11)
    tref = gpu_forward(synth.jitter_scene(scene, 12), cam)
    tc = torch.tensor(tref["color"]).cuda()
    td = torch.tensor(np.where(tref["depth"] > 0, tref["depth"], 0)).cuda()
    ctx = ctx_for(scene.n, cam)
    g = m.Gaussians.from_scene(scene)
    mask = torch.zeros(1, 80, 112, dtype=torch.uint8, device="cuda")
    m.unstable_mask(ctx, cam, g, m.RenderSettings(), mask)
    nu = int(scene.unstable.sum())

    def bufs():
        return (torch.zeros(1, 3, 80, 112, device="cuda"), torch.full((1, 80, 112), -1.0, device="cuda"),
                torch.zeros(1, 80, 112, device="cuda"), torch.zeros(3, device="cuda"),
                [torch.zeros(nu, 3, device="cuda"), torch.zeros(nu, 3, device="cuda"),
                 torch.zeros(nu, 4, device="cuda"), torch.zeros(nu, device="cuda"), torch.zeros(nu, 3, device="cuda")])

    c1, d1, a1, l1, g1 = bufs()
    m.render_forward(ctx, cam, g, mask, m.RenderSettings(), c1, d1, a1)
    dc, dd = torch.zeros_like(c1), torch.zeros_like(d1)
    m.l1_loss(ctx, c1, d1, tc, td, mask, 1.0, 1.0, l1, dc, dd)
    m.render_backward(ctx, dc, dd, *g1)
    c2, d2, a2, l2, g2 = bufs()
    m.render_forward_l1(ctx, cam, g, mask, m.RenderSettings(), tc, td, 1.0, 1.0, c2, d2, a2, l2)
    m.render_backward_l1(ctx, *g2)
    torch.cuda.synchronize()
    assert torch.equal(c1, c2) and torch.equal(d1, d2)
    np.testing.assert_allclose(l2.cpu().numpy(), l1.cpu().numpy(), rtol=1e-5)
    # the gradient rows are float32 sums formed by atomics whose order varies between runs:
    # an element with cancellation differs by a few ulp of its largest terms, so the
    # absolute tolerance scales with the array's magnitude
    for a, b in zip(g1, g2):
        a, b = a.cpu().numpy(), b.cpu().numpy()
        np.testing.assert_allclose(b, a, rtol=1e-5, atol=1e-6 * float(np.abs(a).max()))
    assert float(l1[0]) > 0


def test_forward_masked_equals_mask_then_forward():
    """rtg_render_forward_masked gives bit for bit the mask of rtg_unstable_mask and the
    render of rtg_render_forward on it (and the fused loss of rtg_render_forward_l1)."""
    m = rtg()
    scene, layout = synth.room_scene(2070, 20000)
    cams = [c for _, c in zip(range(2), synth.room_camera_candidates(2071, layout, 112, 80, 100.0))]
    scene.unstable = synth.flag_blobs(scene, cams, 3000, 3, seed=13)
    tref = gpu_forward(synth.jitter_scene(scene, 14), cams)
    tc = torch.tensor(tref["color"]).cuda()
    td = torch.tensor(np.where(tref["depth"] > 0, tref["depth"], 0)).cuda()
    ctx = ctx_for(scene.n, cams)
    g = m.Gaussians.from_scene(scene)

    def bufs():
        return (torch.zeros(2, 80, 112, dtype=torch.uint8, device="cuda"), torch.zeros(2, 3, 80, 112, device="cuda"),
                torch.full((2, 80, 112), -1.0, device="cuda"), torch.zeros(2, 80, 112, device="cuda"),
                torch.full((2, 80, 112), -1, dtype=torch.int32, device="cuda"), torch.zeros(3, device="cuda"))

    mk1, c1, d1, a1, i1, l1 = bufs()
    m.unstable_mask(ctx, cams, g, m.RenderSettings(), mk1)
    m.render_forward_l1(ctx, cams, g, mk1, m.RenderSettings(), tc, td, 1.0, 1.0, c1, d1, a1, l1, i1)
    s1 = m.get_stats(ctx)
    mk2, c2, d2, a2, i2, l2 = bufs()
    m.render_forward_masked(ctx, cams, g, m.RenderSettings(), mk2, c2, d2, a2, tc, td, 1.0, 1.0, l2, i2)
    s2 = m.get_stats(ctx)
    torch.cuda.synchronize()
    for a, b in ((mk1, mk2), (c1, c2), (d1, d2), (a1, a2), (i1, i2), (l1, l2)):
        assert torch.equal(a, b)
    assert s1["pairs"] == s2["pairs"] and s1["fragments"] == s2["fragments"] and s1["visible"] == s2["visible"]
    assert s2["masked_pixels"] == int(mk2.sum()) > 0 and s2["status"] == 0
