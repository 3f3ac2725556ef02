"""Pins for the FP64 oracle: closed forms, invariants and special cases that the paper's
definitions (Section 3.1 Eq. 1-5, Section 3.2 Eq. 7, Supplement B) fix independently of
the oracle's own code.  CPU only."""

import json
import math
import os

import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

import oracle
import synth
from oracle.rasterizer import Settings, project

ST = Settings()
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def quat_wxyz(R):
    x, y, z, w = Rotation.from_matrix(R).as_quat()
    return np.array([w, x, y, z])


def one_gaussian(mean, scales, quat, alpha, color):
    return synth.Scene(means=np.asarray(mean, np.float32).reshape(1, 3),
                       scales=np.asarray(scales, np.float32).reshape(1, 3),
                       quats=np.asarray(quat, np.float32).reshape(1, 4),
                       opacity=np.array([alpha], np.float32),
                       colors=np.asarray(color, np.float32).reshape(1, -1),
                       unstable=np.ones(1, np.uint8))


def cat(*scenes):
    return synth.concat_scenes(scenes)


def small_cam(W=32, H=32, f=40.0):
    return synth.identity_camera(W, H, f, (W - 1) / 2, (H - 1) / 2)


def on_pixel_ray(cam, x, y, z):
    return np.array([z * (x - cam.cx) / cam.fx, z * (y - cam.cy) / cam.fy, z])


def t64(a):
    return torch.as_tensor(np.asarray(a, np.float64))


def proj(scene, cam):
    return project(t64(scene.means), t64(scene.scales), t64(scene.quats), t64(scene.opacity),
                   t64(scene.colors), cam, ST)


# ----------------------------------------------------------------------------- constants

def test_constants_match_paper():
    g = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    assert ST.delta_alpha == pytest.approx(g["delta_alpha"]["value"], rel=1e-15)
    assert ST.cos_max_angle == pytest.approx(math.cos(math.radians(g["max_angle_deg"]["value"])), rel=1e-12)
    assert ST.mask_tile == g["tile_size"]["value"]
    assert ST.tile_discard_frac == g["tile_discard_frac"]["value"]
    hp = oracle.AdamHyper()
    assert hp.lr_means == g["lr_position"]["value"]
    assert hp.lr_quats == g["lr_rotation"]["value"]
    assert hp.lr_opacity == g["lr_opacity"]["value"]
    assert hp.lr_scales == g["lr_scale_replica"]["value"]
    assert hp.lr_colors == g["lr_sh0_replica"]["value"]


# ----------------------------------------------------------------------------- projection

@pytest.mark.parametrize("posed", [False, True])
def test_projection_on_axis_closed_form(posed):
    """A Gaussian axis-aligned with the camera on its optical axis: mu = (cx, cy) and
    Sigma_2D = diag(fx^2 sx^2 / z^2, fy^2 sy^2 / z^2) + lowpass I."""
    fx, fy, cx, cy, z = 300.0, 250.0, 40.5, 30.25, 2.5
    sx, sy, sz = 0.03, 0.012, 0.004
    if posed:
        cam = synth.look_at_camera([1.0, -2.0, 0.7], 0.8, 0.3, 81, 61, fx, cx, cy)
        cam.fy = fy
        Rc = cam.R.astype(np.float64)
        mean = cam.t.astype(np.float64) + Rc @ np.array([0, 0, z])
        q = quat_wxyz(Rc)
    else:
        cam = synth.identity_camera(81, 61, fx, cx, cy)
        cam.fy = fy
        mean, q = np.array([0, 0, z]), np.array([1.0, 0, 0, 0])
    sc = synth.Scene(means=mean.reshape(1, 3), scales=np.array([[sx, sy, sz]]), quats=q.reshape(1, 4),
                     opacity=np.array([0.9]), colors=np.ones((1, 3)), unstable=np.ones(1, np.uint8))
    pr = proj(sc, cam)
    # a float32 rotation matrix is orthonormal only to ~1e-7, hence the posed tolerance
    tol = 1e-5 if posed else 1e-12
    assert pr.mu[0].tolist() == pytest.approx([cx, cy], abs=1e3 * tol)
    a, b, c = pr.cov2d[0].tolist()
    assert a == pytest.approx(fx * fx * sx * sx / z / z + ST.lowpass, rel=tol)
    assert c == pytest.approx(fy * fy * sy * sy / z / z + ST.lowpass, rel=tol)
    assert abs(b) < 1e3 * tol
    assert pr.Z[0].item() == pytest.approx(z, rel=tol)


def test_projection_matches_numerical_jacobian():
    """Off-axis, posed camera, anisotropic rotated Gaussian: Sigma_2D - lowpass I must equal
    J Sigma J^T with J the finite-difference Jacobian of the pinhole map."""
    cam = synth.look_at_camera([0.3, 0.2, 1.1], 0.4, -0.2, 200, 150, 180.0)
    Rc, tc = cam.R.astype(np.float64), cam.t.astype(np.float64)
    mean = tc + Rc @ np.array([0.35, -0.22, 1.7])
    Rg = Rotation.from_euler("xyz", [0.3, -1.1, 0.7]).as_matrix()
    s = np.array([0.04, 0.015, 0.002])
    sc = synth.Scene(means=mean.reshape(1, 3), scales=s.reshape(1, 3), quats=quat_wxyz(Rg).reshape(1, 4),
                     opacity=np.array([0.9]), colors=np.ones((1, 3)), unstable=np.ones(1, np.uint8))

    def pin(p):
        X, Y, Z = Rc.T @ (p - tc)
        return np.array([cam.fx * X / Z + cam.cx, cam.fy * Y / Z + cam.cy])

    h = 1e-6
    J = np.stack([(pin(mean + h * e) - pin(mean - h * e)) / (2 * h) for e in np.eye(3)], 1)
    Sigma = Rg @ np.diag(s * s) @ Rg.T
    ref = J @ Sigma @ J.T
    pr = proj(sc, cam)
    a, b, c = pr.cov2d[0].tolist()
    got = np.array([[a - ST.lowpass, b], [b, c - ST.lowpass]])
    np.testing.assert_allclose(got, ref, rtol=1e-7, atol=1e-9)
    np.testing.assert_allclose(pr.mu[0].numpy(), pin(mean), rtol=0, atol=1e-9)
    # the conic is the inverse of Sigma_2D
    ca, cb, cc = pr.conic[0].tolist()
    np.testing.assert_allclose(np.array([[ca, cb], [cb, cc]]) @ np.array([[a, b], [b, c]]), np.eye(2), atol=1e-12)


# ----------------------------------------------------------------------------- compositing

@pytest.mark.parametrize("alpha,expect", [(0.7, 0.7), (0.99, 0.99), (1.0, 0.99), (0.3, 0.3)])
def test_peak_colour(alpha, expect):
    """A single Gaussian centred exactly on a pixel centre: C = c * min(alpha, f_max)."""
    cam = small_cam()
    R = Rotation.from_euler("zyx", [0.3, 0.2, 0.1]).as_matrix()
    c = np.array([0.2, 0.5, 0.9])
    sc = one_gaussian(on_pixel_ray(cam, 10, 20, 2.0), [0.05, 0.03, 0.01], quat_wxyz(R), alpha, c)
    r = oracle.render(sc, cam, ST, pixels=[[10, 20]])
    np.testing.assert_allclose(r.color[0].numpy(), c.astype(np.float32) * expect, rtol=1e-6)
    assert r.alpha[0].item() == pytest.approx(expect, rel=1e-6)


def test_two_layers_and_offcentre_closed_form():
    """Two Gaussians on one pixel ray: C = c1 f1 + c2 f2 (1 - f1), front one first; off the
    centre, f follows the closed-form footprint of an axis-aligned Gaussian on the axis."""
    cam = small_cam(33, 33, 40.0)  # principal point on pixel (16, 16)
    c1, c2 = np.array([1.0, 0.0, 0.0]), np.array([0.0, 1.0, 0.5])
    s1, s2 = [0.05, 0.03, 0.02], [0.04, 0.04, 0.02]
    q = [1.0, 0, 0, 0]
    front = one_gaussian([0, 0, 2.0], s1, q, 0.6, c1)
    back = one_gaussian([0, 0, 3.0], s2, q, 0.5, c2)
    for sc in (cat(front, back), cat(back, front)):
        pix = [[16, 16], [18, 15], [13, 19], [20, 16]]
        r = oracle.render(sc, cam, ST, pixels=pix)
        for k, (x, y) in enumerate(pix):
            def fval(s, z, al):
                a = (cam.fx * s[0] / z) ** 2 + ST.lowpass
                c = (cam.fy * s[1] / z) ** 2 + ST.lowpass
                f = min(ST.f_max, al * math.exp(-0.5 * ((x - 16) ** 2 / a + (y - 16) ** 2 / c)))
                return f if f >= ST.alpha_min else 0.0  # below alpha_min a fragment is skipped
            f1 = fval(np.float32(s1).astype(np.float64), 2.0, float(np.float32(0.6)))
            f2 = fval(np.float32(s2).astype(np.float64), 3.0, float(np.float32(0.5)))
            exp_c = c1 * f1 + c2 * f2 * (1 - f1)
            np.testing.assert_allclose(r.color[k].numpy(), exp_c, rtol=1e-9, atol=1e-12)
            assert r.alpha[k].item() == pytest.approx(1 - (1 - f1) * (1 - f2), rel=1e-9)
        # 0.6 < delta_alpha: no opaque hit anywhere
        assert (r.depth == -1).all() and (r.index == -1).all()


def test_telescoping_sum_equals_alpha():
    """With unit colours, Eq. 1 sums the weights f_i T_i, which telescope to 1 - T_final."""
    sc, cam = synth.scatter_scene(7, n=400)
    sc.colors[:] = 1.0
    r = oracle.render(sc, cam, ST)
    for ch in range(3):
        np.testing.assert_allclose(r.color[:, ch].numpy(), r.alpha.numpy(), rtol=0, atol=1e-12)
    assert (r.alpha > 0).any()


def test_empty_scene_and_all_behind():
    cam = small_cam()
    empty = synth.Scene(means=np.zeros((0, 3), np.float32), scales=np.zeros((0, 3), np.float32),
                        quats=np.zeros((0, 4), np.float32), opacity=np.zeros(0, np.float32),
                        colors=np.zeros((0, 3), np.float32), unstable=np.zeros(0, np.uint8))
    behind = one_gaussian([0, 0, -2.0], [0.5, 0.5, 0.5], [1, 0, 0, 0], 0.99, [1, 1, 1])
    for sc in (empty, behind):
        img = oracle.render_image(sc, cam, ST)
        assert (img["color"] == 0).all() and (img["depth"] == -1).all()
        assert (img["alpha"] == 0).all() and (img["index"] == -1).all()


def test_early_stop_count():
    """Identical fronto-parallel discs with f = 0.8 at a shared centre pixel: exactly
    floor(log(t_eps) / log(0.2)) = 5 fragments are composited before T drops below t_eps."""
    cam = small_cam(33, 33, 40.0)
    cols = np.eye(10, 3) + 0.05
    discs = [synth.disc_gaussian([0, 0, 2.0 + 0.1 * k], [0, 0, 1], 0.05, 0.001, 0.8, cols[k])
             for k in range(10)]
    sc = cat(*discs[::-1])
    r = oracle.render(sc, cam, ST, pixels=[[16, 16]])
    assert int(r.n_proc[0]) == 5 == math.floor(math.log(ST.t_eps) / math.log(0.2))
    f = np.float64(np.float32(0.8))
    exp_c = sum(cols[k].astype(np.float32) * f * (1 - f) ** k for k in range(5))
    np.testing.assert_allclose(r.color[0].numpy(), exp_c, rtol=1e-9)
    assert r.alpha[0].item() == pytest.approx(1 - (1 - f) ** 5, rel=1e-12)


# ----------------------------------------------------------------------------- depth

def test_fronto_parallel_disc_depth_and_hit_ellipse():
    """Opaque disc facing the camera at z0: depth z0 wherever f > delta_alpha, and that set
    is the ellipse d^T Sigma_2D^-1 d < 1 + 2 ln(0.99) of the closed-form footprint."""
    cam = small_cam(33, 33, 40.0)
    z0, r = 2.0, 0.1
    sc = synth.disc_gaussian([0, 0, z0], [0, 0, -1], r, 0.001, 0.99, [0.3, 0.3, 0.3], twist=0.7)
    img = oracle.render_image(sc, cam, ST)
    a = (cam.fx * float(np.float32(r)) / z0) ** 2 + ST.lowpass
    yy, xx = np.mgrid[0:33, 0:33]
    m2 = ((xx - 16.0) ** 2 + (yy - 16.0) ** 2) / a
    ellipse = m2 < 1 + 2 * math.log(float(np.float32(0.99)))
    assert ellipse.sum() > 5
    np.testing.assert_array_equal(img["depth"] != -1, ellipse)
    np.testing.assert_allclose(img["depth"][ellipse], z0, rtol=0, atol=1e-12)
    assert (img["index"][ellipse] == 0).all()


@pytest.mark.parametrize("tilt_deg", [25.0, 58.0])
def test_tilted_disc_plane_depth(tilt_deg):
    """Posed camera, tilted opaque disc: at each hit pixel the depth is the camera-frame
    ray/plane intersection t = (n.p)/(n.u) when |n.u|/|u| >= cos 60 deg, else the centre z."""
    cam = synth.look_at_camera([0.5, -0.3, 1.2], 1.0, 0.15, 64, 48, 60.0)
    Rc, tc = cam.R.astype(np.float64), cam.t.astype(np.float64)
    pc = np.array([0.05, -0.02, 1.8])
    t = math.radians(tilt_deg)
    nc = np.array([math.sin(t) * 0.8, math.sin(t) * 0.6, -math.cos(t)])
    sc = synth.disc_gaussian(tc + Rc @ pc, Rc @ nc, 0.25, 0.002, 0.99, [1, 1, 1], twist=0.3)
    img = oracle.render_image(sc, cam, ST)
    hit = img["depth"] != -1
    assert hit.sum() > 30
    pc32 = Rc.T @ (sc.means[0].astype(np.float64) - tc)
    n32 = Rc.T @ Rotation.from_quat(np.roll(sc.quats[0].astype(np.float64), -1)).as_matrix()[:, 2]
    branches = set()
    for y, x in zip(*np.nonzero(hit)):
        u = np.array([(x - cam.cx) / cam.fx, (y - cam.cy) / cam.fy, 1.0])
        cosang = abs(n32 @ u) / np.linalg.norm(u)
        assert abs(cosang - 0.5) > 1e-6
        exp_d = (n32 @ pc32) / (n32 @ u) if cosang >= 0.5 else pc32[2]
        branches.add(cosang >= 0.5)
        # float32 pose matrices are orthonormal to ~1e-7 only, so the world-frame and
        # camera-frame routes agree to that level, not to FP64 rounding
        assert img["depth"][y, x] == pytest.approx(exp_d, rel=1e-6)
    if tilt_deg < 30:
        assert branches == {True}


def test_sixty_degree_rule_both_branches():
    """A disc whose normal is about 60 degrees from the view rays: both Eq. 5 branches
    appear across its hit pixels, split exactly at |cos| = 0.5."""
    cam = small_cam(65, 65, 60.0)
    pc = np.array([0.0, 0.0, 2.0])
    t = math.radians(60.0)
    n = np.array([math.sin(t), 0.0, -math.cos(t)])
    sc = synth.disc_gaussian(pc, n, 0.4, 0.002, 0.99, [1, 1, 1])
    img = oracle.render_image(sc, cam, ST)
    hit = img["depth"] != -1
    plane, centre = 0, 0
    n64 = Rotation.from_quat(np.roll(sc.quats[0].astype(np.float64), -1)).as_matrix()[:, 2]
    p64 = sc.means[0].astype(np.float64)
    for y, x in zip(*np.nonzero(hit)):
        u = np.array([(x - cam.cx) / cam.fx, (y - cam.cy) / cam.fy, 1.0])
        cosang = abs(n64 @ u) / np.linalg.norm(u)
        if cosang >= 0.5:
            plane += 1
            assert img["depth"][y, x] == pytest.approx((n64 @ p64) / (n64 @ u), rel=1e-9)
        else:
            centre += 1
            assert img["depth"][y, x] == pytest.approx(p64[2], rel=1e-12)
    assert plane > 0 and centre > 0


def test_transparent_gaussians_never_set_depth():
    sc, cam = synth.scatter_scene(11, n=300)
    sc.opacity[:] = 0.05
    img = oracle.render_image(sc, cam, ST)
    assert (img["depth"] == -1).all() and (img["index"] == -1).all()
    assert img["color"].max() > 0


def test_two_stacked_opaque_discs_front_wins():
    cam = small_cam(33, 33, 40.0)
    front = synth.disc_gaussian([0, 0, 2.0], [0, 0, 1], 0.06, 0.001, 0.99, [1, 0, 0])
    back = synth.disc_gaussian([0, 0, 2.5], [0, 0, 1], 0.2, 0.001, 0.99, [0, 1, 0])
    img = oracle.render_image(cat(back, front), cam, ST)
    assert img["depth"][16, 16] == pytest.approx(2.0, abs=1e-12)
    assert img["index"][16, 16] == 1
    vals = set(np.round(img["depth"][img["depth"] != -1], 9).tolist())
    assert vals == {2.0, 2.5}


def test_permutation_invariance():
    sc, cam = synth.scatter_scene(5, n=500)
    perm = np.random.default_rng(0).permutation(sc.n)
    a = oracle.render(sc, cam, ST)
    b = oracle.render(sc.subset(perm), cam, ST)
    np.testing.assert_allclose(a.color.numpy(), b.color.numpy(), atol=1e-12)
    np.testing.assert_allclose(a.depth.numpy(), b.depth.numpy(), atol=1e-12)
    ia, ib = a.index.numpy(), b.index.numpy()
    np.testing.assert_array_equal(ia, np.where(ib >= 0, perm[np.maximum(ib, 0)], -1))


def test_borderline_rate_is_small():
    sc, cam = synth.scatter_scene(1000, n=2000)
    r = oracle.render(sc, cam, ST)
    assert r.borderline.float().mean().item() < 1e-3


# ----------------------------------------------------------------------------- gradients

def _mini_problem(seed=3, n=24):
    rng = np.random.default_rng(seed)
    sc, _ = synth.scatter_scene(seed, n=n)
    sc.means[:, :2] *= 0.4
    cam = synth.identity_camera(24, 20, 22.0, 11.5, 9.5)
    sc.unstable = (rng.random(n) < 0.7).astype(np.uint8)
    ys, xs = np.mgrid[0:20, 0:24]
    pix = np.stack([xs.ravel(), ys.ravel()], 1)
    tc = rng.uniform(0, 1, (pix.shape[0], 3))
    td = rng.uniform(1.0, 4.0, pix.shape[0])
    return sc, cam, pix, tc, td


def test_autograd_matches_finite_differences():
    """The oracle's analytic gradient agrees with FP64 central differences of its own
    forward on every parameter whose perturbation leaves all decisions unchanged."""
    sc, cam, pix, tc, td = _mini_problem()
    res = oracle.loss_and_grads(sc, cam, ST, pix, tc, td)
    uns = np.flatnonzero(sc.unstable)
    which, ref = [], []
    for name, width in (("means", 3), ("scales", 3), ("quats", 4), ("opacity", 1), ("colors", 3)):
        g = res["grads"][name].reshape(len(uns), -1)
        for k, gi in enumerate(uns):
            for comp in range(width):
                which.append((name, gi, comp))
                ref.append(g[k, comp])
    fd, stable = oracle.finite_difference_grads(sc, cam, ST, pix, tc, td, which)
    ref = np.array(ref)
    assert stable.mean() > 0.9
    scale = np.abs(ref).max()
    err = np.abs(fd - ref)[stable]
    assert (err <= 1e-6 * scale + 1e-5 * np.abs(ref[stable])).all(), err.max()


def test_gradient_special_cases():
    """Peak pixel of one Gaussian: dC/dc = alpha, dC/dalpha = c.  Fronto-parallel opaque
    disc: dD/dz = 1 and dD/dx = dD/dy = 0 (Eq. 4 is linear in the plane offset)."""
    cam = small_cam(33, 33, 40.0)
    c = np.array([0.2, 0.5, 0.9])
    sc = one_gaussian([0, 0, 2.0], [0.05, 0.03, 0.01], [1, 0, 0, 0], 0.5, c)
    res = oracle.loss_and_grads(sc, cam, ST, [[16, 16]], np.zeros((1, 3)), np.array([0.0]), w_c=1.0, w_d=0.0)
    # L = mean_c |C_c - 0| with C_c = alpha c_c > 0: dL/dc_c = alpha / 3, dL/dalpha = sum_c c_c / 3
    np.testing.assert_allclose(res["grads"]["colors"][0], np.full(3, float(np.float32(0.5)) / 3), rtol=1e-12)
    assert res["grads"]["opacity"][0] == pytest.approx(float(c.astype(np.float32).astype(np.float64).sum()) / 3, rel=1e-9)
    disc = synth.disc_gaussian([0, 0, 2.0], [0, 0, 1], 0.1, 0.001, 0.99, [1, 1, 1])
    pix = [[16, 16], [17, 16], [16, 17], [15, 15]]
    res = oracle.loss_and_grads(disc, cam, ST, pix, np.zeros((4, 3)), np.full(4, 1.0), w_c=0.0, w_d=1.0)
    # L = mean |D - 1| over 4 hit pixels, D = z: dL/dz = 1, dL/dx = dL/dy = 0
    np.testing.assert_allclose(res["grads"]["means"][0], [0.0, 0.0, 1.0], atol=1e-12)


# ----------------------------------------------------------------------------- mask, loss, adam

def test_unstable_mask_single_disc_closed_form():
    cam = small_cam(48, 40, 40.0)
    st = Settings(tile_discard_frac=0.0)
    s = float(np.float32(0.06)), float(np.float32(0.03))
    sc = one_gaussian([0, 0, 2.0], [s[0], s[1], 0.01], [1, 0, 0, 0], 0.99, [1, 1, 1])
    other = one_gaussian([0.3, 0.2, 2.0], [0.08, 0.08, 0.01], [1, 0, 0, 0], 0.99, [1, 1, 1])
    other.unstable[:] = 0  # stable Gaussians never enter the mask
    mask, border = oracle.unstable_mask(cat(sc, other), cam, st)
    a = (cam.fx * s[0] / 2.0) ** 2 + ST.lowpass
    c = (cam.fy * s[1] / 2.0) ** 2 + ST.lowpass
    yy, xx = np.mgrid[0:40, 0:48]
    m2 = (xx - cam.cx) ** 2 / a + (yy - cam.cy) ** 2 / c
    exp_m = m2 <= 2 * math.log(float(np.float32(0.99)) / ST.alpha_min)
    np.testing.assert_array_equal(mask[~border], exp_m[~border])
    assert exp_m.sum() > 30


def test_tile_rule_patterns():
    H, W = 24, 40  # 2 x 3 tiles, the last row and column ragged
    cover = np.zeros((H, W), bool)
    cover[0:16, 0:16].flat[:128] = True     # exactly 50% -> kept
    cover[0:16, 16:32].flat[:127] = True    # just below -> cleared
    cover[16:24, 32:40].flat[:32] = True    # ragged 8x8 tile, 50% -> kept
    cover[16:24, 0:16].flat[:63] = True     # ragged 8x16 tile, 63/128 -> cleared
    mask, tb = oracle.apply_tile_rule(cover, np.zeros_like(cover), 0.5, 16)
    assert mask[0:16, 0:16].sum() == 128
    assert mask[0:16, 16:32].sum() == 0
    assert mask[16:24, 32:40].sum() == 32
    assert mask[16:24, 0:16].sum() == 0
    off, _ = oracle.apply_tile_rule(cover, np.zeros_like(cover), 0.0, 16)
    np.testing.assert_array_equal(off, cover)


def test_l1_loss_hand_values():
    color = np.array([[0.5, 0.2, 0.0], [1.0, 1.0, 1.0]])
    tcol = np.array([[0.0, 0.2, 0.3], [0.5, 1.0, 1.0]])
    depth = np.array([2.0, -1.0])
    tdep = np.array([1.5, 3.0])
    L, Lc, Ld, P, Pd = oracle.l1_loss(color, depth, tcol, tdep)
    assert float(Lc) == pytest.approx((0.5 + 0 + 0.3 + 0.5) / 6)
    assert float(Ld) == pytest.approx(0.5) and Pd == 1 and P == 2
    assert float(L) == pytest.approx(float(Lc) + float(Ld))
    _, _, Ld2, _, Pd2 = oracle.l1_loss(color, np.array([2.0, 2.0]), tcol, np.array([1.5, 0.0]))
    assert Pd2 == 1 and float(Ld2) == pytest.approx(0.5)  # invalid input depth excluded


def test_adam_matches_torch_optim():
    rng = np.random.default_rng(4)
    n = 50
    params = dict(means=rng.normal(size=(n, 3)), scales=np.exp(rng.normal(-4, 0.5, (n, 3))),
                  quats=rng.normal(size=(n, 4)), opacity=rng.uniform(0, 1, n), colors=rng.uniform(0, 1, (n, 3)))
    hp = oracle.AdamHyper()
    m = {k: np.zeros_like(v) for k, v in params.items()}
    v = {k: np.zeros_like(val) for k, val in params.items()}
    tparams = {k: torch.tensor(np.log(val) if k == "scales" else val, requires_grad=True)
               for k, val in params.items()}
    opt = torch.optim.Adam([{"params": [tparams[k]], "lr": getattr(hp, "lr_" + k)} for k in oracle.adam.GROUPS],
                           betas=(hp.beta1, hp.beta2), eps=hp.eps, foreach=False)
    cur = params
    for step in range(1, 4):
        grads = {k: rng.normal(size=val.shape) for k, val in params.items()}
        cur, m, v = oracle.adam_step(cur, grads, m, v, step, hp)
        for k in oracle.adam.GROUPS:
            g = grads[k] * (np.exp(tparams[k].detach().numpy()) if k == "scales" else 1.0)
            tparams[k].grad = torch.tensor(g)
        opt.step()
        for k in oracle.adam.GROUPS:
            got = np.log(cur[k]) if k == "scales" else cur[k]
            np.testing.assert_allclose(got, tparams[k].detach().numpy(), rtol=1e-12, atol=1e-14)
