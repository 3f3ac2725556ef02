"""Gaussian adding on the GPU (Section 3.2, "Gaussians adding", Eq. 6) against the oracle:
on the same float32 maps the new Gaussians (pixels, kinds, colours, opacities; positions to
float32 rounding) and their count are identical, for random maps with every case present,
ragged sizes, several frames, a capacity below the count, and the full pass on a room
scene with a region missing from the map."""

import numpy as np
import pytest
import torch

import synth
from gpu_util import rtg
from oracle import adding as ad

pytestmark = pytest.mark.gpu


def random_maps(seed, F, C, H, W, n):
    rng = np.random.default_rng(seed)
    rc = rng.uniform(0, 1, (F, C, H, W)).astype(np.float32)
    ic = (rc + rng.choice([0.0, 0.05, 0.2], (F, C, H, W)) * rng.choice([-1, 1], (F, C, H, W))).astype(np.float32)
    alpha = rng.choice([1.0, 0.9, 0.45, 0.0], (F, H, W)).astype(np.float32)
    D = rng.uniform(0.5, 4.0, (F, H, W)).astype(np.float32)
    D[rng.random((F, H, W)) < 0.1] = 0.0  # no measurement
    Dh = (D + rng.choice([0.0, 0.02, 0.3], (F, H, W))).astype(np.float32)
    Dh[rng.random((F, H, W)) < 0.1] = -1.0
    idx = rng.integers(-1, n, (F, H, W)).astype(np.int32)
    unstable = (rng.random(n) < 0.3).astype(np.uint8)
    return rc, alpha, Dh, idx, ic, D, unstable


def cams_for(F, H, W, seed):
    rng = np.random.default_rng(seed)
    out = []
    for f in range(F):
        a = rng.uniform(0, 2 * np.pi)
        R = np.array([[np.cos(a), 0, np.sin(a)], [0, 1, 0], [-np.sin(a), 0, np.cos(a)]], np.float32)
        out.append(synth.Camera(fx=float(W), fy=float(W), cx=(W - 1) / 2, cy=(H - 1) / 2, width=W, height=H, R=R,
                                t=rng.normal(size=3).astype(np.float32)))
    return out


def gpu_add(cams, maps, settings, seed, capacity):
    m = rtg()
    rc, alpha, Dh, idx, ic, D, unstable = maps
    F, C, H, W = rc.shape
    ctx = m.Context(max_gaussians=max(len(unstable), 1), max_frames=F, max_width=W, max_height=H,
                    max_channels=3, max_pairs=1 << 10)
    t = lambda a, dt=torch.float32: torch.as_tensor(np.ascontiguousarray(a)).to("cuda", dt)  # noqa: E731
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    pix = torch.full((capacity,), -7, dtype=torch.int32, device="cuda")
    kind = torch.zeros(capacity, dtype=torch.uint8, device="cuda")
    pos = torch.zeros(capacity, 3, device="cuda")
    col = torch.zeros(capacity, C, device="cuda")
    op = torch.zeros(capacity, device="cuda")
    m.add_candidates(ctx, cams, t(rc), t(alpha), t(Dh), t(idx, torch.int32), t(ic), t(D), t(unstable, torch.uint8),
                     settings, seed, count, pix, kind, pos, col, op)
    torch.cuda.synchronize()
    n = int(count.item())
    k = min(n, capacity)
    return n, dict(pixel=pix[:k].cpu().numpy(), kind=kind[:k].cpu().numpy(), position=pos[:k].cpu().numpy(),
                   color=col[:k].cpu().numpy(), opacity=op[:k].cpu().numpy()), pix[k:].cpu().numpy()


def compare(got, ref, k):
    np.testing.assert_array_equal(got["pixel"], ref["pixel"][:k])
    np.testing.assert_array_equal(got["kind"], ref["kind"][:k])
    np.testing.assert_array_equal(got["color"], ref["color"][:k])
    np.testing.assert_array_equal(got["opacity"], ref["opacity"][:k])
    np.testing.assert_allclose(got["position"], ref["position"][:k], rtol=1e-6, atol=1e-5)


@pytest.mark.parametrize("F,C,H,W", [(1, 3, 7, 5), (3, 3, 37, 53), (2, 8, 120, 160)])
@pytest.mark.parametrize("rate", [1.0, 0.05, 0.0])
def test_add_candidates_match_oracle(F, C, H, W, rate):
    m = rtg()
    maps = random_maps(F * 100 + W, F, C, H, W, 50)
    cams = cams_for(F, H, W, 3)
    st = m.AddSettings(sample_rate=rate)
    seed = 0x1234_5678_9ABC
    ref = ad.add_candidates(cams, *maps, ad.AddParams(sample_rate=rate, seed=seed))
    n, got, _ = gpu_add(cams, maps, st, seed, capacity=F * H * W)
    assert n == len(ref["pixel"])
    compare(got, ref, n)
    if rate == 1.0 and H * W >= 1000:  # every case of Eq. 6 occurs
        assert set(np.unique(got["kind"])) == {1, 2} and ref["m_c"].sum() > (got["kind"] == 2).sum()


def test_capacity_below_count_and_seeds():
    m = rtg()
    F, C, H, W = 2, 3, 64, 96
    maps = random_maps(9, F, C, H, W, 40)
    cams = cams_for(F, H, W, 4)
    ref = ad.add_candidates(cams, *maps, ad.AddParams(sample_rate=0.5, seed=11))
    n, got, rest = gpu_add(cams, maps, m.AddSettings(sample_rate=0.5), 11, capacity=100)
    assert n == len(ref["pixel"]) > 100
    compare(got, ref, 100)
    assert (rest == -7).all()  # nothing written past the capacity
    n2, got2, _ = gpu_add(cams, maps, m.AddSettings(sample_rate=0.5), 12, capacity=F * H * W)
    assert not np.array_equal(got2["pixel"][:50], got["pixel"][:50])


def test_adding_pass_on_a_room_with_a_missing_region():
    """The map lacks the Gaussians of one blob that the input frame (a render of the whole
    scene) shows: the pass adds opaque Gaussians there.  Its outputs equal the oracle's on
    the pass's own render maps."""
    m = rtg()
    scene, layout = synth.room_scene(7000, 60_000)
    cam = next(synth.room_camera_candidates(7001, layout, 160, 120, 150.0))
    blob = synth.flag_blobs(scene, [cam], 6000, 1, seed=7002, n_in_view=1).astype(bool)
    full = m.Gaussians.from_scene(scene)
    ctx = m.Context(max_gaussians=scene.n, max_frames=1, max_width=160, max_height=120)
    ic = torch.zeros(1, 3, 120, 160, device="cuda")
    D = torch.full((1, 120, 160), -1.0, device="cuda")
    m.render_forward(ctx, [cam], full, None, m.RenderSettings(), ic, D, torch.zeros(1, 120, 160, device="cuda"))
    D = torch.where(D > 0, D, torch.zeros_like(D))
    part = scene.subset(np.flatnonzero(~blob))
    part.unstable = (np.random.default_rng(1).random(part.n) < 0.2).astype(np.uint8)
    g = m.Gaussians.from_scene(part)
    ap = m.AddingPass(ctx, 160, 120, capacity=20_000, add=m.AddSettings(sample_rate=1.0))
    count = ap.run([cam], g, ic, D, seed=5)
    torch.cuda.synchronize()
    n = int(count.item())
    ref = ad.add_candidates([cam], ap.color.cpu().numpy(), ap.alpha.cpu().numpy(), ap.depth.cpu().numpy(),
                            ap.index.cpu().numpy(), ic.cpu().numpy(), D.cpu().numpy(), part.unstable,
                            ad.AddParams(sample_rate=1.0, seed=5))
    assert n == len(ref["pixel"]) and (ref["kind"] == 1).sum() > 50
    got = dict(pixel=ap.pixel[:n].cpu().numpy(), kind=ap.kind[:n].cpu().numpy(), position=ap.position[:n].cpu().numpy(),
               color=ap.new_color[:n].cpu().numpy(), opacity=ap.opacity[:n].cpu().numpy())
    compare(got, ref, n)
    # the opaque additions sit on the missing blob's surface: near its Gaussians
    from scipy.spatial import cKDTree
    opaque = got["position"][got["kind"] == 1]
    d = cKDTree(scene.means[blob].astype(np.float64)).query(opaque.astype(np.float64))[0]
    assert np.median(d) < 0.05 and (d < 0.15).mean() > 0.9, (np.median(d), (d < 0.15).mean())
