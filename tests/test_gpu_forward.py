"""GPU forward (rtg_render_forward) vs the FP64 oracle, element by element."""

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import assert_forward_matches, ctx_for, gpu_forward, rtg

pytestmark = pytest.mark.gpu
ST = oracle.Settings()


def test_scatter_scene_160x120_matches_oracle():
    """2,000 random ellipsoids, half opaque / half transparent, 160x120 (10 x 7.5 tiles)."""
    scene, cam = synth.scatter_scene(1000, n=2000)
    ref = oracle.render_image(scene, cam, ST)
    got = gpu_forward(scene, cam)
    n_b = assert_forward_matches(ref, got["color"][0], got["depth"][0], got["alpha"][0], got["index"][0])
    # fragments: the GPU counts every composited fragment; the oracle agrees away from borderline pixels
    ok = ~ref["borderline"]
    assert abs(got["stats"]["fragments"] - ref["n_proc"].sum()) <= ref["n_proc"][~ok].sum() + 64 * n_b
    assert got["stats"]["status"] == 0


def test_room_crop_ragged_matches_oracle():
    """Flattened surfel Gaussians on a box room seen by a ragged 100x75 camera
    (partial tiles on the right and bottom edges)."""
    scene, layout = synth.room_scene(2002, 50000)
    cam = next(synth.room_camera_candidates(2003, layout, 100, 75, 94.0))
    ref = oracle.render_image(scene, cam, ST)
    got = gpu_forward(scene, cam)
    assert (ref["depth"] > 0).mean() > 0.3  # opaque surfaces cover a good part of the view
    assert_forward_matches(ref, got["color"][0], got["depth"][0], got["alpha"][0], got["index"][0])


def test_masked_equals_full_restricted_and_mask_respected():
    scene, cam = synth.scatter_scene(1001, n=1500)
    full = gpu_forward(scene, cam)
    mask = synth.random_masks(5, 1, cam.height, cam.width, 0.2, 0.4)[0]
    part = gpu_forward(scene, cam, mask=mask)
    m = mask.astype(bool)
    np.testing.assert_array_equal(part["color"][0][:, m], full["color"][0][:, m])
    np.testing.assert_array_equal(part["depth"][0][m], full["depth"][0][m])
    np.testing.assert_array_equal(part["index"][0][m], full["index"][0][m])
    # outside the mask the outputs keep their fill values
    assert (part["color"][0][:, ~m] == 0).all() and (part["depth"][0][~m] == -1).all()
    assert part["stats"]["masked_pixels"] == int(m.sum())
    empty = gpu_forward(scene, cam, mask=np.zeros_like(mask))
    assert (empty["color"] == 0).all() and empty["stats"]["pairs"] == 0


def test_permutation_invariance_bitwise():
    scene, cam = synth.scatter_scene(1002, n=1500)
    perm = np.random.default_rng(1).permutation(scene.n)
    a = gpu_forward(scene, cam)
    b = gpu_forward(scene.subset(perm), cam)
    np.testing.assert_array_equal(a["color"], b["color"])
    np.testing.assert_array_equal(a["depth"], b["depth"])
    ib = b["index"]
    np.testing.assert_array_equal(a["index"], np.where(ib >= 0, perm[np.maximum(ib, 0)], -1))


def test_batched_frames_equal_single_frames_bitwise():
    scene, layout = synth.room_scene(2004, 30000)
    cams = [c for _, c in zip(range(3), synth.room_camera_candidates(2005, layout, 96, 64, 80.0))]
    masks = synth.random_masks(6, 3, 64, 96, 0.3, 0.9)
    batch = gpu_forward(scene, cams, mask=masks)
    for f in range(3):
        single = gpu_forward(scene, cams[f], mask=masks[f])
        np.testing.assert_array_equal(batch["color"][f], single["color"][0])
        np.testing.assert_array_equal(batch["depth"][f], single["depth"][0])
        np.testing.assert_array_equal(batch["index"][f], single["index"][0])


def test_run_twice_is_deterministic():
    scene, cam = synth.scatter_scene(1003, n=1000)
    ctx = ctx_for(scene.n, cam)
    a = gpu_forward(scene, cam, ctx=ctx)
    b = gpu_forward(scene, cam, ctx=ctx)
    for k in ("color", "depth", "alpha", "index"):
        np.testing.assert_array_equal(a[k], b[k])


def test_nan_and_degenerate_gaussians_are_culled():
    scene, cam = synth.scatter_scene(1004, n=400)
    bad = scene.copy()
    bad.means[3, 0] = np.nan
    bad.quats[7] = 0.0           # zero quaternion cannot be normalised
    bad.colors[11, 1] = np.inf
    keep = np.setdiff1d(np.arange(scene.n), [3, 7, 11])
    a = gpu_forward(bad, cam)
    b = gpu_forward(scene.subset(keep), cam)
    np.testing.assert_array_equal(a["color"], b["color"])
    np.testing.assert_array_equal(a["depth"], b["depth"])
    ib = b["index"]
    np.testing.assert_array_equal(a["index"], np.where(ib >= 0, keep[np.maximum(ib, 0)], -1))


def test_empty_scene():
    scene, cam = synth.scatter_scene(1005, n=10)
    empty = scene.subset(np.arange(0))
    got = gpu_forward(empty, cam)
    assert (got["color"] == 0).all() and (got["depth"] == -1).all() and (got["index"] == -1).all()
    assert (got["alpha"] == 0).all()


def test_eight_channel_features_match_oracle():
    scene, cam = synth.scatter_scene(1006, n=800)
    rng = np.random.default_rng(3)
    scene.colors = rng.normal(0, 0.5, (scene.n, 8)).astype(np.float32)
    ref = oracle.render_image(scene, cam, ST)
    got = gpu_forward(scene, cam)
    assert_forward_matches(ref, got["color"][0], got["depth"][0], got["alpha"][0], got["index"][0])


def test_full_size_room_sampled_pixels():
    """300k surfels at 640x480 (the full single-frame workload), checked on sampled pixels
    that the oracle evaluates one by one."""
    scene, layout = synth.room_scene(2000, 300_000)
    cam = next(synth.room_camera_candidates(2001, layout))
    got = gpu_forward(scene, cam)
    rng = np.random.default_rng(7)
    pix = np.stack([rng.integers(0, cam.width, 160), rng.integers(0, cam.height, 160)], 1)
    ref = oracle.render(scene, cam, ST, pixels=pix)
    ok = ~ref.borderline.numpy()
    xs, ys = pix[:, 0], pix[:, 1]
    gc = got["color"][0][:, ys, xs].T.astype(np.float64)
    rc = ref.color.numpy()
    assert (np.abs(gc - rc)[ok] <= 1e-4 + 1e-4 * np.abs(rc[ok])).all()
    assert (np.abs(got["depth"][0][ys, xs] - ref.depth.numpy())[ok] <= 1e-4).all()
    np.testing.assert_array_equal(got["index"][0][ys, xs][ok], ref.index.numpy()[ok])
    assert got["stats"]["status"] == 0
