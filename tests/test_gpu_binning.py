"""Tile binning and per-tile depth order are bit-exact: the bucket offsets and sorted index
lists must equal a CPU rebuild (numpy lexsort on (tile, depth-key bits, index)) from the
GPU's own float32 projection outputs (tile rectangles, depth-key bits) and the mask."""

import numpy as np
import pytest

import synth
from gpu_util import gpu_forward, rtg

pytestmark = pytest.mark.gpu


def cpu_rebuild(rect, zbits, n, F, W, H, masks, tw=16, th=16):
    tx, ty = (W + tw - 1) // tw, (H + th - 1) // th
    T = tx * ty
    active = np.ones((F, T), dtype=bool)
    if masks is not None:
        m = np.zeros((F, ty * th, tx * tw), dtype=bool)
        m[:, :H, :W] = masks.reshape(F, H, W).astype(bool)
        active = m.reshape(F, ty, th, tx, tw).any(axis=(2, 4)).reshape(F, T)
    tiles, keys, ids = [], [], []
    for f in range(F):
        for i in range(n):
            x0, y0, x1, y1 = rect[f * n + i]
            if x0 < 0:
                continue
            for yy in range(y0, y1 + 1):
                for xx in range(x0, x1 + 1):
                    t = yy * tx + xx
                    if active[f, t]:
                        tiles.append(f * T + t)
                        keys.append(zbits[f * n + i])
                        ids.append(i)
    tiles, keys, ids = np.array(tiles, np.int64), np.array(keys, np.uint64), np.array(ids, np.int64)
    order = np.lexsort((ids, keys, tiles))
    counts = np.bincount(tiles, minlength=F * T)
    offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.uint32)
    return offsets, ids[order].astype(np.uint32)


def check(scene, cams, masks=None, tuning=None):
    cams = cams if isinstance(cams, list) else [cams]
    F, H, W = len(cams), cams[0].height, cams[0].width
    ctx = None
    if tuning is not None:
        from gpu_util import ctx_for
        ctx = ctx_for(scene.n, cams)
        ctx.set_tuning(tuning)
    got = gpu_forward(scene, cams, mask=masks, ctx=ctx)
    d = rtg().debug_binning(got["ctx"], F, W, H, scene.n)
    tw, th = got["stats"]["tile_w"], got["stats"]["tile_h"]
    offs, ids = cpu_rebuild(d["rect"], d["zbits"], scene.n, F, W, H, masks, tw, th)
    np.testing.assert_array_equal(d["tile_offsets"], offs)
    np.testing.assert_array_equal(d["sorted_ids"], ids)
    assert d["pairs"] == len(ids) > 0
    return d, got


def test_binning_bit_exact_scatter_scene():
    scene, cam = synth.scatter_scene(1000, n=2000)
    check(scene, cam)


def test_binning_bit_exact_masked_multiframe_ragged():
    scene, layout = synth.room_scene(2010, 8000)
    cams = [c for _, c in zip(range(2), synth.room_camera_candidates(2011, layout, 84, 60, 70.0))]
    masks = synth.random_masks(12, 2, 60, 84, 0.2, 0.6)
    check(scene, cams, masks)


def test_binning_long_bucket_uses_global_sort_path():
    """3,000 Gaussians stacked over one 16x16 tile: the bucket exceeds the shared-memory
    sort capacity (2,048 keys), so the chunked global-memory passes are exercised; the
    depth keys include exact ties, broken by index."""
    rng = np.random.default_rng(9)
    n = 3000
    cam = synth.identity_camera(16, 16, 20.0, 7.5, 7.5)
    z = np.round(rng.uniform(1.0, 3.0, n), 2)  # many equal depths
    means = np.stack([rng.uniform(-0.2, 0.2, n) * z, rng.uniform(-0.2, 0.2, n) * z, z], 1)
    scene = synth.Scene(means=means.astype(np.float32),
                        scales=np.exp(rng.uniform(np.log(0.02), np.log(0.2), (n, 3))).astype(np.float32),
                        quats=rng.normal(size=(n, 4)).astype(np.float32),
                        opacity=rng.choice([0.99, 0.05], n).astype(np.float32),
                        colors=rng.uniform(0, 1, (n, 3)).astype(np.float32), unstable=np.ones(n, np.uint8))
    d, got = check(scene, cam)
    assert got["stats"]["max_tile_pairs"] > 2048
    zb = d["zbits"][d["sorted_ids"]]
    assert (np.diff(zb.astype(np.int64)) == 0).any()  # ties present


@pytest.mark.parametrize("tile", [(8, 8), (8, 16), (16, 8), (32, 8)])
def test_binning_bit_exact_every_render_tile(tile):
    """Every render tile shape bins bit-exactly, and its tile rectangles are the 8 x 8
    rectangles coarsened (the pixel rectangle behind them does not depend on the tile)."""
    m = rtg()
    scene, layout = synth.room_scene(2012, 8000)
    cams = [c for _, c in zip(range(2), synth.room_camera_candidates(2013, layout, 92, 66, 70.0))]
    masks = synth.random_masks(14, 2, 66, 92, 0.2, 0.6)
    tw, th = tile
    d, got = check(scene, cams, masks, m.Tuning(tw, th, schedule=1, sort_rank_max=512))
    assert (got["stats"]["tile_w"], got["stats"]["tile_h"]) == tile
    d8, _ = check(scene, cams, masks, m.Tuning(8, 8))
    # which Gaussians reach a masked tile depends on the tile, the rectangle itself does not
    both = (d8["rect"][:, 0] >= 0) & (d["rect"][:, 0] >= 0)
    assert both.sum() > 100
    ratio = np.array([tw // 8, th // 8, tw // 8, th // 8])
    np.testing.assert_array_equal(d8["rect"][both] // ratio, d["rect"][both])
    np.testing.assert_array_equal(d["zbits"][both], d8["zbits"][both])


def test_binning_bit_exact_multiblock_scan():
    """3 frames at 640x480 in 8x8 tiles (14,400 tiles): the tile scan runs as its multi-block
    form; offsets and lists stay bit-exact, and the render equals the single-frame calls."""
    m = rtg()
    scene, layout = synth.room_scene(2014, 8000)
    cams = [c for _, c in zip(range(3), synth.room_camera_candidates(2015, layout, 640, 480, 600.0))]
    masks = synth.random_masks(16, 3, 480, 640, 0.2, 0.6)
    d, got = check(scene, cams, masks, m.Tuning(8, 8, schedule=1))
    assert len(d["tile_offsets"]) == 3 * 80 * 60 + 1
    from gpu_util import ctx_for
    for f in range(3):
        c1 = ctx_for(scene.n, cams[f])
        c1.set_tuning(m.Tuning(8, 8, schedule=1))
        single = gpu_forward(scene, cams[f], mask=masks[f], ctx=c1)
        np.testing.assert_array_equal(got["color"][f], single["color"][0])
        np.testing.assert_array_equal(got["depth"][f], single["depth"][0])
