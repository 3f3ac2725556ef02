"""Helpers shared by the GPU parity tests (they call the CUDA path through the C ABI)."""

import numpy as np
import torch

import synth

# Parity bar: GPU vs FP64 oracle within 1e-4 relative on colour (with a 1e-4 absolute
# floor, colours being O(1)) and 1e-4 m on depth; index maps exact.  Pixels whose
# discrete decisions sit within FP32 rounding of flipping (the oracle's borderline set)
# are excluded and counted.
COLOR_RTOL = 1e-4
COLOR_ATOL = 1e-4
DEPTH_ATOL = 1e-4


def rtg():
    import paper_2404_19706_b300 as m
    return m


def ctx_for(n, cams, channels=3, max_pairs=None):
    cams = cams if isinstance(cams, (list, tuple)) else [cams]
    return rtg().Context(max_gaussians=max(n, 1), max_frames=len(cams), max_width=cams[0].width,
                         max_height=cams[0].height, max_channels=channels, max_pairs=max_pairs)


def gpu_forward(scene, cams, mask=None, settings=None, ctx=None, fill=True):
    """Renders through rtg_render_forward; returns numpy arrays (and the context)."""
    m = rtg()
    cams = cams if isinstance(cams, (list, tuple)) else [cams]
    F, H, W = len(cams), cams[0].height, cams[0].width
    C = 3 if np.asarray(scene.colors).ndim == 3 else scene.colors.shape[1]  # SH coefficients render RGB
    g = m.Gaussians.from_scene(scene)
    own = ctx is None
    if own:
        ctx = ctx_for(scene.n, cams, C)
    color = torch.zeros(F, C, H, W, device="cuda")
    depth = torch.full((F, H, W), -1.0, device="cuda")
    alpha = torch.zeros(F, H, W, device="cuda")
    index = torch.full((F, H, W), -1, dtype=torch.int32, device="cuda")
    mk = None
    if mask is not None:
        mk = torch.as_tensor(np.ascontiguousarray(mask, dtype=np.uint8)).reshape(F, H, W).cuda()
    m.render_forward(ctx, cams, g, mk, settings or m.RenderSettings(), color, depth, alpha, index)
    torch.cuda.synchronize()
    stats = m.get_stats(ctx)
    out = dict(color=color.cpu().numpy(), depth=depth.cpu().numpy(), alpha=alpha.cpu().numpy(),
               index=index.cpu().numpy(), stats=stats, ctx=ctx, g=g)
    return out


def assert_forward_matches(ref, got_color, got_depth, got_alpha, got_index, max_border_frac=1e-3):
    """ref: oracle.render_image dict for one frame; got_*: [C,H,W] / [H,W] numpy."""
    ok = ~ref["borderline"]
    n_border = int((~ok).sum())
    assert n_border <= max(2, max_border_frac * ok.size), f"{n_border} borderline pixels of {ok.size}"
    rc, gc = ref["color"][:, ok], got_color[:, ok].astype(np.float64)
    bad = np.abs(gc - rc) > COLOR_ATOL + COLOR_RTOL * np.abs(rc)
    assert not bad.any(), f"colour: {bad.sum()} values off, max err {np.abs(gc - rc).max():.3e}"
    ra, ga = ref["alpha"][ok], got_alpha[ok].astype(np.float64)
    assert np.abs(ga - ra).max(initial=0) <= COLOR_ATOL + COLOR_RTOL, f"alpha max err {np.abs(ga - ra).max():.3e}"
    rd, gd = ref["depth"][ok], got_depth[ok].astype(np.float64)
    assert np.abs(gd - rd).max(initial=0) <= DEPTH_ATOL, f"depth max err {np.abs(gd - rd).max():.3e}"
    np.testing.assert_array_equal(got_index[ok], ref["index"][ok])
    return n_border


def room_crop_camera(width, height, f, seed, layout):
    cam = next(synth.room_camera_candidates(seed, layout, width, height, f))
    return cam
