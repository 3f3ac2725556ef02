"""The masked step under the persistent schedule with programmatic dependent launch (some
kernels do work before they wait on the kernel in front: the forward sets up its first
item before the tile sort ends, the projection backward runs its light pass before the
compositing backward ends) against the same step with every launch serialised: renders,
mask and loss are identical, gradients and the Adam step equal to float32 atomic-order
rounding."""

import numpy as np
import pytest
import torch

import synth
from gpu_util import rtg

pytestmark = pytest.mark.gpu


def group_close(a, b, rel=2e-5):
    a, b = a.detach().cpu().numpy(), b.detach().cpu().numpy()
    scale = max(np.abs(a).max(initial=0), np.abs(b).max(initial=0), 1e-30)
    assert np.abs(a - b).max(initial=0) <= rel * scale, f"max diff {np.abs(a - b).max():.3e} of {scale:.3e}"


def run(scene, cam, tc, td, overlap, steps):
    m = rtg()
    H, W = cam.height, cam.width
    ctx = m.Context(max_gaussians=scene.n, max_width=W, max_height=H)
    ctx.set_tuning(m.Tuning(8, 8, 32, 1, 2, 8, 512, overlap))
    g = m.Gaussians.from_scene(scene)
    mask = torch.zeros(1, H, W, dtype=torch.uint8, device="cuda")
    m.unstable_mask(ctx, [cam], g, m.RenderSettings(), mask)
    step = m.MaskedStep(ctx, g, [cam], mask, tc, td)
    first = step.step().clone()
    grads = [t.clone() for t in step.grads]
    img = [step.state.color.clone(), step.state.depth.clone(), step.state.alpha.clone()]
    for _ in range(steps - 1):
        step.step()
    torch.cuda.synchronize()
    assert m.get_status(ctx) == 0
    out = dict(mask=mask.clone(), loss=first, grads=grads, img=img, params=[t.clone() for t in step.u],
               counter=step.step_counter.tolist())
    ctx.close()
    return out


@pytest.mark.parametrize("seed,n,nu", [(8100, 30000, 6000), (8200, 120000, 30000)])
def test_programmatic_launch_on_and_off_agree(seed, n, nu):
    m = rtg()
    scene, layout = synth.room_scene(seed, n)
    cam = next(synth.room_camera_candidates(seed + 1, layout, 320, 240, 240.0))
    scene.unstable = synth.flag_blobs(scene, [cam], nu, 3, seed=seed + 2)
    H, W = cam.height, cam.width
    ref = m.Gaussians.from_scene(synth.jitter_scene(scene, seed + 3))
    ctx0 = m.Context(max_gaussians=scene.n, max_width=W, max_height=H)
    tc = torch.zeros(1, 3, H, W, device="cuda")
    td = torch.full((1, H, W), -1.0, device="cuda")
    m.render_forward(ctx0, cam, ref, None, m.RenderSettings(), tc, td, torch.zeros(1, H, W, device="cuda"))
    td.clamp_(min=0)
    ctx0.close()
    on, off = run(scene, cam, tc, td, 1, 3), run(scene, cam, tc, td, 0, 3)
    assert int(on["mask"].sum()) > 0 and torch.equal(on["mask"], off["mask"])
    for a, b in zip(on["img"], off["img"]):
        assert torch.equal(a, b)
    np.testing.assert_allclose(on["loss"].cpu().numpy(), off["loss"].cpu().numpy(), rtol=1e-6)
    for a, b in zip(on["grads"], off["grads"]):
        group_close(a, b)
    assert on["counter"] == off["counter"] == [3, 0]
    # Adam divides each gradient by its own running RMS: where a gradient's atomic sum is
    # near zero the summation order decides the sign of a full step, so almost every element
    # agrees closely and the whole arrays to 1e-4 of their norm
    for a, b in zip(on["params"], off["params"]):
        a, b = a.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)
        assert (~np.isclose(b, a, rtol=1e-4, atol=1e-6)).mean() <= 1e-3
        assert np.linalg.norm(b - a) <= 1e-4 * np.linalg.norm(a)
