"""Fusion and state management on the GPU (Section 3.2, Eq. 9 and "State management")
against the oracle, bit for bit: confidence counts, the Eq. 9 blend (float32, one rounding
per operation), error counts through the index map, state transitions, order-preserving
pruning; and a MaskedStep window that counts confidence and ends with the fusion."""

import numpy as np
import pytest
import torch

import synth
from gpu_util import ctx_for, gpu_forward, rtg
from oracle import state as so

pytestmark = pytest.mark.gpu
GROUPS = ("means", "scales", "quats", "opacity", "colors")
WIDTH = {"means": 3, "scales": 3, "quats": 4, "opacity": 1, "colors": 3}


def t(a, dt=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to("cuda", dt)


def test_confidence_update_matches_oracle():
    m = rtg()
    rng = np.random.default_rng(1)
    n, nu = 5000, 1800
    ids = np.sort(rng.choice(n, nu, replace=False)).astype(np.int32)
    g = rng.normal(size=(nu, 3)).astype(np.float32)
    g[rng.random(nu) < 0.4] = 0.0
    g[rng.random(nu) < 0.1, 1] = -0.0
    eta = rng.integers(0, 50, n).astype(np.int32)
    et = t(eta, torch.int32)
    m.confidence_update(t(ids, torch.int32), t(g), et)
    np.testing.assert_array_equal(et.cpu().numpy(), so.confidence_update(eta, ids, g))


def test_fuse_window_matches_oracle_bitwise():
    m = rtg()
    rng = np.random.default_rng(2)
    n, nu = 7000, 2500
    ids = np.sort(rng.choice(n, nu, replace=False)).astype(np.int32)
    full = {k: rng.normal(size=(n, WIDTH[k]) if WIDTH[k] > 1 else n).astype(np.float32) for k in GROUPS}
    comp = {k: rng.normal(size=(nu, WIDTH[k]) if WIDTH[k] > 1 else nu).astype(np.float32) for k in GROUPS}
    e0 = rng.integers(0, 30, n).astype(np.int32)
    e1 = (e0 + rng.integers(0, 8, n)).astype(np.int32)
    e1[rng.random(n) < 0.05] = 0
    g = m.Gaussians(*[t(full[k]) for k in GROUPS], t(np.zeros(n, np.uint8), torch.uint8))
    m.fuse_window(t(ids, torch.int32), t(e0, torch.int32), t(e1, torch.int32), [t(comp[k]) for k in GROUPS], g)
    want = so.fuse_window(full, comp, ids, e0, e1)
    for k in GROUPS:
        np.testing.assert_array_equal(getattr(g, k).cpu().numpy(), want[k], err_msg=k)


def test_error_count_matches_oracle():
    m = rtg()
    rng = np.random.default_rng(3)
    F, C, H, W, n = 3, 3, 37, 53, 400
    rc = rng.uniform(0, 1, (F, C, H, W)).astype(np.float32)
    ic = (rc + rng.choice([0.0, 0.05, 0.2], (F, C, H, W))).astype(np.float32)
    D = rng.uniform(0.5, 4, (F, H, W)).astype(np.float32)
    D[rng.random((F, H, W)) < 0.1] = 0
    Dh = (D + rng.choice([0.0, 0.05, 0.3], (F, H, W))).astype(np.float32)
    idx = rng.integers(-1, n, (F, H, W)).astype(np.int32)
    unstable = (rng.random(n) < 0.3).astype(np.uint8)
    err0 = rng.integers(0, 5, n).astype(np.int32)
    ctx = m.Context(max_gaussians=n, max_frames=F, max_width=W, max_height=H, max_pairs=1 << 10)
    st = m.StateSettings()
    err = t(err0, torch.int32)
    m.error_count(ctx, t(rc), t(Dh), t(idx, torch.int32), t(ic), t(D), t(unstable, torch.uint8), st, err)
    want = err0 + so.error_flags(rc, Dh, idx, ic, D, unstable)
    np.testing.assert_array_equal(err.cpu().numpy(), want)
    # the scratch bits are left clear: a second call counts again from scratch
    m.error_count(ctx, t(rc), t(Dh), t(idx, torch.int32), t(ic), t(D), t(unstable, torch.uint8), st, err)
    np.testing.assert_array_equal(err.cpu().numpy(), want + so.error_flags(rc, Dh, idx, ic, D, unstable))


def test_update_states_and_compaction_match_oracle():
    m = rtg()
    rng = np.random.default_rng(4)
    n, C = 10_000, 3
    p = so.StateParams(delta_eta=100, delta_e=10, delta_t=200)
    unstable = (rng.random(n) < 0.5).astype(np.uint8)
    eta = rng.integers(0, 200, n).astype(np.int32)
    err = rng.integers(0, 20, n).astype(np.int32)
    t0 = rng.integers(0, 1000, n).astype(np.int32)
    u_t, e_t, r_t = t(unstable, torch.uint8), t(eta, torch.int32), t(err, torch.int32)
    rm = torch.zeros(n, dtype=torch.uint8, device="cuda")
    st = m.StateSettings(100, 10, 200)
    m.update_states(1000, t(t0, torch.int32), st, u_t, e_t, r_t, rm)
    wu, we, wr, wrm = so.update_states(unstable, eta, err, t0, 1000, p)
    np.testing.assert_array_equal(u_t.cpu().numpy(), wu)
    np.testing.assert_array_equal(e_t.cpu().numpy(), we)
    np.testing.assert_array_equal(r_t.cpu().numpy(), wr)
    np.testing.assert_array_equal(rm.cpu().numpy().astype(bool), wrm)
    assert 0 < wrm.sum() < n
    # pruning the flagged Gaussians
    arr = {k: rng.normal(size=(n, WIDTH[k]) if WIDTH[k] > 1 else n).astype(np.float32) for k in GROUPS}
    src = m.MapArrays(*[t(arr[k]) for k in GROUPS], u_t, e_t, r_t, t(t0, torch.int32))
    dst = m.MapArrays.empty_like(src)
    ctx = m.Context(max_gaussians=n, max_frames=1, max_width=8, max_height=8, max_pairs=1 << 10)
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    m.compact_gaussians(ctx, rm, src, dst, cnt)
    k = int(cnt.item())
    want = so.compact(dict(arr, unstable=wu, eta=we, err=wr, t0=t0), wrm)
    assert k == n - wrm.sum()
    for name, v in want.items():
        np.testing.assert_array_equal(getattr(dst, name)[:k].cpu().numpy(), v, err_msg=name)


def test_masked_step_with_state_counts_and_fuses():
    """A window of MaskedStep iterations with a MapState: eta rises by one per iteration for
    the unstable Gaussians whose colour gradient was non-zero (checked on the first one),
    and finish() blends with the weights of Eq. 9 (checked against the oracle on the same
    arrays)."""
    m = rtg()
    scene, layout = synth.room_scene(2050, 20000)
    cam = next(synth.room_camera_candidates(2051, layout, 128, 96, 120.0))
    scene.unstable = synth.flag_blobs(scene, [cam], 4000, 3, seed=12)
    tref = gpu_forward(synth.jitter_scene(scene, 13), cam)
    tc = torch.tensor(tref["color"]).cuda()
    td = torch.tensor(np.where(tref["depth"] > 0, tref["depth"], 0)).cuda()
    ctx = ctx_for(scene.n, cam)
    g = m.Gaussians.from_scene(scene)
    state = m.MapState(ctx, g)
    state.eta.copy_(torch.randint(0, 5, (scene.n,), dtype=torch.int32, device="cuda"))
    mask = torch.zeros(1, 96, 128, dtype=torch.uint8, device="cuda")
    step = m.MaskedStep(ctx, g, [cam], mask, tc, td, recompute_mask=True, map_state=state)
    eta_start = state.eta.cpu().numpy().copy()
    step.step()
    torch.cuda.synchronize()
    ids = step.ids.cpu().numpy()
    g_col = step.grads[4].cpu().numpy()
    np.testing.assert_array_equal(state.eta.cpu().numpy(), so.confidence_update(eta_start, ids, g_col))
    for _ in range(4):
        step.step()
    torch.cuda.synchronize()
    full_before = {k: getattr(g, k).cpu().numpy().copy() for k in GROUPS}
    comp = {k: u.cpu().numpy() for k, u in zip(GROUPS, step.u)}
    eta_now = state.eta.cpu().numpy()
    assert (eta_now[ids] - eta_start[ids]).max() == 5
    step.finish()
    torch.cuda.synchronize()
    want = so.fuse_window(full_before, comp, ids, eta_start, eta_now)
    for k in GROUPS:
        np.testing.assert_array_equal(getattr(g, k).cpu().numpy(), want[k], err_msg=k)
