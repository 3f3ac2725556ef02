"""Frame-sharded keyframe batches on CPU ranks (gloo): the host logic of
paper_2404_19706_b300.sharding -- the frame split, the all-reduce of the pixel counts and
of the compact gradient array, and the replicated Adam step -- with the FP64 oracle
computing each rank's share of the batch gradient (there is no GPU here).

Each rank's share uses the batch's pixel totals in the means of Eq. 7; the test checks that
two gloo ranks end with the gradient and the Adam update of the whole batch, computed in
one process frame by frame, and with bit-equal replicas on both ranks."""

import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2404_19706_b300.sharding import allreduce_sum, flat_gradients, frame_shard  # noqa: E402

GROUPS = ("means", "scales", "quats", "opacity", "colors")


def test_frame_shard_covers_every_frame_once_in_order():
    for F in range(1, 21):
        for world in range(1, min(F, 8) + 1):
            got = []
            sizes = []
            for r in range(world):
                sl = frame_shard(F, r, world)
                got.extend(range(F)[sl])
                sizes.append(sl.stop - sl.start)
            assert got == list(range(F))
            assert max(sizes) - min(sizes) <= 1


def test_frame_shard_rejects_more_ranks_than_frames():
    with pytest.raises(ValueError):
        frame_shard(2, 0, 3)
    with pytest.raises(ValueError):
        frame_shard(4, 4, 4)


def test_flat_gradient_views_partition_the_buffer():
    nu, C = 5, 3
    flat, views = flat_gradients(nu, C, "cpu")
    assert flat.numel() == nu * (11 + C)
    assert [tuple(v.shape) for v in views] == [(nu, 3), (nu, 3), (nu, 4), (nu,), (nu, C)]
    for k, v in enumerate(views):
        v.fill_(k + 1)
    expect = torch.cat([torch.full((nu * n,), float(k + 1)) for k, n in enumerate((3, 3, 4, 1, C))])
    assert torch.equal(flat, expect)


def _problem():
    """A small scene seen by four cameras, with per-frame pixel samples and targets."""
    import oracle
    import synth
    scene, cam0 = synth.scatter_scene(77, n=90)
    scene.unstable = (np.arange(scene.n) % 2 == 0).astype(np.uint8)
    cams = []
    for k, dx in enumerate((-0.15, -0.05, 0.05, 0.15)):
        c = cam0.copy()
        c.t = np.array([dx, 0.03 * k, 0.0], dtype=np.float32)
        cams.append(c)
    rng = np.random.default_rng(5)
    st = oracle.Settings()
    frames = []
    for c in cams:
        pix = np.stack([rng.integers(20, 140, 24), rng.integers(15, 105, 24)], 1)
        tc = rng.uniform(0, 1, (24, 3))
        td = rng.uniform(1.5, 4.0, 24)
        td[::5] = 0.0  # pixels without input depth
        frames.append((pix, tc, td))
    return scene, cams, frames, st


def _share(scene, cams, frames, st, which, totals):
    """Gradient of the batch loss restricted to frames `which` (global means): each frame's
    local-mean gradient weighted by its share of the batch's pixels."""
    import oracle
    g = {k: 0.0 for k in GROUPS}
    for f in which:
        pix, tc, td = frames[f]
        n = oracle.loss_and_grads(scene, cams[f], st, pix, tc, td, 1.0, 1.0)
        w_c = n["n_pixels"] / totals[0]
        w_d = n["n_depth"] / totals[1] if totals[1] > 0 else 0.0
        r = oracle.loss_and_grads(scene, cams[f], st, pix, tc, td, w_c, w_d)
        for k in GROUPS:
            g[k] = g[k] + r["grads"][k]
    return g


def _counts(scene, cams, frames, st, which):
    import oracle
    c = np.zeros(4)
    for f in which:
        pix, tc, td = frames[f]
        r = oracle.loss_and_grads(scene, cams[f], st, pix, tc, td, 1.0, 1.0)
        c += [r["n_pixels"], r["n_depth"], r["loss_color"] * r["n_pixels"] * 3, r["loss_depth"] * r["n_depth"]]
    return c


def _flatten(g, nu):
    return torch.cat([torch.as_tensor(np.asarray(g[k], dtype=np.float64)).reshape(-1) for k in GROUPS])


def _adam(scene, flat, nu):
    """One Adam step of the oracle on the unstable Gaussians from the flat batch gradient."""
    from oracle import adam as oadam
    sel = np.flatnonzero(scene.unstable)
    params = {"means": scene.means[sel].astype(np.float64), "scales": scene.scales[sel].astype(np.float64),
              "quats": scene.quats[sel].astype(np.float64), "opacity": scene.opacity[sel].astype(np.float64),
              "colors": scene.colors[sel].astype(np.float64)}
    grads, o = {}, 0
    for k, w in zip(GROUPS, (3, 3, 4, 1, 3)):
        v = flat[o:o + nu * w].numpy()
        grads[k] = v.reshape(nu) if w == 1 else v.reshape(nu, w)
        o += nu * w
    zeros = {k: np.zeros_like(v) for k, v in params.items()}
    newp, _, _ = oadam.adam_step(params, grads, zeros, dict(zeros), 1, oadam.AdamHyper())
    return np.concatenate([newp[k].reshape(-1) for k in GROUPS])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.set_num_threads(2)
    scene, cams, frames, st = _problem()
    nu = int(scene.unstable.sum())
    mine = range(len(cams))[frame_shard(len(cams), rank, world)]
    counts = torch.as_tensor(_counts(scene, cams, frames, st, mine))
    allreduce_sum(counts)  # the batch's pixel counts and L1 sums
    flat = _flatten(_share(scene, cams, frames, st, mine, counts.tolist()), nu)
    allreduce_sum(flat)  # the batch gradient
    out[rank] = (counts.numpy(), flat.numpy(), _adam(scene, flat, nu), list(mine))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_batch_gradient_and_adam_step():
    world, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        got = dict(out)
    assert got[0][3] == [0, 1] and got[1][3] == [2, 3]
    # the replicas agree exactly: same summed counts, gradient and parameters on both ranks
    for a, b in zip(got[0][:3], got[1][:3]):
        np.testing.assert_array_equal(a, b)
    # against the whole batch in one process, frame by frame
    scene, cams, frames, st = _problem()
    nu = int(scene.unstable.sum())
    totals = _counts(scene, cams, frames, st, range(4))
    np.testing.assert_allclose(got[0][0], totals, rtol=1e-12)
    flat = _flatten(_share(scene, cams, frames, st, range(4), totals.tolist()), nu)
    assert np.abs(flat.numpy()).max() > 0
    np.testing.assert_allclose(got[0][1], flat.numpy(), rtol=1e-9, atol=1e-12 * np.abs(flat.numpy()).max())
    np.testing.assert_allclose(got[0][2], _adam(scene, flat, nu), rtol=1e-9, atol=1e-12)
    # the batch loss from the summed sums equals the mean over every pixel of the batch
    Lc = totals[2] / (totals[0] * 3)
    assert Lc > 0
