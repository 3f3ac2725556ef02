"""Fusion and state management (paper Section 3.2, "Gaussian optimization" (Eq. 9) and
"State management"): TEST INFRASTRUCTURE ONLY, like the rest of this package.

  - Confidence count: eta_i grows by 1 whenever the colour of Gaussian i is updated.
  - Fusion after the window o: G_o = (1 - w) G_{o-1} + w G'_o with
    w = (eta'_o - eta_{o-1}) / eta'_o, where G'_o is the optimised Gaussian and eta'_o its
    count after the window; the count becomes eta'_o.
  - Error count: the optimised map is rendered on frame k; a stable Gaussian whose pixels
    (the pixels whose depth hit it is, by the index map) show a colour or depth error
    above delta_c / delta_d has e_i incremented by 1.
  - States: stable with e_i > delta_e -> unstable; unstable with eta_i > delta_eta ->
    stable; unstable with k - t_i > delta_t -> removed.

Readings (the paragraphs leave them open):
  - an update of the colour (the count's trigger): in an optimisation iteration, the Gaussian's colour gradient
    is non-zero in some channel (it was rendered on the iteration's pixels);
  - fusion uses float32 arithmetic: w = float(eta' - eta) / float(eta'), then
    (1 - w) * a + w * b rounded per operation, applied to every stored parameter
    (position, linear scale, raw quaternion, opacity, colour); eta' = 0 keeps G_{o-1};
  - the error of a pixel is the mean absolute colour difference over channels (tested as
    the float32 sum > C * delta_c, as in the adding pass) or |D_hat - D| > delta_d where
    the input depth is valid (D > 0); pixels without a depth hit (index -1) count for no
    Gaussian; a Gaussian counts at most once per frame however many of its pixels err;
  - converting stable -> unstable resets eta and e to 0 (otherwise the next update would
    convert it straight back); converting unstable -> stable resets e to 0;
  - a Gaussian converted in this update is not removed in the same update; removal keeps
    the order of the remaining Gaussians.
"""

from __future__ import annotations

import dataclasses

import numpy as np

GROUPS = ("means", "scales", "quats", "opacity", "colors")


@dataclasses.dataclass(frozen=True)
class StateParams:
    delta_eta: int = 100
    delta_e: int = 10
    delta_t: int = 200
    delta_c: float = 0.1
    delta_d: float = 0.1


def confidence_update(eta: np.ndarray, ids: np.ndarray, g_colors: np.ndarray) -> np.ndarray:
    """eta [n] int32 after one iteration: +1 for each optimised Gaussian ids[k] whose colour
    gradient row g_colors[k] is non-zero."""
    out = np.asarray(eta, np.int32).copy()
    g = np.asarray(g_colors, np.float32).reshape(len(ids), -1)
    upd = (g != 0).any(axis=1)
    out[np.asarray(ids)[upd]] += 1
    return out


def fuse_window(full: dict, compact: dict, ids: np.ndarray, eta_start: np.ndarray, eta_now: np.ndarray) -> dict:
    """Eq. 9 on the optimised Gaussians ids[k]: full[name][i] <- (1 - w) full + w compact[k].
    full / compact map GROUPS to float32 arrays ([n, .] / [nu, .])."""
    ids = np.asarray(ids)
    e0 = np.asarray(eta_start, np.int64)[ids]
    e1 = np.asarray(eta_now, np.int64)[ids]
    w = np.where(e1 > 0, (e1 - e0).astype(np.float32) / np.maximum(e1, 1).astype(np.float32), np.float32(0))
    w = w.astype(np.float32)
    one_w = (np.float32(1) - w).astype(np.float32)
    out = {}
    for name in GROUPS:
        a = np.asarray(full[name], np.float32).copy()
        shape = a.shape
        a2 = a.reshape(shape[0], -1)
        b = np.asarray(compact[name], np.float32).reshape(len(ids), -1)
        prev = a2[ids]
        blended = ((one_w[:, None] * prev).astype(np.float32) + (w[:, None] * b).astype(np.float32)).astype(np.float32)
        a2[ids] = np.where((e1 > 0)[:, None], blended, prev)
        out[name] = a2.reshape(shape)
    return out


def error_flags(render_color, render_depth, index_map, color, depth, unstable, p: StateParams = StateParams()):
    """[n] int32: the number of frames in which each stable Gaussian has an erring pixel."""
    rc = np.asarray(render_color, np.float32)
    ic = np.asarray(color, np.float32)
    Dh = np.asarray(render_depth, np.float32)
    D = np.asarray(depth, np.float32)
    idx = np.asarray(index_map, np.int64)
    flags = np.asarray(unstable)
    n = flags.shape[0]
    F, C = rc.shape[0], rc.shape[1]
    err = np.zeros(D.shape, np.float32)
    for c in range(C):
        err = (err + np.abs(rc[:, c] - ic[:, c])).astype(np.float32)
    bad = (err > np.float32(C) * np.float32(p.delta_c)) | ((D > np.float32(0)) & (np.abs(Dh - D) > np.float32(p.delta_d)))
    counts = np.zeros(n, np.int32)
    for f in range(F):
        hit = idx[f][bad[f] & (idx[f] >= 0) & (idx[f] < n)]
        g = np.unique(hit)
        g = g[flags[g] == 0]
        counts[g] += 1
    return counts


def update_states(unstable, eta, err, t0, k: int, p: StateParams = StateParams()):
    """One state update at frame k: returns (unstable, eta, err, remove) as new arrays."""
    u = np.asarray(unstable, np.uint8).copy()
    e = np.asarray(eta, np.int32).copy()
    r = np.asarray(err, np.int32).copy()
    t = np.asarray(t0, np.int64)
    was_stable = u == 0
    to_unstable = was_stable & (r > p.delta_e)
    to_stable = ~was_stable & (e > p.delta_eta)
    remove = ~was_stable & ~to_stable & ((k - t) > p.delta_t)
    u[to_unstable] = 1
    e[to_unstable] = 0
    r[to_unstable] = 0
    u[to_stable] = 0
    r[to_stable] = 0
    return u, e, r, remove


def compact(arrays: dict, remove: np.ndarray) -> dict:
    """Every per-Gaussian array without the removed rows, order kept."""
    keep = ~np.asarray(remove, bool)
    return {k: np.asarray(v)[keep] for k, v in arrays.items()}
