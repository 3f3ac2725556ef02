"""Pins of the oracle's fusion and state management (paper Section 3.2, Eq. 9 and "State
management"): hand-made cases with their expected counts, weights and transitions."""

import numpy as np

from oracle import state as sm


def test_confidence_counts_updated_colours_only():
    eta = np.array([5, 0, 7, 1], np.int32)
    ids = np.array([0, 2, 3])
    g = np.array([[0, 0, 0], [0.1, 0, 0], [0, 0, -1e-30]], np.float32)
    np.testing.assert_array_equal(sm.confidence_update(eta, ids, g), [5, 0, 8, 2])


def test_fusion_weights_closed_form():
    n = 4
    full = {k: np.zeros((n, w), np.float32) for k, w in (("means", 3), ("scales", 3), ("quats", 4), ("colors", 3))}
    full["opacity"] = np.zeros(n, np.float32)
    full["means"][:] = 1.0
    comp = {k: np.full((3,) + v.shape[1:], 5.0, np.float32) for k, v in full.items()}
    ids = np.array([0, 1, 3])
    eta0 = np.array([3, 2, 9, 0], np.int32)
    eta1 = np.array([4, 2, 9, 0], np.int32)
    out = sm.fuse_window(full, comp, ids, eta0, eta1)
    # Gaussian 0: w = (4 - 3) / 4 = 0.25 -> 0.75 * 1 + 0.25 * 5 = 2
    np.testing.assert_array_equal(out["means"][0], [2, 2, 2])
    np.testing.assert_array_equal(out["opacity"][0], np.float32(1.25))  # 0.75 * 0 + 0.25 * 5
    # Gaussian 1: not updated in the window (w = 0): unchanged
    np.testing.assert_array_equal(out["means"][1], [1, 1, 1])
    # Gaussian 2: not optimised: unchanged; Gaussian 3: eta' = 0: unchanged
    np.testing.assert_array_equal(out["means"][2], [1, 1, 1])
    np.testing.assert_array_equal(out["means"][3], [1, 1, 1])
    # first window of a new Gaussian (eta 0 -> 6): w = 1, the optimised value
    one = {k: v[:1] for k, v in comp.items()}
    out = sm.fuse_window(full, one, np.array([2]), np.array([0, 0, 0, 0]), np.array([0, 0, 6, 0]))
    np.testing.assert_array_equal(out["quats"][2], [5, 5, 5, 5])


def test_error_counts_once_per_frame_and_stable_only():
    # 2 frames of 2x3, C = 3, Gaussians 0, 1 stable and 2 unstable
    rc = np.zeros((2, 3, 2, 3), np.float32)
    ic = np.zeros((2, 3, 2, 3), np.float32)
    Dh = np.full((2, 2, 3), 2.0, np.float32)
    D = np.full((2, 2, 3), 2.0, np.float32)
    idx = np.full((2, 2, 3), -1, np.int64)
    # frame 0: colour error (mean 0.2) at a pixel of Gaussian 0; two erring pixels of
    # Gaussian 1 (depth error 0.3); an erring pixel of unstable Gaussian 2; an erring pixel
    # without a Gaussian; a depth error where the input has no depth (not an error)
    ic[0, :, 0, 0] = 0.2
    idx[0, 0, 0] = 0
    D[0, 0, 1] = 2.3
    D[0, 0, 2] = 2.3
    idx[0, 0, 1] = idx[0, 0, 2] = 1
    ic[0, :, 1, 0] = 0.5
    idx[0, 1, 0] = 2
    ic[0, :, 1, 1] = 0.5
    D[0, 1, 2] = 0.0
    Dh[0, 1, 2] = 5.0
    idx[0, 1, 2] = 0
    # frame 1: Gaussian 1 errs again; Gaussian 0's pixel is fine (error 0.05 mean)
    D[1, 1, 1] = 1.0
    idx[1, 1, 1] = 1
    ic[1, :, 0, 0] = 0.05
    idx[1, 0, 0] = 0
    got = sm.error_flags(rc, Dh, idx, ic, D, np.array([0, 0, 1], np.uint8))
    np.testing.assert_array_equal(got, [1, 2, 0])


def test_state_transitions():
    p = sm.StateParams(delta_eta=100, delta_e=10, delta_t=200)
    #            stable->unstable, stable stays, unstable->stable, unstable stays, unstable removed, removed? no: converts
    unstable = np.array([0, 0, 1, 1, 1, 1], np.uint8)
    eta = np.array([150, 150, 101, 50, 50, 120], np.int32)
    err = np.array([11, 10, 3, 0, 0, 0], np.int32)
    t0 = np.array([0, 0, 0, 900, 700, 500], np.int64)
    u, e, r, rm = sm.update_states(unstable, eta, err, t0, k=1000, p=p)
    np.testing.assert_array_equal(u, [1, 0, 0, 1, 1, 0])
    np.testing.assert_array_equal(e, [0, 150, 101, 50, 50, 120])
    np.testing.assert_array_equal(r, [0, 10, 0, 0, 0, 0])
    # the old unstable Gaussian (k - t = 300 > 200) is removed; the one that just turned
    # stable (also old) is kept
    np.testing.assert_array_equal(rm, [False, False, False, False, True, False])


def test_compaction_keeps_order():
    arr = {"a": np.arange(6) * 10, "b": np.arange(12).reshape(6, 2)}
    out = sm.compact(arr, np.array([0, 1, 0, 0, 1, 0], bool))
    np.testing.assert_array_equal(out["a"], [0, 20, 30, 50])
    np.testing.assert_array_equal(out["b"], [[0, 1], [4, 5], [6, 7], [10, 11]])
