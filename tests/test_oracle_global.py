"""Pins of the oracle's global keyframe optimisation pieces (paper, "Keyframes and global
optimization"): the top-40% colour-error pixel selection, the Adam settings and the
keyframe rule, each against hand-made cases or closed forms."""

import math

import numpy as np

from oracle import AdamHyper, global_opt as go


def test_color_error_hand_values():
    color = np.array([[[[0.5, 1.0]], [[0.25, 0.0]], [[1.0, 0.5]]]], dtype=np.float32)   # [1, 3, 1, 2]
    target = np.array([[[[0.0, 1.0]], [[0.75, 0.25]], [[1.0, 0.0]]]], dtype=np.float32)
    err = go.color_error(color, target)
    np.testing.assert_array_equal(err, np.array([[[0.5 + 0.5 + 0.0, 0.0 + 0.25 + 0.5]]], dtype=np.float32))


def test_keep_count_exact():
    assert go.keep_count(0.4, 640 * 480) == 122880
    assert go.keep_count(0.4, 10) == 4
    assert go.keep_count(0.4, 11) == 4
    assert go.keep_count(0.0, 100) == 0 and go.keep_count(1.0, 100) == 100


def _mask_of(err_row, frac):
    """err_row: one frame's errors (H=1); colour = err, target = 0, one channel."""
    e = np.asarray(err_row, dtype=np.float32)[None, None, None, :]
    return go.top_error_mask(e, np.zeros_like(e), frac)[0, 0]


def test_top_error_mask_hand_made_with_ties():
    # errors at indices 0..9; 40% of 10 pixels = 4 kept
    err = [0.1, 0.7, 0.3, 0.7, 0.2, 0.3, 0.9, 0.3, 0.0, 0.3]
    # largest: 0.9 (6), 0.7 (1), 0.7 (3); then one of the four 0.3s: the lowest index, 2
    np.testing.assert_array_equal(_mask_of(err, 0.4), [0, 1, 1, 1, 0, 0, 1, 0, 0, 0])
    # 60%: six kept: the three above, then 0.3 at 2, 5, 7 (not 9)
    np.testing.assert_array_equal(_mask_of(err, 0.6), [0, 1, 1, 1, 0, 1, 1, 1, 0, 0])
    # all equal: the first k pixels
    np.testing.assert_array_equal(_mask_of([0.5] * 5, 0.4), [1, 1, 0, 0, 0])
    # nothing and everything
    assert _mask_of(err, 0.0).sum() == 0 and _mask_of(err, 1.0).sum() == 10


def test_top_error_mask_per_frame_and_count():
    rng = np.random.default_rng(3)
    color = rng.uniform(0, 1, (3, 3, 7, 9)).astype(np.float32)
    target = rng.uniform(0, 1, (3, 3, 7, 9)).astype(np.float32)
    m = go.top_error_mask(color, target, 0.4)
    err = go.color_error(color, target)
    for f in range(3):
        assert m[f].sum() == math.floor(0.4 * 63)
        # every kept error is at least every dropped one
        assert err[f][m[f] == 1].min() >= err[f][m[f] == 0].max()


def test_global_hyper_freezes_positions_and_scales_rates():
    base = AdamHyper()
    h = go.global_hyper(base)
    assert h.lr_means == 0.0
    assert math.isclose(h.lr_scales, 0.1 * base.lr_scales) and math.isclose(h.lr_quats, 0.1 * base.lr_quats)
    assert math.isclose(h.lr_colors, 0.1 * base.lr_colors) and h.lr_opacity == 0.1 * base.lr_opacity
    assert (h.beta1, h.beta2, h.eps) == (base.beta1, base.beta2, base.eps)


def _rz(deg):
    a = math.radians(deg)
    return np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1.0]])


def test_keyframe_rule_thresholds():
    I, t0 = np.eye(3), np.zeros(3)
    assert math.isclose(go.rotation_angle_deg(I, _rz(37.0)), 37.0, rel_tol=1e-12)
    assert math.isclose(go.rotation_angle_deg(_rz(10.0), _rz(-25.0)), 35.0, rel_tol=1e-12)
    assert not go.is_new_keyframe(I, t0, _rz(29.0), t0)
    assert go.is_new_keyframe(I, t0, _rz(31.0), t0)
    assert not go.is_new_keyframe(I, t0, I, np.array([0.2, 0.2, 0.0]))   # 0.283 m
    assert go.is_new_keyframe(I, t0, I, np.array([0.0, 0.0, 0.31]))
