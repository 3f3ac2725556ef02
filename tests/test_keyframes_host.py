"""Host logic of the global keyframe optimisation (Section 3.2, "Keyframes and global
optimization"): the keyframe rule, the keyframe draw of a global step and the global Adam
settings, against the oracle and by their stated properties."""

import math

import numpy as np

import oracle
from oracle import global_opt as go
from paper_2404_19706_b300 import AdamSettings, KeyframeSet, global_adam
from paper_2404_19706_b300.keyframes import rotation_angle_deg


def _rot(axis, deg):
    a = np.asarray(axis, np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    t = math.radians(deg)
    return np.eye(3) + math.sin(t) * K + (1 - math.cos(t)) * K @ K


def test_rule_agrees_with_oracle_on_random_poses():
    rng = np.random.default_rng(11)
    agree = 0
    for _ in range(400):
        R0 = _rot(rng.normal(size=3), rng.uniform(0, 180))
        R1 = R0 @ _rot(rng.normal(size=3), rng.uniform(0, 60))
        t0 = rng.normal(size=3)
        t1 = t0 + rng.normal(size=3) * rng.uniform(0, 0.3)
        ang = go.rotation_angle_deg(R0, R1)
        assert abs(rotation_angle_deg(R0, R1) - ang) < 1e-6
        if abs(ang - 30.0) < 1e-6 or abs(np.linalg.norm(t1 - t0) - 0.3) < 1e-9:
            continue
        ks = KeyframeSet()
        ks.offer(0, R0, t0)
        assert ks.is_new(R1, t1) == go.is_new_keyframe(R0, t0, R1, t1)
        agree += 1
    assert agree > 390


def test_offer_builds_the_list_against_the_last_keyframe():
    ks = KeyframeSet()
    I = np.eye(3)
    assert ks.offer(0, I, np.zeros(3))                  # first frame
    assert not ks.offer(1, _rot([0, 0, 1], 20), np.zeros(3))
    assert not ks.offer(2, _rot([0, 0, 1], 29), np.array([0.2, 0, 0]))
    assert ks.offer(3, _rot([0, 0, 1], 31), np.zeros(3))  # rotation
    assert not ks.offer(4, _rot([0, 0, 1], 50), np.zeros(3))  # 19 degrees from frame 3
    assert ks.offer(5, _rot([0, 0, 1], 31), np.array([0, 0.31, 0]))  # translation
    assert ks.frames == [0, 3, 5]


def test_pick_latest_plus_three_distinct_random():
    ks = KeyframeSet()
    for i in range(12):
        ks.offer(i, _rot([0, 1, 0], 40 * i), np.zeros(3))
    assert len(ks) == 12
    counts = np.zeros(11)
    rng = np.random.default_rng(3)
    for _ in range(3000):
        p = ks.pick(rng)
        assert p[0] == 11 and len(p) == 4 and len(set(p)) == 4 and all(0 <= i < 11 for i in p[1:])
        counts[p[1:]] += 1
    assert counts.min() > 0.8 * counts.mean() and counts.max() < 1.2 * counts.mean()  # uniform draw
    assert ks.pick(np.random.default_rng(5)) == ks.pick(np.random.default_rng(5))
    small = KeyframeSet()
    small.offer(0, np.eye(3), np.zeros(3))
    assert small.pick(rng) == [0]
    small.offer(1, np.eye(3), np.ones(3))
    assert small.pick(rng) == [1, 0]
    assert KeyframeSet().pick(rng) == []


def test_final_schedule_ten_passes():
    ks = KeyframeSet()
    for i in range(5):
        ks.offer(i, np.eye(3), np.full(3, float(i)))
    sch = ks.final_schedule()
    assert len(sch) == 50 and np.bincount(sch).tolist() == [10] * 5


def test_global_adam_matches_oracle_settings():
    ours, ref = global_adam(AdamSettings()), go.global_hyper(oracle.AdamHyper())
    for f in ("lr_means", "lr_scales", "lr_quats", "lr_opacity", "lr_colors", "beta1", "beta2", "eps"):
        assert math.isclose(getattr(ours, f), getattr(ref, f), rel_tol=1e-15, abs_tol=0.0), f
    assert ours.lr_means == 0.0
