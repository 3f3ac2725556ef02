"""Pins of the oracle's Gaussian-adding pass (paper Section 3.2, "Gaussians adding", Eq. 6):
the counter-based draw against SplitMix64's published outputs, the masks and the
opaque/transparent decision on a hand-made frame, the draw rate, and the back-projection
in closed form."""

import math

import numpy as np

from oracle import adding as ad
from synth import Camera


def test_splitmix64_published_outputs():
    # first outputs of the reference SplitMix64 generator (Steele, Lea and Flood, 2014) for
    # seeds 0 and 1234567, as published with its reference implementation
    got0 = [int(v) for v in ad.splitmix64(0, np.arange(3))]
    assert got0 == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    got1 = [int(v) for v in ad.splitmix64(1234567, np.arange(3))]
    assert got1 == [6457827717110365317, 3203168211198807973, 9817491932198370423]
    # the counter form is the stream: output k does not depend on which others are drawn
    assert int(ad.splitmix64(1234567, np.array([2]))[0]) == got1[2]


def _frame():
    """One 2x4 frame, C = 3, each pixel one case of Eq. 6 (params: 0.5, 0.1 m, 0.1)."""
    H, W = 2, 4
    rc = np.zeros((1, 3, H, W), np.float32)
    ic = np.zeros((1, 3, H, W), np.float32)
    alpha = np.ones((1, H, W), np.float32)
    Dh = np.full((1, H, W), 2.0, np.float32)
    D = np.full((1, H, W), 2.0, np.float32)
    idx = np.zeros((1, H, W), np.int64)
    # (0,0): nothing wrong
    # (0,1): T_hat = 0.6 > 0.5                   -> M_s
    alpha[0, 0, 1] = 0.4
    # (0,2): depth error 0.2 > 0.1                -> M_s
    D[0, 0, 2] = 2.2
    # (0,3): colour error only (mean 0.2 > 0.1)   -> M_c, hit Gaussian 1 (stable)
    ic[0, :, 0, 3] = 0.2
    idx[0, 0, 3] = 1
    # (1,0): colour and depth error               -> M_s only
    ic[0, :, 1, 0] = 0.5
    D[0, 1, 0] = 3.0
    # (1,1): invalid input depth, everything off  -> neither
    D[0, 1, 1] = 0.0
    alpha[0, 1, 1] = 0.0
    ic[0, :, 1, 1] = 1.0
    # (1,2): colour error, hit Gaussian 2 (unstable) -> M_c, nothing added
    ic[0, :, 1, 2] = 0.3
    idx[0, 1, 2] = 2
    # (1,3): no depth hit (D_hat = -1), valid D   -> M_s
    Dh[0, 1, 3] = -1.0
    idx[0, 1, 3] = -1
    # colour error just below the threshold: sum 0.29 < 0.3 at (0,0) keeps it out
    ic[0, 0, 0, 0] = 0.29
    unstable = np.array([0, 0, 1], np.uint8)
    return rc, alpha, Dh, idx, ic, D, unstable


def test_masks_and_decisions_by_hand():
    rc, alpha, Dh, idx, ic, D, unstable = _frame()
    m_s, m_c = ad.adding_masks(rc, alpha, Dh, ic, D)
    np.testing.assert_array_equal(m_s[0], [[0, 1, 1, 0], [1, 0, 0, 1]])
    np.testing.assert_array_equal(m_c[0], [[0, 0, 0, 1], [0, 0, 1, 0]])
    cam = Camera(fx=2.0, fy=2.0, cx=1.5, cy=0.5, width=4, height=2, R=np.eye(3, dtype=np.float32),
                 t=np.zeros(3, np.float32))
    out = ad.add_candidates([cam], rc, alpha, Dh, idx, ic, D, unstable, ad.AddParams(sample_rate=1.0))
    # every masked pixel drawn: opaque at (0,1) (0,2) (1,0) (1,3), transparent at (0,3)
    np.testing.assert_array_equal(out["pixel"], [1, 2, 3, 4, 7])
    np.testing.assert_array_equal(out["kind"], [1, 1, 2, 1, 1])
    np.testing.assert_allclose(out["opacity"], np.float32([0.99, 0.99, 0.1, 0.99, 0.99]))
    np.testing.assert_array_equal(out["color"][2], np.full(3, 0.2, np.float32))
    # pixel (x=3, y=0) at D = 2: ((3 - 1.5) / 2 * 2, (0 - 0.5) / 2 * 2, 2)
    np.testing.assert_allclose(out["position"][2], [1.5, -0.5, 2.0])
    none = ad.add_candidates([cam], rc, alpha, Dh, idx, ic, D, unstable, ad.AddParams(sample_rate=0.0))
    assert len(none["pixel"]) == 0


def test_back_projection_with_a_pose():
    """A camera rotated 90 degrees about z and moved: V = R (D K^-1 (x, y, 1)) + t."""
    H, W = 3, 3
    R = np.array([[0, -1, 0], [1, 0, 0], [0, 0, 1]], np.float32)
    t = np.array([1.0, 2.0, 3.0], np.float32)
    cam = Camera(fx=1.0, fy=1.0, cx=1.0, cy=1.0, width=W, height=H, R=R, t=t)
    rc = np.zeros((1, 3, H, W), np.float32)
    alpha = np.zeros((1, H, W), np.float32)  # T_hat = 1: every pixel in M_s
    D = np.full((1, H, W), 4.0, np.float32)
    out = ad.add_candidates([cam], rc, alpha, np.full((1, H, W), -1, np.float32), np.full((1, H, W), -1),
                            rc, D, np.zeros(1, np.uint8), ad.AddParams(sample_rate=1.0))
    assert len(out["pixel"]) == 9
    k = list(out["pixel"]).index(2 * W + 2)  # pixel (x=2, y=2): camera ray (1, 1, 1) * 4
    np.testing.assert_allclose(out["position"][k], R.astype(np.float64) @ [4.0, 4.0, 4.0] + t)


def test_draw_rate_and_threshold():
    assert ad.sample_threshold(0.05) == math.floor(0.05 * 2 ** 24)
    assert ad.sample_threshold(1.0) == 2 ** 24 and ad.sample_threshold(0.0) == 0
    keep = ad.sample_keep(7, 4, 480, 640, 0.05)
    n = keep.size
    # binomial: mean 0.05 n, sd sqrt(n 0.05 0.95) ~ 241; allow 6 sd
    assert abs(int(keep.sum()) - 0.05 * n) < 6 * math.sqrt(n * 0.05 * 0.95)
    # the draws of different frames differ (the counter runs over frames)
    assert not np.array_equal(keep[0], keep[1])
    assert sorted(np.unique(ad.sample_keep(7, 1, 8, 8, 1.0))) == [True]
