"""Pins of the oracle's SH colour, transparent regulariser and per-coefficient Adam rates
(paper Section 3.1 view-dependent colour; Section 3.2 L_reg of Eq. 8; Supplement C):
the real SH basis against scipy's complex spherical harmonics, the addition theorem,
orthonormality by quadrature, a hand-computed colour, the regulariser's closed form, and
Adam against torch.optim.Adam with two parameter groups."""

import math

import numpy as np
import scipy.special as sp
import torch

from oracle import AdamHyper, adam_step
from oracle import sh


def _real_from_scipy(l, m, theta, phi):
    """Real SH without the Condon-Shortley phase from scipy's complex Y_l^m (which has it)."""
    if m == 0:
        return sp.sph_harm_y(l, 0, theta, phi).real
    Y = sp.sph_harm_y(l, abs(m), theta, phi)
    sgn = (-1) ** abs(m)
    return math.sqrt(2) * sgn * (Y.real if m > 0 else Y.imag)


def _dirs(n, seed):
    v = np.random.default_rng(seed).normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def test_basis_equals_scipy_real_harmonics():
    d = _dirs(200, 1)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))
    phi = np.arctan2(d[:, 1], d[:, 0])
    Y = sh.sh_basis(torch.as_tensor(d), 3).numpy()
    for l in range(4):
        for m in range(-l, l + 1):
            k = l * l + l + m
            np.testing.assert_allclose(Y[:, k], _real_from_scipy(l, m, theta, phi), atol=1e-12, err_msg=f"l={l} m={m}")


def test_addition_theorem_and_orthonormality():
    d = torch.as_tensor(_dirs(500, 2))
    Y = sh.sh_basis(d, 3)
    for l in range(4):
        band = Y[:, l * l:(l + 1) ** 2]
        np.testing.assert_allclose((band * band).sum(1).numpy(), (2 * l + 1) / (4 * math.pi), rtol=1e-12)
    # Gauss-Legendre x uniform quadrature on the sphere: integral of Y_k Y_j = delta_kj
    xg, wg = np.polynomial.legendre.leggauss(16)
    ph = np.arange(32) * 2 * math.pi / 32
    ct, P = np.meshgrid(xg, ph, indexing="ij")
    st = np.sqrt(1 - ct * ct)
    dirs = np.stack([st * np.cos(P), st * np.sin(P), ct], -1).reshape(-1, 3)
    w = (wg[:, None] * np.full(32, 2 * math.pi / 32)[None, :]).reshape(-1)
    Yq = sh.sh_basis(torch.as_tensor(dirs), 3).numpy()
    G = (Yq * w[:, None]).T @ Yq
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_colour_by_hand():
    # one Gaussian straight along +x from the camera: r = (1, 0, 0); degree 1 coefficients
    coeffs = torch.zeros(1, 4, 3, dtype=torch.float64)
    coeffs[0, 0] = torch.tensor([1.0, 2.0, 3.0])
    coeffs[0, 3] = torch.tensor([0.5, 0.0, -0.5])  # the l=1, m=1 term (x)
    c = sh.sh_colors(coeffs, torch.tensor([[5.0, 1.0, 2.0]], dtype=torch.float64),
                     torch.tensor([1.0, 1.0, 2.0], dtype=torch.float64))
    y0, y1 = 0.5 / math.sqrt(math.pi), math.sqrt(3 / (4 * math.pi))
    np.testing.assert_allclose(c.numpy()[0], [y0 + 0.5 * y1, 2 * y0, 3 * y0 - 0.5 * y1], rtol=1e-14)


def test_transparent_regulariser_closed_form():
    rng = np.random.default_rng(3)
    n = 6
    m0, s0, q0 = rng.normal(size=(n, 3)), rng.uniform(0.01, 0.1, (n, 3)), rng.normal(size=(n, 4))
    m, s, q = m0 + 0.01, s0 * 1.0, q0.copy()
    q[:, 0] += 0.02
    op = np.array([0.1, 0.99, 0.1, 0.99, 0.99, 0.1])
    L, g = sh.transparent_reg(m, s, q, op, m0, s0, q0, w_reg=1000.0)
    # three transparent Gaussians x 10 components: 9 squared diffs of 1e-4 (positions) and
    # 3 of 4e-4 (quaternion w) out of 30
    assert math.isclose(L, 1000 * (9 * 1e-4 + 3 * 4e-4) / 30, rel_tol=1e-12)
    np.testing.assert_allclose(g["means"][op < 0.5], 2 * 1000 * 0.01 / 30, rtol=1e-12)
    assert (g["means"][op > 0.5] == 0).all() and (g["scales"] == 0).all()
    np.testing.assert_allclose(g["quats"][op < 0.5, 0], 2 * 1000 * 0.02 / 30, rtol=1e-12)


def test_adam_split_colour_rates_match_torch():
    rng = np.random.default_rng(4)
    nu, K = 5, 4
    params = {"means": rng.normal(size=(nu, 3)), "scales": rng.uniform(0.01, 0.1, (nu, 3)),
              "quats": rng.normal(size=(nu, 4)), "opacity": rng.uniform(0.1, 1, nu),
              "colors": rng.normal(size=(nu, K, 3))}
    grads = {k: rng.normal(size=v.shape) for k, v in params.items()}
    hp = AdamHyper(colors_dc=3, lr_colors=5e-4, lr_colors_rest=2.5e-5)
    zeros = {k: np.zeros_like(v) for k, v in params.items()}
    newp, _, _ = adam_step(params, grads, zeros, dict(zeros), 1, hp)
    dc = torch.tensor(params["colors"][:, :1], requires_grad=True)
    rest = torch.tensor(params["colors"][:, 1:], requires_grad=True)
    opt = torch.optim.Adam([{"params": [dc], "lr": 5e-4}, {"params": [rest], "lr": 2.5e-5}], betas=(0.9, 0.999),
                           eps=1e-15)
    dc.grad = torch.tensor(grads["colors"][:, :1])
    rest.grad = torch.tensor(grads["colors"][:, 1:])
    opt.step()
    np.testing.assert_allclose(newp["colors"][:, :1], dc.detach().numpy(), rtol=1e-12)
    np.testing.assert_allclose(newp["colors"][:, 1:], rest.detach().numpy(), rtol=1e-12)


def _sh_scene(n, degree, seed):
    import synth
    rng = np.random.default_rng(seed)
    K = (degree + 1) ** 2
    means = np.stack([rng.uniform(-0.3, 0.3, n), rng.uniform(-0.3, 0.3, n), rng.uniform(1.8, 2.6, n)], 1)
    q = rng.normal(size=(n, 4))
    colors = (rng.normal(size=(n, K, 3)) * 0.3).astype(np.float32)
    colors[:, 0] += 1.5
    return synth.Scene(means=means.astype(np.float32), scales=rng.uniform(0.02, 0.06, (n, 3)).astype(np.float32),
                       quats=q.astype(np.float32), opacity=rng.choice([0.99, 0.1], n).astype(np.float32),
                       colors=colors, unstable=np.ones(n, np.uint8))


def test_render_peak_colour_of_one_sh_gaussian():
    import oracle
    import synth
    cam = synth.identity_camera(33, 33, 40.0, 16.0, 16.0)
    s = _sh_scene(1, 3, 5)
    s.means[0] = [0.0, 0.0, 2.0]
    s.opacity[0] = 0.5
    r = oracle.render(s, cam, oracle.Settings(), pixels=np.array([[16, 16]]))
    Y = sh.sh_basis(torch.tensor([[0.0, 0.0, 1.0]], dtype=torch.float64), 3).numpy()[0]
    want = 0.5 * (Y[:, None] * s.colors[0].astype(np.float64)).sum(0)
    np.testing.assert_allclose(r.color.numpy()[0], want, rtol=1e-12)


def test_sh_gradients_against_finite_differences():
    """The analytic gradient of the L1 loss with respect to SH coefficients and positions
    (through the view direction as well as the footprint) against central differences."""
    import oracle
    import synth
    cam = synth.identity_camera(24, 24, 30.0, 11.5, 11.5)
    s = _sh_scene(12, 2, 6)
    st = oracle.Settings()
    ys, xs = np.mgrid[0:24:3, 0:24:3]
    pix = np.stack([xs.ravel(), ys.ravel()], 1)
    rng = np.random.default_rng(7)
    tc = rng.uniform(0, 1, (len(pix), 3))
    td = rng.uniform(1.5, 3, len(pix))
    ref = oracle.loss_and_grads(s, cam, st, pix, tc, td)
    which = [("colors", i, c) for i in range(0, 12, 3) for c in (0, 4, 13, 26)] + \
            [("means", i, c) for i in range(0, 12, 4) for c in range(3)]
    fd, stable = oracle.finite_difference_grads(s, cam, st, pix, tc, td, which)
    got = np.array([ref["grads"][nm][gi].reshape(-1)[c] for nm, gi, c in which])
    assert stable.mean() > 0.8
    scale = np.abs(fd[stable]).max()
    assert scale > 0
    np.testing.assert_allclose(got[stable], fd[stable], rtol=1e-5, atol=1e-6 * scale)
