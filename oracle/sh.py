"""View-dependent colour by spherical harmonics and the transparent-Gaussian regulariser
(paper Section 3.1 colour c_i from the view direction r_i and the SH coefficients; Section
3.2, the L_reg term of Eq. 8; Supplement C learning rates): TEST INFRASTRUCTURE ONLY, like
the rest of this package.

Readings (the paper builds on 3DGS and gives no formulas):
  - the basis is the real, orthonormal spherical harmonics up to degree 3 without the
    Condon-Shortley phase, ordered k = l^2 + l + m; the colour of Gaussian i seen from a
    camera centred at t is c = sum_k SH_i[k] Y_k(r), r = (p_i - t) / |p_i - t|, with no
    offset and no clamping (transparent Gaussians carry signed residual colours);
  - L_reg is the mean squared difference over the position, rotation (raw quaternion) and
    scale components of the optimised transparent Gaussians (opacity < 0.5) from their
    values when they were added, weighted by w_reg = 1000;
  - Adam uses lr_SH0 for the three degree-0 coefficients and 0.05 lr_SH0 for the others.
"""

from __future__ import annotations

import math

import numpy as np
import torch

DT = torch.float64


def n_coeffs(degree: int) -> int:
    return (degree + 1) ** 2


def sh_basis(dirs: torch.Tensor, degree: int) -> torch.Tensor:
    """[m, (degree+1)^2] real SH of unit directions [m, 3] (differentiable)."""
    x, y, z = dirs[:, 0], dirs[:, 1], dirs[:, 2]
    one = torch.ones_like(x)
    out = [one * (0.5 / math.sqrt(math.pi))]
    if degree >= 1:
        c1 = math.sqrt(3.0 / (4.0 * math.pi))
        out += [c1 * y, c1 * z, c1 * x]
    if degree >= 2:
        a = 0.5 * math.sqrt(15.0 / math.pi)
        b = 0.25 * math.sqrt(5.0 / math.pi)
        c = 0.25 * math.sqrt(15.0 / math.pi)
        out += [a * x * y, a * y * z, b * (3 * z * z - 1), a * x * z, c * (x * x - y * y)]
    if degree >= 3:
        a = 0.25 * math.sqrt(35.0 / (2.0 * math.pi))
        b = 0.5 * math.sqrt(105.0 / math.pi)
        c = 0.25 * math.sqrt(21.0 / (2.0 * math.pi))
        d = 0.25 * math.sqrt(7.0 / math.pi)
        e = 0.25 * math.sqrt(105.0 / math.pi)
        out += [a * y * (3 * x * x - y * y), b * x * y * z, c * y * (5 * z * z - 1), d * z * (5 * z * z - 3),
                c * x * (5 * z * z - 1), e * z * (x * x - y * y), a * x * (x * x - 3 * y * y)]
    return torch.stack(out, 1)


def degree_of(coeffs) -> int:
    K = coeffs.shape[1]
    d = int(round(math.sqrt(K))) - 1
    if (d + 1) ** 2 != K or not 1 <= d <= 3:
        raise ValueError(f"{K} SH coefficients per channel is not a degree 1..3 set")
    return d


def sh_colors(coeffs: torch.Tensor, means: torch.Tensor, cam_t: torch.Tensor) -> torch.Tensor:
    """[n, 3] colours seen from the camera centre cam_t: coeffs [n, K, 3], means [n, 3]."""
    d = means - cam_t
    r = d / torch.linalg.vector_norm(d, dim=1, keepdim=True)
    Y = sh_basis(r, degree_of(coeffs))  # [n, K]
    return torch.einsum("nk,nkc->nc", Y, coeffs)


def transparent_reg(means, scales, quats, opacity, means0, scales0, quats0, w_reg: float = 1000.0,
                    alpha_split: float = 0.5):
    """(w_reg * L_reg, gradients {means, scales, quats}) over the optimised Gaussians whose
    opacity is below alpha_split, in FP64."""
    t = lambda a: torch.as_tensor(np.asarray(a), dtype=DT)  # noqa: E731
    m, s, q = (t(a).clone().requires_grad_(True) for a in (means, scales, quats))
    sel = t(opacity) < alpha_split
    if int(sel.sum()) == 0:
        z = {k: np.zeros(np.asarray(a).shape) for k, a in (("means", means), ("scales", scales), ("quats", quats))}
        return 0.0, z
    diff = torch.cat([(m - t(means0))[sel], (q - t(quats0))[sel], (s - t(scales0))[sel]], 1)
    L = w_reg * (diff * diff).mean()
    L.backward()
    return float(L.detach()), {"means": m.grad.numpy(), "scales": s.grad.numpy(), "quats": q.grad.numpy()}
