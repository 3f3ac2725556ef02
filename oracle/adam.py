"""Adam on the unstable Gaussians — TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Kingma & Ba, "Adam: A Method for Stochastic Optimization", Algorithm 1, written out in
FP64, applied per parameter group with the learning rates of Supplement C:
lr_position = 1e-3, lr_SH0 (colour) = 5e-4 (Replica/ScanNet++) or 1e-3 (Azure/TUM),
lr_alpha = 0 (opacity is fixed, Section 3.2), lr_scale = 4e-3 or 2e-3, lr_rotation =
1e-3.  Reading: the scale is optimised in log space (theta = log s, the 3DGS
convention the learning rates come from), so its gradient is s * dL/ds and the
update is s <- exp(log s - step); the quaternion is optimised raw (normalised inside
the renderer).  beta = (0.9, 0.999) and eps = 1e-15 follow 3DGS; the paper is silent.
"""

from __future__ import annotations

import dataclasses
from typing import Dict

import numpy as np

GROUPS = ("means", "scales", "quats", "opacity", "colors")


@dataclasses.dataclass(frozen=True)
class AdamHyper:
    lr_means: float = 1e-3
    lr_scales: float = 4e-3
    lr_quats: float = 1e-3
    lr_opacity: float = 0.0
    lr_colors: float = 5e-4
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-15
    # with SH colour: the first colors_dc values of a colour row (the degree-0 coefficients)
    # use lr_colors, the others lr_colors_rest (0.05 lr_SH0, Supplement C); 0 = all lr_colors
    lr_colors_rest: float = 2.5e-5
    colors_dc: int = 0


def adam_step(params: Dict[str, np.ndarray], grads: Dict[str, np.ndarray], m: Dict[str, np.ndarray],
              v: Dict[str, np.ndarray], step: int, hp: AdamHyper = AdamHyper()):
    """One Adam step (``step`` counts from 1) on compact unstable arrays.

    ``params['scales']`` holds linear scales; the optimised variable is their log.
    Returns new (params, m, v) dictionaries in FP64.
    """
    newp, newm, newv = {}, {}, {}
    for name in GROUPS:
        lr = getattr(hp, "lr_" + name)
        x = np.asarray(params[name], dtype=np.float64)
        g = np.asarray(grads[name], dtype=np.float64)
        if name == "scales":
            theta = np.log(x)
            g = g * x
        else:
            theta = x
        mm = hp.beta1 * np.asarray(m[name], dtype=np.float64) + (1 - hp.beta1) * g
        vv = hp.beta2 * np.asarray(v[name], dtype=np.float64) + (1 - hp.beta2) * g * g
        m_hat = mm / (1 - hp.beta1 ** step)
        v_hat = vv / (1 - hp.beta2 ** step)
        if name == "colors" and hp.colors_dc > 0:  # per-coefficient rate within each row
            width = int(np.prod(x.shape[1:])) if x.ndim > 1 else 1
            j = np.arange(width).reshape((1,) + tuple(x.shape[1:])) if x.ndim > 1 else np.zeros(1)
            lr = np.where(j < hp.colors_dc, hp.lr_colors, hp.lr_colors_rest)
        theta = theta - lr * m_hat / (np.sqrt(v_hat) + hp.eps)
        newp[name] = np.exp(theta) if name == "scales" else theta
        newm[name], newv[name] = mm, vv
    return newp, newm, newv
