"""CPU oracle for the masked, depth-split Gaussian rasterizer — TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, FP64 restatement of what the rasterizer computes,
written from the paper's equations (Section 3.1: the pixel ray, Eq. 1 colour
compositing, Eq. 2 footprint, Eq. 3 transmission, Eq. 4 ray/disc-plane
intersection, Eq. 5 depth cases; Section 3.2: Eq. 7/8 L1 losses; Supplement B:
Eq. S2 unstable-pixel mask and the 50% tile rule; Supplement C: learning rates).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may import it.  It shares no code with the CUDA path and never
imports the product package; the product never imports it.

Parity status per function (pins live in ``tests/test_oracle_pins.py``):
  project            pinned (closed form on the optical axis; Jacobian vs finite differences)
  render             pinned (peak colour, two-layer closed form, telescoping sum,
                     empty scene, early-stop count, planar depth, tilted plane,
                     60-degree rule, transparent-only, hit ellipse, permutation)
  loss_and_grads     pinned (finite differences of the forward; closed-form special cases)
  unstable_mask      pinned (single-disc ellipse closed form; tile rule on a hand-made pattern)
  l1_loss            pinned (hand-computed values)
  adam_step          pinned (torch.optim.Adam on the same gradients)
  global_opt.*       pinned (hand-made error patterns with ties and their masks, exact keep
                     counts, closed-form rotation angles, the keyframe thresholds)
  adding.*           pinned (SplitMix64's published outputs, a hand-made frame with every
                     case of Eq. 6 and the opaque/transparent decision, the draw rate,
                     back-projection in closed form)
  state.*            pinned (hand-made confidence, fusion-weight, error-count, transition and
                     compaction cases)
  sh.*               pinned (the real SH basis against scipy's complex harmonics, the addition
                     theorem, orthonormality by quadrature, a hand colour, the peak colour of
                     one SH Gaussian, SH gradients against central differences, the
                     regulariser's closed form, Adam with split colour rates against
                     torch.optim.Adam)
"""

from .rasterizer import (  # noqa: F401
    Settings,
    project,
    render,
    render_image,
    loss_and_grads,
    l1_loss,
    unstable_mask,
    apply_tile_rule,
    finite_difference_grads,
    decision_signature,
)
from .adam import adam_step, AdamHyper  # noqa: F401
from . import adding, global_opt, sh, state  # noqa: F401
