"""The oracle: a plain, slow FP64 CPU statement of the R^2-Gaussian hot path.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline / reference leg of ``bench.py`` may import it.  It shares no
code with the CUDA library; the two meet only at the seeded input generators in
``paper_2405_20693_b300.inputs``.

Pins (tests/test_oracle_pins.py) tie each function to something other than
itself:
  * O2 closed-form ray integral == O3 quadrature (FP64, 1e-12);
  * O1 parallel beam, no gate == O2 exactly; mu by determinants == mu by the
    ray-direction identity; cone-beam O1 vs O2 error shrinks ~4x when scales halve;
    the wrong third Jacobian row shows the predicted 1/cos bias;
  * projected mass == sum rho (2 pi)^{3/2} sqrt|Sigma|;
  * scatter form == all-pixels / all-voxels brute force; invariants (isotropic
    view-independence, permutation, z-rotation vs angle shift, theta vs theta+pi mirror);
  * hand adjoints == complex-step derivatives (rasterizer, voxelizer, SSIM, TV);
  * SSIM(x, x) = 1 with zero gradient; phantom chords == quadrature of the indicator.
  * the FP32 tile-bound replica is pinned to the FP64 projection (same p^, Sigma^
    to FP32 rounding) and to the gate: every pixel with q <= Q lies in its box.
  * the Adam step: a constant gradient moves every raw parameter by exactly
    -lr g / (|g| + eps), and two steps with different gradients match the unrolled
    closed form of the moment recursions (which fixes both decay rates).
"""
from . import core, losses  # noqa: F401
from .core import build  # noqa: F401
