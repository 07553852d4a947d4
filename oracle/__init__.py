"""Oracle for the time-domain BEM hot path (TEST INFRASTRUCTURE ONLY).

Plain, slow, FP64 CPU code that restates the method of Takahashi, Tanigawa &
Miyazawa (arXiv 2111.05205) from the paper.  Only ``tests/``, the smoke
check of ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may
import it; the CUDA library never does, and the two share no code.

Modules:
  ``coeffs``  B-spline basis and influence coefficients (C core, ctypes)
  ``mot``     marching-on-in-time with the direct (no FMM) history sum
  ``tree``    octree, interaction lists and near-pair lists (integers)
  ``fmm``     plain per-pass definitions of the space-time FMM
"""

from . import coeffs  # noqa: F401
