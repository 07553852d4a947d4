"""GB300-native time-domain BEM for the 3-D wave equation (Takahashi,
Tanigawa & Miyazawa, arXiv 2111.05205): CUDA library libtdbem (sm_103a)
behind a C ABI (include/tdbem.h), with this thin ctypes binding.

``abi``     one Python function per C entry point (marshalling only)
``solver``  a convenience wrapper owning one context
``build``   in-tree nvcc build of libtdbem.so
"""

from . import abi, build  # noqa: F401
from .solver import Solver  # noqa: F401
