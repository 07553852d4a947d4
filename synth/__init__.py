"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package only builds inputs: triangle meshes (icospheres and seeded
ellipsoids), the time-step rule and the parameters of the incident pulse or
of the prescribed boundary data.  It holds none of the method's arithmetic
(no geometry of the collocation scheme, no B-splines, no influence
coefficients, no time marching); both sides compute those on their own.
"""

from .meshes import icosphere, ellipsoid, mean_edge  # noqa: F401
from .workloads import Workload, workload  # noqa: F401
