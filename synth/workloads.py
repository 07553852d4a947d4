"""Seeded workload recipes: mesh, wave speed, time step, boundary data.

A workload fixes the inputs of one time-domain BEM run (Section 2.1): the
triangulated surface S, the wave speed c, the step length dt, the number of
steps Nt, the B-spline order d, the integral equation (OBIE, Eq. bie, or
BMBIE, Eq. bmbie), the boundary condition and the excitation.  The
excitation is either

* ``"uniform"``: prescribed data f(t) = exp(-((t - 4 sigma) / sigma)^2) that is
  the same on every element (known u for Dirichlet, known du/dr for
  Neumann), no incident wave; or
* ``"plane"``: a plane Gaussian pulse u_in(x, t) = exp(-((t - t0 - k.x/c) /
  sigma)^2) hitting a sound-soft (u = 0) or sound-hard (q = 0) scatterer.

The step rule is c dt = 0.5 x (mean edge length).  Nothing here evaluates
the method; only the numbers that define its inputs are produced.
"""

from dataclasses import dataclass, field

import numpy as np

from .meshes import ellipsoid, geodesic, icosphere, mean_edge


@dataclass
class Workload:
    name: str
    xyz: np.ndarray
    tri: np.ndarray
    c: float
    dt: float
    nt: int
    d: int
    bie: str  # "obie" | "bmbie"
    bc: str  # "dirichlet" | "neumann"
    excitation: str  # "uniform" | "plane"
    sigma: float  # Gaussian width, or the raised cosine's pulse length (shape 1)
    t0: float = 0.0
    direction: np.ndarray = field(default_factory=lambda: np.array([1.0, 0.0, 0.0]))
    # space-time FMM parameters (leaf level, nodes per dimension, mu)
    depth: int = 0
    ps: int = 0
    pt: int = 0
    mu: int = 8
    # incident pulse profile: 0 Gaussian, 1 raised cosine (Section 5.1.1)
    shape: int = 0

    @property
    def ns(self):
        return int(self.tri.shape[0])


def _unit(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def workload(name, nt=None):
    """Build one of the named workloads; ``nt`` overrides the step count."""
    c = 1.0
    if name == "sphere320_obie_d1_dirichlet_uniform":
        # icosphere radius 1, 320 flat triangles, OBIE d=1, u = f(t) on S
        xyz, tri = icosphere(2)
        w = Workload(name, xyz, tri, c, 0.5 * mean_edge(xyz, tri) / c, 64, 1,
                     "obie", "dirichlet", "uniform", sigma=0.5)
    elif name.startswith("sphere") and "_uniform" in name:
        # e.g. sphere1280_bmbie_d1_neumann_uniform
        parts = name.split("_")
        ns = int(parts[0][len("sphere"):])
        subdiv = {80: 1, 320: 2, 1280: 3, 5120: 4, 20480: 5}[ns]
        d = int(parts[2][1:])
        xyz, tri = icosphere(subdiv)
        w = Workload(name, xyz, tri, c, 0.5 * mean_edge(xyz, tri) / c, 64, d,
                     parts[1], parts[3], "uniform", sigma=0.5)
    elif name.startswith("sphere") and "_plane" in name and name != "sphere5120_bmbie_d1_soft_plane":
        # icospheres (radius 1) under the seeded Gaussian plane pulse, e.g. the
        # 81920-element sphere sphere81920_bmbie_d2_hard_plane
        parts = name.split("_")
        ns = int(parts[0][len("sphere"):])
        subdiv = {80: 1, 320: 2, 1280: 3, 5120: 4, 20480: 5, 81920: 6}[ns]
        seed = int(parts[-1][1:]) if parts[-1].startswith("s") else 0
        xyz, tri = icosphere(subdiv)
        rng = np.random.default_rng(seed)
        sig = 0.3
        bc = {"hard": "neumann", "soft": "dirichlet"}[parts[3]]
        w = Workload(name, xyz, tri, c, 0.5 * mean_edge(xyz, tri) / c, 2048, int(parts[2][1:]),
                     parts[1], bc, "plane", sigma=sig,
                     t0=4 * sig + float(np.linalg.norm(xyz, axis=1).max()) / c,
                     direction=_unit(rng))
    elif name == "sphere5120_bmbie_d1_soft_plane":
        xyz, tri = icosphere(4)
        rng = np.random.default_rng(2)
        sig = 0.3
        w = Workload(name, xyz, tri, c, 0.5 * mean_edge(xyz, tri) / c, 512, 1,
                     "bmbie", "dirichlet", "plane", sigma=sig,
                     t0=4 * sig + float(np.linalg.norm(xyz, axis=1).max()) / c,
                     direction=_unit(rng), depth=4, ps=4, pt=4)
    elif name == "ellipsoid20480_bmbie_d2_hard_plane":
        xyz, tri, _ = ellipsoid(5, seed=3)
        rng = np.random.default_rng(3)
        sig = 0.3
        w = Workload(name, xyz, tri, c, 0.5 * mean_edge(xyz, tri) / c, 1024, 2,
                     "bmbie", "neumann", "plane", sigma=sig,
                     t0=4 * sig + float(np.linalg.norm(xyz, axis=1).max()) / c,
                     direction=_unit(rng), depth=5, ps=5, pt=5)
    elif name.startswith("paper_sphere"):
        # the sphere example of Section 5.1.1: radius 0.5, centre (0.5, 0, 0),
        # geodesic mesh of 2880 / 5120 / 11520 elements, dt = 0.04 / 0.03 /
        # 0.02 and Nt = 240 / 320 / 480 (analysis time 9.6), raised-cosine
        # plane pulse along +x_1 of length 0.5 with t0 = 0 (Eq. uin);
        # e.g. paper_sphere2880_bmbie_d2_hard
        parts = name.split("_")
        ns = int(parts[1][len("sphere"):])
        n, dt, steps = {2880: (12, 0.04, 240), 5120: (16, 0.03, 320), 11520: (24, 0.02, 480),
                        80: (2, 0.25, 40), 320: (4, 0.12, 80)}[ns]
        xyz, tri = geodesic(n, radius=0.5, center=(0.5, 0.0, 0.0))
        bc = {"hard": "neumann", "soft": "dirichlet"}[parts[4]]
        w = Workload(name, xyz, tri, c, dt, steps, int(parts[3][1:]), parts[2], bc, "plane", sigma=0.5, t0=0.0,
                     direction=np.array([1.0, 0.0, 0.0]), shape=1)
    elif name.startswith("ellipsoid") and "_plane" in name:
        # small seeded ellipsoids for tests, e.g. ellipsoid320_bmbie_d2_hard_plane_s7
        parts = name.split("_")
        ns = int(parts[0][len("ellipsoid"):])
        subdiv = {80: 1, 320: 2, 1280: 3, 5120: 4, 20480: 5}[ns]
        seed = int(parts[-1][1:]) if parts[-1].startswith("s") else 0
        d = int(parts[2][1:])
        xyz, tri, _ = ellipsoid(subdiv, seed=seed)
        rng = np.random.default_rng(seed)
        sig = 0.3
        bc = {"hard": "neumann", "soft": "dirichlet"}[parts[3]]
        w = Workload(name, xyz, tri, c, 0.5 * mean_edge(xyz, tri) / c, 64, d,
                     parts[1], bc, "plane", sigma=sig,
                     t0=4 * sig + float(np.linalg.norm(xyz, axis=1).max()) / c,
                     direction=_unit(rng))
    else:
        raise KeyError(name)
    if nt is not None:
        w.nt = int(nt)
    return w
