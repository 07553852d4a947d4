"""Seeded triangle meshes: icospheres, geodesic spheres and ellipsoids.

Every mesh is returned as ``(xyz, tri)`` with ``xyz`` a float64 array
``[nv, 3]`` and ``tri`` an int32 array ``[ns, 3]``.  Triangles are ordered
counter-clockwise when seen from outside the enclosed domain V, so that
``(v1 - v0) x (v2 - v0)`` points out of V.  These are the sphere-shaped
scatterers of the paper's numerical examples (Section 5.1), with flat
elements whose vertices lie on the surface.
"""

import numpy as np

_PHI = (1.0 + 5.0 ** 0.5) / 2.0


def _icosahedron():
    v = np.array(
        [
            [-1, _PHI, 0], [1, _PHI, 0], [-1, -_PHI, 0], [1, -_PHI, 0],
            [0, -1, _PHI], [0, 1, _PHI], [0, -1, -_PHI], [0, 1, -_PHI],
            [_PHI, 0, -1], [_PHI, 0, 1], [-_PHI, 0, -1], [-_PHI, 0, 1],
        ],
        dtype=np.float64,
    )
    f = np.array(
        [
            [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
            [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
            [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
            [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
        ],
        dtype=np.int64,
    )
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v, f


def icosphere(subdiv, radius=1.0, center=(0.0, 0.0, 0.0)):
    """Unit icosahedron refined ``subdiv`` times by edge midpoints.

    Returns 20 * 4**subdiv flat triangles whose vertices lie on the sphere
    of the given radius and centre.
    """
    v, f = _icosahedron()
    verts = [tuple(p) for p in v]
    for _ in range(int(subdiv)):
        cache = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                p = (np.asarray(verts[a]) + np.asarray(verts[b])) * 0.5
                p /= np.linalg.norm(p)
                cache[key] = len(verts)
                verts.append(tuple(p))
            return cache[key]

        nf = []
        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
        f = np.array(nf, dtype=np.int64)
    xyz = np.asarray(verts, dtype=np.float64) * float(radius) + np.asarray(center, dtype=np.float64)
    return xyz, f.astype(np.int32)


def geodesic(n, radius=1.0, center=(0.0, 0.0, 0.0)):
    """Geodesic sphere with 20 n^2 flat triangles: every face of the
    icosahedron cut into n^2 triangles by its n-fold edge subdivision, the
    vertices pushed out to the sphere (n = 12, 16, 24 give the element
    counts 2880, 5120 and 11520 of the paper's sphere, Section 5.1.1)."""
    v, f = _icosahedron()
    verts, index = [], {}

    def vert(a, b, c, i, j):
        # point i/n along a->b and j/n along a->c of face (a, b, c), keyed
        # by its barycentric weights on the global vertices (shared edges)
        wts = {a: n - i - j, b: i, c: j}
        key = tuple(sorted((g, w) for g, w in wts.items() if w))
        if key not in index:
            p = sum(v[g] * w for g, w in wts.items()) / n
            index[key] = len(verts)
            verts.append(p / np.linalg.norm(p))
        return index[key]

    tris = []
    for a, b, c in f:
        for i in range(n):
            for j in range(n - i):
                p0, p1, p2 = vert(a, b, c, i, j), vert(a, b, c, i + 1, j), vert(a, b, c, i, j + 1)
                tris.append([p0, p1, p2])
                if i + j + 1 < n:
                    p3 = vert(a, b, c, i + 1, j + 1)
                    tris.append([p1, p3, p2])
    xyz = np.asarray(verts) * float(radius) + np.asarray(center, dtype=np.float64)
    return xyz, np.asarray(tris, dtype=np.int32)


def ellipsoid(subdiv, seed, lo=0.5, hi=1.5):
    """Icosphere mapped by (x, y, z) -> (a x, b y, c z), a, b, c ~ U[lo, hi].

    The axes are drawn from ``numpy.random.default_rng(seed)``; the map keeps
    the outward orientation of the triangles.  Returns ``(xyz, tri, axes)``.
    """
    xyz, tri = icosphere(subdiv)
    axes = np.random.default_rng(seed).uniform(lo, hi, size=3)
    return xyz * axes[None, :], tri, axes


def mean_edge(xyz, tri):
    """Mean length over the unique edges of the mesh."""
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
    e = np.unique(np.sort(e, axis=1), axis=0)
    return float(np.linalg.norm(xyz[e[:, 0]] - xyz[e[:, 1]], axis=1).mean())
