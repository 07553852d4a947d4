"""Octree, neighbour and interaction lists of the space-time FMM (oracle,
TEST INFRASTRUCTURE ONLY).

The spatial hierarchy of the interpolation-based FMM (Section 3, Fig. 2;
the interaction list of at most 189 cells over 316 relative offsets of
Section 4.2, Remark precomp, and Algorithm 1).  The paper defers the
construction to its earlier study, so the definition here is the reading
used by this project, written out plainly:

- root cube: lo = componentwise minimum of the collocation points,
  side = (largest extent over the three axes) * (1 + 2^-20);
- leaf level L (root = level 0); element i sits in the leaf cell with
  integer coordinates c_k = floor((x_ik - lo_k) / side * 2^L), clamped to
  [0, 2^L - 1], computed in FP64 without fused operations;
- Morton key: bit b of c_x, c_y, c_z goes to bit 3b, 3b+1, 3b+2;
- elements ordered by (leaf key, element index);
- at level l the cell of an element is its leaf key >> 3 (L - l); the
  occupied cells of a level are the distinct such keys in increasing order;
- neighbours N(O): occupied cells of the same level whose coordinates
  differ from O's by at most 1 in every axis (O included), by key;
- interaction list IL(O), level >= 2: occupied children of the neighbours
  of O's parent that are not neighbours of O, by key (relative offsets in
  [-3, 3]^3 minus [-1, 1]^3: 316 possible, at most 189 occupied);
- near list of element i: every element of the leaf cells in N(leaf(i)), in
  the order of the cells' keys and, within a cell, the element order.
"""

import numpy as np


def morton(cx, cy, cz, bits):
    k = 0
    for b in range(bits):
        k |= ((cx >> b) & 1) << (3 * b)
        k |= ((cy >> b) & 1) << (3 * b + 1)
        k |= ((cz >> b) & 1) << (3 * b + 2)
    return k


def demorton(k, bits):
    c = [0, 0, 0]
    for b in range(bits):
        for a in range(3):
            c[a] |= ((k >> (3 * b + a)) & 1) << b
    return tuple(c)


def root_box(xc):
    lo = xc.min(axis=0)
    ext = xc.max(axis=0) - lo
    side = float(ext.max()) * (1.0 + 2.0 ** -20)
    return lo, side


def leaf_coords(xc, L):
    lo, side = root_box(xc)
    n = 1 << L
    c = np.floor((xc - lo[None, :]) / side * float(n)).astype(np.int64)
    return np.clip(c, 0, n - 1)


def build(xc, L):
    """Returns a dict with the element order ``perm`` and, per level l in
    0..L, ``keys[l]`` (occupied cells), ``start[l]`` (first position in
    ``perm`` of each cell, plus the end), ``nbr[l]`` / ``il[l]`` as lists of
    lists of cell indices of that level, and ``near`` as a list (per element
    in original numbering) of element lists."""
    xc = np.asarray(xc, dtype=np.float64)
    ns = xc.shape[0]
    c = leaf_coords(xc, L)
    leaf = np.array([morton(int(a), int(b), int(d), L) for a, b, d in c], dtype=np.int64)
    perm = sorted(range(ns), key=lambda i: (int(leaf[i]), i))
    T = {"L": L, "perm": np.array(perm, dtype=np.int64), "leafkey": leaf, "keys": [], "start": [], "nbr": [],
         "il": [], "lo": root_box(xc)[0], "side": root_box(xc)[1]}
    for lev in range(L + 1):
        sh = 3 * (L - lev)
        ck = [int(leaf[i]) >> sh for i in perm]
        keys, start = [], []
        for p, k in enumerate(ck):
            if not keys or k != keys[-1]:
                keys.append(k)
                start.append(p)
        start.append(ns)
        index = {k: n for n, k in enumerate(keys)}
        coords = [demorton(k, lev) for k in keys]
        nbr = []
        for (x, y, z) in coords:
            found = []
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        q = (x + dx, y + dy, z + dz)
                        if min(q) < 0 or max(q) >= (1 << lev):
                            continue
                        kk = morton(q[0], q[1], q[2], lev)
                        if kk in index:
                            found.append(kk)
            nbr.append([index[kk] for kk in sorted(found)])
        il = []
        for n, (x, y, z) in enumerate(coords):
            if lev < 2:
                il.append([])
                continue
            pk = keys[n] >> 3
            pidx = {k: m for m, k in enumerate(T["keys"][lev - 1])}
            pn = T["nbr"][lev - 1][pidx[pk]]
            cand = []
            for m in pn:
                pkey = T["keys"][lev - 1][m]
                for ch in range(8):
                    kk = (pkey << 3) | ch
                    if kk not in index:
                        continue
                    q = demorton(kk, lev)
                    if max(abs(q[0] - x), abs(q[1] - y), abs(q[2] - z)) <= 1:
                        continue
                    cand.append(kk)
            il.append([index[kk] for kk in sorted(cand)])
        T["keys"].append(np.array(keys, dtype=np.int64))
        T["start"].append(np.array(start, dtype=np.int64))
        T["nbr"].append(nbr)
        T["il"].append(il)
    # near lists at the leaf level
    keysL = T["keys"][L]
    cell_of_pos = np.searchsorted(T["start"][L], np.arange(ns), side="right") - 1
    near = [None] * ns
    for p, i in enumerate(perm):
        cell = cell_of_pos[p]
        lst = []
        for m in T["nbr"][L][cell]:
            lst.extend(perm[T["start"][L][m]:T["start"][L][m + 1]])
        near[i] = lst
    T["near"] = near
    del keysL
    return T
