"""Pins of the oracle's octree and lists (plain definitions, brute force).

- every element lies in the leaf cell its coordinates name;
- neighbour relation symmetric, a cell is its own neighbour;
- interaction lists: at most 189 cells, offsets in [-3,3]^3 minus [-1,1]^3
  (316 possible, Section 4.2 Remark precomp), symmetric;
- completeness of the FMM partition: every ordered element pair (i, j) is
  handled exactly once, either as a near pair (leaf neighbours) or at
  exactly one level l where cell_l(j) is in IL(cell_l(i)).
"""

import itertools

import numpy as np
import pytest

from oracle import coeffs as oc
from oracle import tree as ot
from synth import workload


@pytest.fixture(scope="module", params=[("ellipsoid320_bmbie_d2_hard_plane_s7", 3),
                                        ("sphere1280_obie_d1_dirichlet_uniform", 4)])
def T(request):
    name, L = request.param
    w = workload(name)
    _, xc, _, _ = oc.geometry(w.xyz, w.tri)
    return xc, ot.build(xc, L)


def test_elements_in_their_leaf_cell(T):
    xc, t = T
    L = t["L"]
    h = t["side"] / (1 << L)
    for i, k in enumerate(t["leafkey"]):
        c = np.array(ot.demorton(int(k), L))
        lo = t["lo"] + c * h
        for a in range(3):
            assert lo[a] - 1e-12 <= xc[i, a] <= lo[a] + h + 1e-12


def test_morton_round_trip():
    for c in itertools.product(range(0, 16, 3), repeat=3):
        assert ot.demorton(ot.morton(*c, 4), 4) == c


def test_perm_sorted_by_key_then_index(T):
    _, t = T
    k = [(int(t["leafkey"][i]), int(i)) for i in t["perm"]]
    assert k == sorted(k)


def test_neighbours_and_interaction_lists(T):
    _, t = T
    offsets = set()
    for lev in range(t["L"] + 1):
        keys = t["keys"][lev]
        co = [ot.demorton(int(k), lev) for k in keys]
        for n, lst in enumerate(t["nbr"][lev]):
            assert n in lst
            for m in lst:
                assert n in t["nbr"][lev][m]
                assert max(abs(a - b) for a, b in zip(co[n], co[m])) <= 1
        for n, lst in enumerate(t["il"][lev]):
            assert len(lst) <= 189
            for m in lst:
                d = tuple(a - b for a, b in zip(co[m], co[n]))
                assert max(map(abs, d)) in (2, 3)
                offsets.add(d)
                assert n in t["il"][lev][m]
    assert len(offsets) <= 316


def test_fmm_partition_is_complete_and_disjoint(T):
    xc, t = T
    L = t["L"]
    ns = xc.shape[0]
    cellidx = []
    for lev in range(L + 1):
        index = {int(k): n for n, k in enumerate(t["keys"][lev])}
        cellidx.append([index[int(k) >> (3 * (L - lev))] for k in t["leafkey"]])
    rng = np.random.default_rng(0)
    rows = rng.choice(ns, size=min(ns, 60), replace=False)
    for i in rows:
        near = set(t["near"][i])
        for j in range(ns):
            hits = int(j in near)
            for lev in range(2, L + 1):
                if cellidx[lev][j] in t["il"][lev][cellidx[lev][i]]:
                    hits += 1
            assert hits == 1, (i, j, hits)
