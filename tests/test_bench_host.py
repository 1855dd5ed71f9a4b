"""Host-side logic of bench.py (CPU): the plain primitive-level hash count
that the i-AABB culling is compared with (Sec. 4.2) against a brute-force
count of the same definition on small scenes."""
import os
import sys
from collections import defaultdict

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
from paper_2201_10022_gb300 import scenes  # noqa: E402


def brute_force(s, q, dhat, h):
    """per cell of edge h: the points (their own cell), the triangles' and
    edges' d-hat-dilated boxes (every cell they cover); point-triangle and
    edge-edge pairs of different bodies sharing a cell, once per shared
    cell"""
    x = bench.vertices(s, q)
    vb = s.vbody
    cell = defaultdict(lambda: ([], [], []))

    def cover(lo, hi):
        a = np.floor(lo / h).astype(int)
        b = np.floor(hi / h).astype(int)
        for i in range(a[0], b[0] + 1):
            for j in range(a[1], b[1] + 1):
                for k in range(a[2], b[2] + 1):
                    yield (i, j, k)

    for v in range(len(x)):
        cell[tuple(np.floor(x[v] / h).astype(int))][0].append(vb[v])
    for t, tv in enumerate(s.tri):
        p = x[tv]
        for c in cover(p.min(axis=0) - dhat, p.max(axis=0) + dhat):
            cell[c][1].append(vb[tv[0]])
    for e, ev in enumerate(s.edge):
        p = x[ev]
        for c in cover(p.min(axis=0) - dhat, p.max(axis=0) + dhat):
            cell[c][2].append(vb[ev[0]])
    pt = ee = 0
    for pts, tris, eds in cell.values():
        pt += sum(1 for a in pts for b in tris if a != b)
        ee += sum(1 for i in range(len(eds)) for j in range(i + 1, len(eds)) if eds[i] != eds[j])
    return pt, ee


@pytest.mark.parametrize("h", [0.07, 0.23])
def test_plain_hash_count_matches_brute_force(h):
    s = scenes.lattice_pile(seed=3, nx=2, ny=2, nz=2, pitch=0.25)
    q = s.q0.copy()
    r = bench.plain_hash_tests(s, q, s.params["dhat"], h=h)
    pt, ee = brute_force(s, q, s.params["dhat"], h)
    assert r["point_triangle"] == pt and r["edge_edge"] == ee
    assert r["box_tests"] == pt + ee > 0
