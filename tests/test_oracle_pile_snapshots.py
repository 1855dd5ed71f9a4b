"""The lattice-pile snapshots (tests/golden/pile_snapshots.npz, written by
tests/golden/make_pile_snapshots.py from the oracle alone) cover the regimes
the benchmark's time steps run through: free fall, first ground impacts,
ground contact with friction and body-body stacking with friction between
dynamic bodies (checked on the oracle's own lagged friction sets)."""
import os

import numpy as np

import oracle as O
from paper_2201_10022_gb300 import scenes

HERE = os.path.dirname(os.path.abspath(__file__))
SNAP = np.load(os.path.join(HERE, "golden", "pile_snapshots.npz"))
STEPS = [int(k) for k in SNAP["steps"]]


def _pair_bodies(s, kind, i, j):
    if kind == 0:
        return s.vbody[i], s.vbody[s.tri[j][0]]
    return s.vbody[s.edge[i][0]], s.vbody[s.edge[j][0]]


def test_pile_snapshots_cover_the_regimes():
    d = SNAP["dims"]
    s = scenes.lattice_pile(seed=3, nx=int(d[0]), ny=int(d[1]), nz=int(d[2]))
    orc = O.Oracle(s)
    assert abs(orc.l_bbox - float(SNAP["l_bbox"])) <= 1e-12 * orc.l_bbox
    counts = []
    for step in STEPS:
        q, qd = SNAP[f"q_{step}"], SNAP[f"qdot_{step}"]
        assert q.shape == (s.nb, 12) and np.isfinite(q).all() and np.isfinite(qd).all()
        orc.set_state(q, qd)
        fr = orc.pairs(2)
        dyn_dyn = sum(1 for k in range(len(fr["kind"]))
                      if not any(s.is_static[b] for b in _pair_bodies(s, int(fr["kind"][k]), int(fr["i"][k]),
                                                                      int(fr["j"][k]))))
        counts.append((len(fr["kind"]), dyn_dyn))
    assert counts[0] == (0, 0), counts          # free fall
    assert counts[1][0] > 0, counts             # first impacts
    assert counts[2][0] > counts[1][0], counts  # more ground contact
    assert counts[3][1] > 0, counts             # friction between dynamic bodies
