"""Pins of the oracle's candidate sets (Sec. 4.2 culling) against all-pairs
brute force, and of its additive CCD (Sec. 4.1) against a sampled
time-of-impact search."""
import numpy as np
import pytest

import oracle as O
from paper_2201_10022_gb300 import scenes


def _canon(pairs):
    return set(map(tuple, np.asarray(pairs).tolist()))


@pytest.mark.parametrize("seed,kinds", [(0, ("cube", "cube")), (1, ("cube", "ico1")), (2, ("ico1", "ico1")),
                                        (3, ("box", "cube")), (4, ("tet", "ico1"))])
def test_culled_candidates_equal_brute_force(seed, kinds):
    s = scenes.random_pair(seed, kinds=kinds, sep=0.0004)
    o = O.Oracle(s)
    x = o.vertices(s.q0)
    c = o.candidates(x)
    b = o.candidates(x, brute=True)
    assert len(c) > 0
    assert _canon(c) == _canon(b)
    # swept sets too
    rng = np.random.default_rng(seed)
    dq = rng.normal(size=s.q0.shape) * 0.01
    x1 = x + o.displacements(dq)
    assert _canon(o.candidates(x, x1)) == _canon(o.candidates(x, x1, brute=True))


def test_cube_stack_candidates_equal_brute_force():
    s = scenes.cube_stack(seed=1, gap=0.0005)
    o = O.Oracle(s)
    x = o.vertices(s.q0)
    c = o.candidates(x)
    assert len(c) > 0
    assert _canon(c) == _canon(o.candidates(x, brute=True))
    # every pair is inter-body and not static-static, EE pairs ordered by body
    for kind, i, j in c:
        if kind == 0:
            a, b = s.vbody[i], s.vbody[s.tri[j, 0]]
            assert a != b
        else:
            a, b = s.vbody[s.edge[i, 0]], s.vbody[s.edge[j, 0]]
            assert a < b
        assert not (s.is_static[a] and s.is_static[b])


def _min_dist_on_segment(kind, x, dx, n=100001):
    ts = np.linspace(0.0, 1.0, n)
    d = np.array([np.sqrt(O.pair_dist2(kind, x + t * dx)[0]) for t in ts])
    return ts, d


def test_accd_is_conservative_against_sampled_toi():
    rng = np.random.default_rng(21)
    n_hit = 0
    for trial in range(60):
        kind = trial % 2
        x = rng.normal(size=12) * 0.1
        # aim the first primitive through the second one
        x2 = x.reshape(4, 3)
        tgt = x2[1:].mean(axis=0) if kind == 0 else x2[2:].mean(axis=0)
        src = x2[0] if kind == 0 else x2[:2].mean(axis=0)
        dx = np.zeros((4, 3))
        mv = (tgt - src) * rng.uniform(1.2, 2.0) + rng.normal(size=3) * 0.02
        if kind == 0:
            dx[0] = mv
        else:
            dx[:2] = mv
        dx = dx.ravel() + rng.normal(size=12) * 0.005
        toi, st = O.accd(kind, x, dx)
        assert st == 0 and 0.0 < toi <= 1.0
        ts, d = _min_dist_on_segment(kind, x, dx, n=20001)
        d0 = d[0]
        # ACCD never passes the first time the distance reaches s*d0 ...
        below = np.nonzero(d < 0.1 * d0 * (1 - 1e-9))[0]
        if len(below):
            n_hit += 1
            assert toi <= ts[below[0]] + 1e-12
        else:
            assert toi == 1.0 or d[ts <= toi + 1e-12].min() >= 0.1 * d0 * (1 - 1e-6)
        # ... and the gap at the returned time is at least s*d0
        dt = np.sqrt(O.pair_dist2(kind, x + toi * dx)[0])
        assert dt >= 0.1 * d0 * (1 - 1e-9)
    assert n_hit > 10


def test_accd_no_motion_and_far_apart():
    x = np.array([0, 0, 1.0, 0, 0, 0, 1, 0, 0, 0, 1, 0])
    assert O.accd(0, x, np.zeros(12))[0] == 1.0
    dx = np.tile([0.1, 0.0, 0.0], 4)  # common translation only
    assert O.accd(0, x, dx)[0] == 1.0
    dx = np.zeros(12)
    dx[2] = -0.1  # moves 0.1 towards a plane 1.0 away
    assert O.accd(0, x, dx)[0] == 1.0
