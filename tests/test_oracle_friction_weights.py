"""Pins of the oracle's friction closest-point weights (Sec. 4, lagged
friction: the tangent offset of a pair is sum_v gamma_v x_v, the vector from
the closest point on the second primitive to the closest point on the first).

For every distance type (point-triangle 0..6, edge-edge 0..8) the weights are
checked against a library minimiser of the primitive-to-primitive distance
over the primitives' parameter domains (scipy SLSQP on the barycentric
simplex, L-BFGS-B on the square of segment parameters), started from the best
point of a dense grid: the gap vector must equal the minimiser's, its squared
norm the oracle's d^2, and the weights must form the convex combinations the
type names (exact 0/1 at vertices).  A swapped s/t, a wrong edge index or a
wrong sign in any branch moves the gap vector by the primitives' size."""
import numpy as np
import pytest

import oracle as O

scipy_opt = pytest.importorskip("scipy.optimize")


def _pt_min(x):
    """closest-point gap of point x[0] to triangle x[1..3] by SLSQP over the simplex"""
    p, a, b, c = x

    def f(l):
        d = p - (l[0] * a + l[1] * b + (1.0 - l[0] - l[1]) * c)
        return d @ d

    g = np.linspace(0.0, 1.0, 61)
    best = min(((u, v) for u in g for v in g if u + v <= 1.0), key=f)
    r = scipy_opt.minimize(f, np.array(best), method="SLSQP", bounds=[(0, 1), (0, 1)],
                           constraints=[{"type": "ineq", "fun": lambda l: 1.0 - l[0] - l[1]}],
                           options={"ftol": 1e-16, "maxiter": 500})
    l = r.x if f(r.x) <= f(np.array(best)) else np.array(best)
    return p - (l[0] * a + l[1] * b + (1.0 - l[0] - l[1]) * c)


def _ee_min(x):
    """closest-point gap of segment (x0,x1) to segment (x2,x3) by L-BFGS-B on [0,1]^2"""
    x0, x1, x2, x3 = x

    def gap(st):
        return (x0 + st[0] * (x1 - x0)) - (x2 + st[1] * (x3 - x2))

    def f(st):
        d = gap(st)
        return d @ d

    g = np.linspace(0.0, 1.0, 81)
    best = min(((u, v) for u in g for v in g), key=f)
    r = scipy_opt.minimize(f, np.array(best), method="L-BFGS-B", bounds=[(0, 1), (0, 1)],
                           options={"ftol": 1e-18, "gtol": 1e-14, "maxiter": 1000})
    st = r.x if f(r.x) <= f(np.array(best)) else np.array(best)
    return gap(st)


def _configs(kind, n, rng):
    out = []
    for _ in range(n):
        x = rng.uniform(-1.0, 1.0, size=(4, 3))
        if kind == O.ORC_PT:
            # the point near the triangle's plane, anywhere around it
            x[0] = x[1:].mean(axis=0) + rng.uniform(-1.5, 1.5, 3) * np.array([1.0, 1.0, 0.3])
        out.append(x)
    return out


def _parallel_ee(rng):
    """edges along one direction, offset sideways: the parallel branch"""
    out = []
    for k in range(40):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        w = np.cross(u, rng.normal(size=3))
        w /= np.linalg.norm(w)
        a = rng.uniform(-1, 1, 3)
        s0, s1 = sorted(rng.uniform(-1, 1, 2))
        t0, t1 = sorted(rng.uniform(-1, 1, 2))
        if k % 2:
            t0, t1 = t1, t0
        x = np.array([a + s0 * u, a + s1 * u, a + 0.3 * w + t0 * u, a + 0.3 * w + t1 * u])
        out.append(x)
    return out


@pytest.mark.parametrize("kind,ntypes", [(O.ORC_PT, 7), (O.ORC_EE, 9)])
def test_closest_weights_match_minimiser(kind, ntypes):
    rng = np.random.default_rng(17 + kind)
    cases = _configs(kind, 4000, rng) + (_parallel_ee(rng) if kind == O.ORC_EE else [])
    per_type = {}
    for x in cases:
        d2, ty, gam = O.closest_weights(kind, x.reshape(-1))
        per_type.setdefault(ty, []).append((x, d2, gam))
    assert sorted(per_type) == list(range(ntypes)), sorted(per_type)
    for ty, lst in per_type.items():
        for x, d2, gam in lst[:25]:
            gap = gam @ x
            ref = _pt_min(x) if kind == O.ORC_PT else _ee_min(x)
            scale = np.abs(x).max()
            assert np.abs(gap - ref).max() <= 1e-6 * scale, (kind, ty, gap, ref)
            assert abs(gap @ gap - d2) <= 1e-12 * max(d2, 1e-300) + 1e-15, (kind, ty, gap @ gap, d2)
            # the weights: +1 spread over the first primitive, -1 over the second
            if kind == O.ORC_PT:
                assert gam[0] == 1.0 and abs(gam[1:].sum() + 1.0) <= 1e-12
                assert np.all(gam[1:] <= 1e-12)
            else:
                assert abs(gam[:2].sum() - 1.0) <= 1e-12 and abs(gam[2:].sum() + 1.0) <= 1e-12
                assert np.all(gam[:2] >= -1e-12) and np.all(gam[2:] <= 1e-12)


def test_closest_weights_vertex_types_exact():
    """point-point types put exactly one unit weight on each side"""
    rng = np.random.default_rng(3)
    seen = set()
    for x in _configs(O.ORC_EE, 4000, rng) + _configs(O.ORC_PT, 4000, rng):
        for kind in (O.ORC_PT, O.ORC_EE):
            d2, ty, gam = O.closest_weights(kind, x.reshape(-1))
            vertex = ty <= 2 if kind == O.ORC_PT else ty <= 3
            if vertex:
                seen.add((kind, ty))
                assert sorted(gam.tolist()) in ([-1.0, 0.0, 0.0, 1.0],), (kind, ty, gam)
    assert len(seen) == 7
