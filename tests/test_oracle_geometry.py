"""Pins of the oracle's distances, distance types, barrier and PSD projection
(Sec. 4, Eq. barrier, Eq. clamped-b) against closed forms, a library
minimiser (brute force over the primitives' parameters), finite differences
and numpy's symmetric eigensolver."""
import numpy as np
import pytest
from scipy.optimize import minimize

import oracle as O

DHAT = 1e-3


def _pt_brute(p, a, b, c):
    best = np.inf
    f = lambda uv: np.sum((p - (a + uv[0] * (b - a) + uv[1] * (c - a))) ** 2)
    cons = [{"type": "ineq", "fun": lambda uv: uv[0]}, {"type": "ineq", "fun": lambda uv: uv[1]},
            {"type": "ineq", "fun": lambda uv: 1 - uv[0] - uv[1]}]
    for st in ([1 / 3, 1 / 3], [0.05, 0.05], [0.9, 0.05], [0.05, 0.9]):
        r = minimize(f, st, constraints=cons, method="SLSQP", options=dict(ftol=1e-16, maxiter=500))
        uv = np.clip(r.x, 0, 1)
        if uv.sum() > 1:
            uv = uv / uv.sum()
        best = min(best, f(uv))
    # the three edges, exactly
    for s, e in ((a, b), (b, c), (c, a)):
        t = np.clip((p - s) @ (e - s) / ((e - s) @ (e - s)), 0, 1)
        best = min(best, np.sum((p - s - t * (e - s)) ** 2))
    return best


def _ee_brute(a, b, c, d):
    f = lambda st: np.sum((a + st[0] * (b - a) - c - st[1] * (d - c)) ** 2)
    best = np.inf
    for s0 in ([0.5, 0.5], [0.1, 0.9], [0.9, 0.1]):
        r = minimize(f, s0, bounds=[(0, 1), (0, 1)], method="L-BFGS-B", options=dict(ftol=1e-18, gtol=1e-14))
        best = min(best, f(r.x))
    for p, s, e in ((a, c, d), (b, c, d), (c, a, b), (d, a, b)):
        t = np.clip((p - s) @ (e - s) / ((e - s) @ (e - s)), 0, 1)
        best = min(best, np.sum((p - s - t * (e - s)) ** 2))
    return best


def test_closed_forms():
    a, b, c = np.array([0.0, 0, 0]), np.array([1.0, 0, 0]), np.array([0.0, 1, 0])
    d2, ty = O.pt_dist2(np.array([0.2, 0.2, 0.3]), a, b, c)
    assert ty == 6 and d2 == pytest.approx(0.09, rel=1e-15)
    d2, ty = O.pt_dist2(np.array([-1.0, -2.0, 2.0]), a, b, c)
    assert ty == 0 and d2 == pytest.approx(9.0, rel=1e-15)
    d2, ty = O.pt_dist2(np.array([0.5, -1.0, 1.0]), a, b, c)
    assert ty == 3 and d2 == pytest.approx(2.0, rel=1e-15)
    # two skew lines at distance 0.5 with interior closest points
    d2, ty = O.ee_dist2(np.array([-1.0, 0, 0]), np.array([1.0, 0, 0]), np.array([0.0, -1, 0.5]),
                        np.array([0.0, 1, 0.5]))
    assert ty == 8 and d2 == pytest.approx(0.25, rel=1e-15)
    # parallel edges fall back to point-edge / point-point
    d2, ty = O.ee_dist2(np.array([0.0, 0, 0]), np.array([1.0, 0, 0]), np.array([0.5, 0, 0.1]),
                        np.array([1.5, 0, 0.1]))
    assert ty in (4, 5, 6, 7) and d2 == pytest.approx(0.01, rel=1e-14)


def test_distances_match_brute_force_minimiser():
    rng = np.random.default_rng(11)
    for _ in range(150):
        p, a, b, c = rng.normal(size=(4, 3))
        d2, ty = O.pt_dist2(p, a, b, c)
        assert d2 == pytest.approx(_pt_brute(p, a, b, c), rel=1e-7, abs=1e-12)
        x0, x1, x2, x3 = rng.normal(size=(4, 3))
        d2, ty = O.ee_dist2(x0, x1, x2, x3)
        assert d2 == pytest.approx(_ee_brute(x0, x1, x2, x3), rel=1e-7, abs=1e-12)


def test_barrier_vanishes_smoothly_at_dhat():
    """B(dhat) = B'(dhat) = B''(dhat) = 0: a point-point pair just inside dhat
    carries vanishing energy, gradient and Hessian (kappa = 1)."""
    assert O.barrier(DHAT, DHAT) == 0.0
    assert O.barrier(2 * DHAT, DHAT) == 0.0
    assert O.barrier(0.5 * DHAT, DHAT) > 0
    tri = np.array([0, 0, 0, 1, 0, 0, 0, 1, 0.0])
    prev = None
    for frac in (0.99, 0.999, 0.9999):
        d = frac * DHAT
        p = -d / np.sqrt(3.0) * np.ones(3)
        act, E, g, H = O.pair_barrier(0, np.concatenate([p, tri]), DHAT, 1.0, False)
        assert act and O.pair_dist2(0, np.concatenate([p, tri]))[1] == 0
        cur = (E, np.abs(g).max(), np.abs(H).max())
        if prev is not None:
            # E ~ delta^3, |g| ~ delta^2, |H| ~ delta with delta = dhat - d
            assert cur[0] < prev[0] * 2e-3 and cur[1] < prev[1] * 2e-2 and cur[2] < prev[2] * 0.2
        prev = cur
    assert prev[0] < 2e-18 and prev[1] < 1e-9 and prev[2] < 1e-2


def _fd(f, x, h):
    out = []
    for i in range(len(x)):
        e = np.zeros_like(x)
        e[i] = h
        out.append((f(x + e) - f(x - e)) / (2 * h))
    return np.array(out)


def _closest_points(kind, ty, x):
    """closest points (on the first, on the second primitive) for a known type"""
    v = x.reshape(4, 3)

    def on_seg(p, a, b):
        t = (p - a) @ (b - a) / ((b - a) @ (b - a))
        return a + t * (b - a)

    if kind == 0:
        p, a, b, c = v
        if ty < 3:
            return p, v[1 + ty]
        if ty < 6:
            s, e = [(a, b), (b, c), (c, a)][ty - 3]
            return p, on_seg(p, s, e)
        n = np.cross(b - a, c - a)
        n /= np.linalg.norm(n)
        return p, p - ((p - a) @ n) * n
    a, b, c, d = v
    if ty < 4:
        return [(a, c), (a, d), (b, c), (b, d)][ty]
    if ty == 4:
        return a, on_seg(a, c, d)
    if ty == 5:
        return b, on_seg(b, c, d)
    if ty == 6:
        return on_seg(c, a, b), c
    if ty == 7:
        return on_seg(d, a, b), d
    e0, e1, w0 = b - a, d - c, a - c
    A, B, C, D, E = e0 @ e0, e0 @ e1, e1 @ e1, e0 @ w0, e1 @ w0
    den = A * C - B * B
    return a + (B * E - C * D) / den * e0, c + (A * E - B * D) / den * e1


def _near_pair(rng, kind, want_type):
    """random pair configuration of the requested distance type at d in
    (0.2, 0.9) dhat: a random configuration of that type is moved rigidly
    along the line joining its closest points, which keeps the closest
    features"""
    for _ in range(20000):
        x = rng.normal(size=12) * 0.05
        d2, ty = O.pair_dist2(kind, x)
        if ty != want_type or d2 == 0:
            continue
        c0, c1 = _closest_points(kind, ty, x)
        D = np.linalg.norm(c1 - c0)
        d = rng.uniform(0.3, 0.8) * DHAT
        x2 = x.copy().reshape(4, 3)
        mv = (c1 - c0) * (1.0 - d / D)
        if kind == 0:
            x2[0] += mv
        else:
            x2[:2] += mv
        x2 = x2.ravel()
        d2b, ty2 = O.pair_dist2(kind, x2)
        if ty2 == want_type and (0.2 * DHAT) ** 2 < d2b < (0.9 * DHAT) ** 2:
            return x2
    raise AssertionError(f"no configuration of type {want_type}")


@pytest.mark.parametrize("kind,types", [(0, range(7)), (1, range(9))])
def test_barrier_derivatives_finite_differences_every_type(kind, types):
    rng = np.random.default_rng(100 + kind)
    for ty in types:
        x = _near_pair(rng, kind, ty)
        act, E, g, H = O.pair_barrier(kind, x, DHAT, 1.0, False)
        assert act
        h = 1e-9
        # finite differences only within the same type
        f = lambda y: O.pair_barrier(kind, y, DHAT, 1.0, False)[1]
        gfd = _fd(f, x, h)
        np.testing.assert_allclose(g, gfd, rtol=1e-4, atol=1e-6 * np.abs(g).max())
        gf = lambda y, i=0: O.pair_barrier(kind, y, DHAT, 1.0, False)[2]
        Hfd = np.array([(gf(x + h * np.eye(12)[i]) - gf(x - h * np.eye(12)[i])) / (2 * h) for i in range(12)])
        np.testing.assert_allclose(H, Hfd, rtol=1e-4, atol=1e-5 * np.abs(H).max())


def test_projection_against_numpy_eigh():
    rng = np.random.default_rng(7)
    for n in (3, 9, 12):
        for _ in range(10):
            A = rng.normal(size=(n, n))
            A = A + A.T
            P = O.project_psd(A)
            w, V = np.linalg.eigh(A)
            ref = (V * np.maximum(w, 0)) @ V.T
            np.testing.assert_allclose(P, ref, atol=1e-12 * np.abs(A).max())
            w2, _ = O.sym_eig(A)
            np.testing.assert_allclose(np.sort(w2), w, atol=1e-12 * np.abs(A).max())
    B = rng.normal(size=(12, 12))
    S = B @ B.T
    np.testing.assert_allclose(O.project_psd(S), S, atol=1e-12 * np.abs(S).max())


def test_projected_barrier_hessian_is_psd():
    rng = np.random.default_rng(8)
    for kind, types in ((0, range(7)), (1, range(9))):
        for ty in types:
            x = _near_pair(rng, kind, ty)
            act, E, g, H = O.pair_barrier(kind, x, DHAT, 1e8, True)
            w = np.linalg.eigvalsh(H)
            assert w.min() >= -1e-12 * np.abs(w).max()


# --- near-parallel edge-edge mollifier ---------------------------------------

def _ee_family(theta, mode, d=0.5 * DHAT, L0=1.0, L1=0.8):
    """edge 0 along x at z=0, edge 1 at height d turned by theta about z.
    mode "line": edge 1 crosses edge 0 at mid-span (line-line type);
    "pe": edge 1 starts above the middle of edge 0, off to one side, so that
    the lines' crossing lies behind it (its end against edge 0);
    "pp": the same just past the end of edge 0 (end against end).  Each
    configuration sits strictly inside its distance type's region."""
    c, s = np.cos(theta), np.sin(theta)
    x0, x1 = np.array([0.0, 0.0, 0.0]), np.array([L0, 0.0, 0.0])
    u = L1 * np.array([c, s, 0.0])
    if mode == "line":
        x2 = np.array([0.5 * L0, 0.0, d]) - 0.5 * u
    elif mode == "pe":
        x2 = np.array([0.5 * L0, 0.3 * DHAT, d])
    else:
        x2 = np.array([L0 + 0.3 * DHAT, 0.3 * DHAT, d])
    return np.concatenate([x0, x1, x2, x2 + u])


def test_mollifier_polynomial_joins():
    """m is 0 with slope 2/eps at c = 0 and joins 1 with zero slope at eps (C1)"""
    for eps in (1e-3, 0.37, 5.0):
        m0, dm0, _ = O.ee_mollifier(0.0, eps)
        assert m0 == 0.0 and dm0 == pytest.approx(2.0 / eps, rel=1e-15)
        m1, dm1, _ = O.ee_mollifier(eps * (1 - 1e-12), eps)
        assert m1 == pytest.approx(1.0, abs=1e-11) and abs(dm1) < 1e-10 / eps
        assert O.ee_mollifier(eps, eps)[:2] == (1.0, 0.0)
        # monotone increasing on [0, eps): a fade-in, never above 1
        cs = np.linspace(0, eps, 50, endpoint=False)
        ms = [O.ee_mollifier(c, eps)[0] for c in cs]
        assert np.all(np.diff(ms) > 0) and max(ms) < 1.0
        # second derivative by differences of the first
        c = 0.3 * eps
        h = 1e-6 * eps
        fd = (O.ee_mollifier(c + h, eps)[1] - O.ee_mollifier(c - h, eps)[1]) / (2 * h)
        assert fd == pytest.approx(O.ee_mollifier(c, eps)[2], rel=1e-7)


def test_ee_cross2_against_numpy():
    rng = np.random.default_rng(31)
    for _ in range(20):
        x = rng.normal(size=12)
        n = np.cross(x[3:6] - x[0:3], x[9:12] - x[6:9])
        assert O.ee_cross2(x) == pytest.approx(n @ n, rel=1e-13)


def test_parallel_edges_carry_no_barrier():
    """exactly parallel edges within d-hat: c = 0, so energy and gradient vanish
    (the contact is left to the point-triangle pairs)"""
    eps = 1e-3 * 1.0 * 0.64
    for mode in ("line", "pe", "pp"):  # parallel: the type is a tie-break
        x = _ee_family(0.0, mode)
        d2, ty = O.pair_dist2(1, x)
        assert d2 < DHAT ** 2
        act, E, g, H = O.pair_barrier(1, x, DHAT, 1e8, False, eps_x=eps)
        assert act and E == 0.0 and np.all(g == 0.0)
        assert np.linalg.eigvalsh(H).min() >= -1e-9 * np.abs(H).max()
        act0, E0, _, _ = O.pair_barrier(1, x, DHAT, 1e8, False)
        assert E0 > 0.0


@pytest.mark.parametrize("mode,want", [("line", 8), ("pe", 6), ("pp", 2)])
def test_mollified_barrier_finite_differences(mode, want):
    eps = 1e-3 * 1.0 * 0.64
    for theta in (2e-4, 1e-3, 2.5e-2):
        x = _ee_family(theta, mode)
        c = O.ee_cross2(x)
        assert c < eps and O.pair_dist2(1, x)[1] == want
        act, E, g, H = O.pair_barrier(1, x, DHAT, 1.0, False, eps_x=eps)
        act0, E0, g0, _ = O.pair_barrier(1, x, DHAT, 1.0, False)
        assert act and E == pytest.approx(E0 * O.ee_mollifier(c, eps)[0], rel=1e-12)
        h = 1e-9
        f = lambda y: O.pair_barrier(1, y, DHAT, 1.0, False, eps_x=eps)[1]
        np.testing.assert_allclose(g, _fd(f, x, h), rtol=1e-4, atol=1e-5 * np.abs(g).max())
        gf = lambda y: O.pair_barrier(1, y, DHAT, 1.0, False, eps_x=eps)[2]
        Hfd = np.array([(gf(x + h * np.eye(12)[i]) - gf(x - h * np.eye(12)[i])) / (2 * h) for i in range(12)])
        np.testing.assert_allclose(H, Hfd, rtol=1e-4, atol=1e-5 * np.abs(H).max())
        # the product-rule terms matter: the mollified gradient is not m * g0
        assert np.abs(g - O.ee_mollifier(c, eps)[0] * g0).max() > 1e-6 * np.abs(g).max()


def test_mollified_barrier_is_c1_across_threshold():
    """energy and its derivative along the rotation are continuous where
    |e0 x e1|^2 crosses eps_x, and nothing changes above it"""
    eps = 1e-3 * 1.0 * 0.64
    theta_c = np.arcsin(np.sqrt(eps / 0.64))  # |e0 x e1|^2 = 0.64 sin^2 theta
    def E_and_slope(theta):
        x = _ee_family(theta, "line")
        dx = (_ee_family(theta + 1e-7, "line") - _ee_family(theta - 1e-7, "line")) / 2e-7
        _, E, g, _ = O.pair_barrier(1, x, DHAT, 1.0, False, eps_x=eps)
        return E, g @ dx
    jumps = []
    for delta in (1e-4, 1e-5, 1e-6):
        Em, sm = E_and_slope(theta_c - delta)
        Ep, sp = E_and_slope(theta_c + delta)
        jumps.append((abs(Ep - Em), abs(sp - sm)))
    # a jump in the value or the slope would not shrink with delta; for a C1
    # join both go to zero (the slope linearly, the value quadratically)
    for (e1, s1), (e2, s2) in zip(jumps, jumps[1:]):
        assert s2 <= 0.15 * s1 and e2 <= 0.02 * e1 + 1e-22
    x = _ee_family(2 * theta_c, "line")
    a = O.pair_barrier(1, x, DHAT, 1.0, True, eps_x=eps)
    b = O.pair_barrier(1, x, DHAT, 1.0, True)
    assert a[1] == b[1] and np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])
