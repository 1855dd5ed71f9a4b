"""Pins of the oracle's assembled IP and its time step (Sec. 4): finite
differences of the assembled energy and gradient, direct against iterative
solve, momentum conservation, non-intersection, contact accuracy, the kappa
trend of the orthogonality residual and Coulomb deceleration under friction."""
import numpy as np
import pytest

import oracle as O
from paper_2201_10022_gb300 import scenes


def _touching_scene(seed=0, mu=0.0):
    s = scenes.random_pair(seed, kinds=("cube", "ico1"), sep=0.0004, mu=mu)
    rng = np.random.default_rng(seed)
    s.qdot0[:, :3] = rng.normal(size=(2, 3)) * 0.05
    return s


def test_assembled_gradient_and_hessian_finite_differences():
    s = _touching_scene(3)
    o = O.Oracle(s)
    q = s.q0.reshape(-1).copy()
    st, E, g = o.energy_grad_hess(q, project=False)
    assert st == 0 and E[3] > 0  # contact active
    H = o.dense_hessian()
    h = 1e-8
    gfd = np.zeros_like(q)
    Hfd = np.zeros((len(q), len(q)))
    for i in range(len(q)):
        e = np.zeros_like(q)
        e[i] = h
        gfd[i] = (o.energy(q + e) - o.energy(q - e)) / (2 * h)
        _, _, gp = o.energy_grad_hess(q + e, project=False)
        _, _, gm = o.energy_grad_hess(q - e, project=False)
        Hfd[i] = (gp.ravel() - gm.ravel()) / (2 * h)
    g = g.ravel()
    scale = np.abs(g).max()
    np.testing.assert_allclose(g, gfd, rtol=1e-5, atol=1e-5 * scale)
    np.testing.assert_allclose(H, Hfd, rtol=1e-4, atol=1e-5 * np.abs(H).max())


def test_projected_system_is_psd_and_solves_agree():
    s = scenes.cube_stack(seed=1, gap=0.0005)
    o = O.Oracle(s)
    q = s.q0.reshape(-1)
    st, E, g = o.energy_grad_hess(q)
    assert st == 0 and E[3] > 0
    H = o.dense_hessian()
    w = np.linalg.eigvalsh(H)
    assert w.min() > 0
    st, dq_dense, _ = o.solve(-g.ravel())
    assert st == 0
    o2 = O.Oracle(s, dense_max_dof=0, cg_tol=1e-14)
    o2.energy_grad_hess(q)
    st, dq_cg, it = o2.solve(-g.ravel())
    assert st == 0 and it > 0
    np.testing.assert_allclose(dq_cg, dq_dense, rtol=1e-8, atol=1e-10 * np.abs(dq_dense).max())
    np.testing.assert_allclose(H @ dq_dense.ravel(), -g.ravel(), atol=1e-9 * np.abs(g).max())


def _min_distance(o, s, q):
    x = o.vertices(q)
    pairs = o.candidates(x, brute=True)
    dmin = np.inf
    for kind, i, j in pairs:
        v = [i, *s.tri[j]] if kind == 0 else [*s.edge[i], *s.edge[j]]
        dmin = min(dmin, np.sqrt(O.pair_dist2(kind, x[v].ravel())[0]))
    return dmin


def test_momentum_conserved_in_collision_without_gravity():
    s = scenes.random_pair(5, kinds=("cube", "ico1"), sep=0.01, gravity=(0.0, 0.0, 0.0))
    p0, p1 = s.q0[0, :3], s.q0[1, :3]
    n = (p1 - p0) / np.linalg.norm(p1 - p0)
    s.qdot0[0, :3] = 0.8 * n
    s.qdot0[1, :3] = -0.3 * n
    o = O.Oracle(s)
    masses = np.array([o.mass_matrix(b)[0, 0] for b in range(2)])
    P0 = (masses[:, None] * s.qdot0[:, :3]).sum(axis=0)
    contact = False
    for k in range(8):
        r, st = o.step(1)
        assert r == 0
        contact |= st["n_active"] > 0
        q, qd = o.get_state()
        P = (masses[:, None] * qd[:, :3]).sum(axis=0)
        # Newton tolerance bound: |dp| <= tol, so |dP| <~ m * tol / dt
        np.testing.assert_allclose(P, P0, atol=masses.sum() * o.newton_tol / s.params["dt"] * 10)
        assert _min_distance(o, s, q.ravel()) > 0
    assert contact


def test_cube_stack_no_intersection_and_contact_accuracy():
    s = scenes.cube_stack(seed=1)
    o = O.Oracle(s)
    dhat = s.params["dhat"]
    for k in range(40):
        r, st = o.step(1)
        assert r == 0, O.ERRORS[r]
        q, _ = o.get_state()
        if k % 8 == 7:
            assert _min_distance(o, s, q.ravel()) > 0
    st, E, g = o.energy_grad_hess(q.ravel())
    act = o.pairs(1)
    assert len(act["kind"]) > 0
    d = np.sqrt(act["val"])
    assert (d > 0).all() and (d < dhat).all()


def test_orthogonality_residual_shrinks_with_kappa():
    """The largest |A A^T - I|_F seen over the first steps of the cube stack
    (impacts included) falls as the orthogonality stiffness grows."""
    res = []
    for kap in (1e6, 1e7, 1e8, 1e9):
        s = scenes.cube_stack(seed=1)
        s.kappa_body[:] = kap
        o = O.Oracle(s)
        peak = 0.0
        for _ in range(16):
            r, st = o.step(1)
            assert r == 0
            q, _ = o.get_state()
            A = q[1:, 3:].reshape(-1, 3, 3)
            peak = max(peak, max(np.linalg.norm(a @ a.T - np.eye(3)) for a in A))
        res.append(peak)
    assert all(res[i + 1] < res[i] for i in range(len(res) - 1)), res


def test_friction_decelerates_sliding_cube_by_mu_g():
    """A cube sliding on the ground loses speed at about mu*g (Coulomb) while
    it slides; the lagged, mollified friction potential reproduces it."""
    mu = 0.3
    B = scenes._Builder("slide", 0)
    gv, gt = scenes.box_mesh(10.0, 10.0, 1.0)
    B.add(gv, gt, p=(0.0, 0.0, -0.5), static=True)
    cv, ct = scenes.cube_mesh(0.2)
    B.add(cv, ct, p=(0.0, 0.0, 0.1 + 0.0015), v=(2.0, 0.0, 0.0))
    s = B.build(dict(mu=mu))
    o = O.Oracle(s)
    vx = []
    for k in range(30):
        r, st = o.step(1)
        assert r == 0
        q, qd = o.get_state()
        vx.append(qd[1, 0])
    vx = np.array(vx)
    dt, g = s.params["dt"], 9.8
    # once the cube rests on the ground (a couple of steps), dv/dt = -mu g
    acc = np.diff(vx[3:]) / dt
    np.testing.assert_allclose(acc, -mu * g, rtol=5e-3)
    # the lagged normal forces carry the weight: sum mu lambda = mu m g dt^2
    mass = o.mass_matrix(1)[0, 0]
    assert o.pairs(2)["val"].sum() == pytest.approx(mu * mass * g * dt * dt, rel=5e-3)


def test_sampled_entry_points_agree_with_full_evaluation():
    """active set by distance alone, the value-only energy and gradient rows
    of selected bodies equal the full evaluation's"""
    s = scenes.packed_cubes(nx=3, ny=2, nz=2)
    o = O.Oracle(s)
    q = s.q0.reshape(-1)
    st, E, g = o.energy_grad_hess(q, project=False)
    act_full = o.pairs(1)
    act = o.active_pairs(q)
    key = lambda d: set(zip(d["kind"].tolist(), d["i"].tolist(), d["j"].tolist(), d["type"].tolist(),
                            d["val"].tolist()))
    assert len(act["kind"]) > 50 and key(act) == key(act_full)
    assert o.energy(q) == pytest.approx(E[0], rel=1e-12)
    sel = np.array([1, 4, 7, 11])
    st, rows = o.grad_rows(q, sel)
    assert st == 0
    np.testing.assert_allclose(rows, g[sel], rtol=1e-12, atol=1e-12 * np.abs(g).max())


def test_scene_barrier_uses_rest_length_mollifier():
    """In a scene the edge-edge terms carry the mollifier with eps_x from the
    edges' rest lengths: the barrier energy of a packed pair of cubes (tiny
    rotations, so every edge-edge pair is near-parallel) equals the sum of the
    per-pair terms with eps_x = 1e-3 |rest e_i|^2 |rest e_j|^2 computed here,
    and stays so after the bodies are scaled (eps_x is not recomputed)."""
    s = scenes.packed_cubes(nx=2, ny=1, nz=1)
    o = O.Oracle(s)
    q = s.q0.reshape(-1).copy()
    rest_l2 = {}
    for e, (a, b) in enumerate(s.edge):
        d = s.xbar[b] - s.xbar[a]
        rest_l2[e] = d @ d
    for scale in (1.0, 1.0 + 2e-4):
        qs = q.copy()
        for b in range(s.nb):
            if not s.is_static[b]:
                qs[12 * b + 3:12 * b + 12] *= scale  # A -> scale * A (about each body's origin)
        st, E, g = o.energy_grad_hess(qs)
        assert st == 0 and E[3] > 0
        P = o.pairs(1)
        x = o.vertices(qs).reshape(-1, 3)
        total, n_moll = 0.0, 0
        for kind, i, j in zip(P["kind"], P["i"], P["j"]):
            if kind == 0:
                v = [i, *s.tri[j]]
                eps = 0.0
            else:
                v = [*s.edge[i], *s.edge[j]]
                eps = 1e-3 * rest_l2[i] * rest_l2[j]
                n_moll += O.ee_cross2(x[v].ravel()) < eps
            total += O.pair_barrier(kind, x[v].ravel(), s.params["dhat"], s.params["kappa"], False, eps_x=eps)[1]
        assert n_moll > 0
        assert E[3] == pytest.approx(total, rel=1e-12)
