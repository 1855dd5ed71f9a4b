"""Pins of the oracle's implicit-function adjoint of the time step: the
closed form of free flight, and central finite differences of a multi-step
loss through contact (frictionless: the lagged friction quantities are held
fixed by the adjoint, so a finite difference of the step map with friction
would also see their dependence on q^t)."""
import numpy as np
import pytest

import oracle as O
from paper_2201_10022_gb300 import scenes


def rollout(o, q0, qd0, n):
    """forward with per-step checkpoints"""
    o.set_state(q0, qd0)
    states = [(q0.copy(), qd0.copy())]
    for _ in range(n):
        r, _ = o.step(1)
        assert r == 0, O.ERRORS[r]
        q, qd = o.get_state()
        states.append((q.copy(), qd.copy()))
    return states


def backward(o, s, states, gq, gqd):
    """chain of adjoint steps: dL/dq_{t+1} (total) -> M lam; dL/dq_t =
    M lam - gqd/dt, dL/dqdot_t = dt M lam (q~ = q + dt qdot + dt^2 g,
    qdot_{t+1} = (q_{t+1} - q_t)/dt)"""
    dt = s.params["dt"]
    gk = np.zeros(s.nb)
    for t in range(len(states) - 2, -1, -1):
        (qt, qdt), (qn, _) = states[t], states[t + 1]
        rhs = gq + gqd / dt
        st, Mlam, gkt = o.adjoint_step(qt, qdt, qn, rhs)
        assert st == 0, O.ERRORS[st]
        gq, gqd = Mlam - gqd / dt, dt * Mlam
        gk += gkt
    dyn = s.is_static == 0
    gq[~dyn] = 0.0
    gqd[~dyn] = 0.0
    return gq, gqd, gk


def _loss(states, s, target):
    qK = states[-1][0]
    dyn = s.is_static == 0
    return float(np.sum((qK[dyn, :3].mean(axis=0) - target) ** 2))


def _dloss(states, s, target):
    qK = states[-1][0]
    dyn = s.is_static == 0
    m = qK[dyn, :3].mean(axis=0)
    g = np.zeros_like(qK)
    g[dyn, :3] = 2.0 * (m - target) / dyn.sum()
    return g


def test_free_flight_closed_form():
    """no contact, A a rotation, centred bodies (M decouples p from A): the
    translation of every step is p~_t, so dp_K / dpdot_0 = K dt I, and a
    loss on translations back-propagates to K dt times itself with nothing
    in the A rows; grad V = 0 on rotations gives dL/dkappa = 0"""
    s = scenes.random_pair(5, kinds=("cube", "cube"), sep=0.5)
    o = O.Oracle(s, newton_rel=1e-13)
    n = 5
    states = rollout(o, s.q0.copy(), s.qdot0.copy(), n)
    rng = np.random.default_rng(0)
    gq = np.zeros_like(s.q0)
    gq[:, :3] = rng.normal(size=(s.nb, 3))
    gq[s.is_static == 1] = 0.0
    _, gqd0, gk = backward(o, s, states, gq, np.zeros_like(gq))
    dt = s.params["dt"]
    np.testing.assert_allclose(gqd0[:, :3], n * dt * gq[:, :3], rtol=1e-9, atol=1e-12)
    assert np.abs(gqd0[:, 3:]).max() < 1e-9
    assert np.abs(gk).max() < 1e-9


def test_adjoint_matches_central_differences_through_contact():
    # a cube in resting contact with a box, pushed sideways: the barrier is
    # active at every step
    B = scenes._Builder("adjoint", 0)
    gv, gt = scenes.box_mesh(2.0, 2.0, 0.4)
    B.add(gv, gt, p=(0.0, 0.0, -0.2), static=True)
    cv, ct = scenes.cube_mesh(0.2)
    B.add(cv, ct, R=scenes.small_rotation(np.random.default_rng(1), 2.0), p=(0.0, 0.0, 0.1 + 0.0012),
          v=(0.4, -0.2, 0.05), kappa=1e6)
    B.add(cv, ct, p=(0.35, 0.0, 0.1 + 0.0012), v=(-0.3, 0.1, 0.0), kappa=2e6)
    s = B.build(dict(mu=0.0))
    target = np.array([0.3, -0.1, 0.2])
    n = 4
    mk = lambda: O.Oracle(s, newton_rel=1e-14, newton_max=200)
    o = mk()
    states = rollout(o, s.q0.copy(), s.qdot0.copy(), n)
    assert o.pairs(1)["kind"].size > 0  # contact active at the last state
    _, gqd0, gk = backward(o, s, states, _dloss(states, s, target), np.zeros_like(s.q0))

    def loss_at(qd0=None, kappa=None):
        s2 = s
        if kappa is not None:
            s2 = scenes.Scene(**{**s.__dict__, "kappa_body": kappa})
        o2 = O.Oracle(s2, newton_rel=1e-14, newton_max=200)
        return _loss(rollout(o2, s.q0.copy(), qd0 if qd0 is not None else s.qdot0.copy(), n), s, target)

    h = 1e-6
    for b in (1, 2):
        for k in (0, 1, 2, 3, 7, 11):
            e = np.zeros_like(s.qdot0)
            e[b, k] = h
            fd = (loss_at(qd0=s.qdot0 + e) - loss_at(qd0=s.qdot0 - e)) / (2 * h)
            assert gqd0[b, k] == pytest.approx(fd, rel=2e-4, abs=1e-9 * np.abs(gqd0).max()), (b, k)
    for b in (1, 2):
        kp = s.kappa_body.copy()
        hk = 1e-5 * kp[b]
        kp[b] += hk
        km = s.kappa_body.copy()
        km[b] -= hk
        fd = (loss_at(kappa=kp) - loss_at(kappa=km)) / (2 * hk)
        assert gk[b] == pytest.approx(fd, rel=2e-3, abs=1e-6 * np.abs(gk).max()), b


def test_unprojected_hessian_is_positive_definite_at_the_step():
    """at a converged step the unprojected IP Hessian is positive definite
    here, so the adjoint's Cholesky solve applies"""
    s = scenes.cube_stack(seed=1, gap=0.0004)
    o = O.Oracle(s, newton_rel=1e-13)
    states = rollout(o, s.q0.copy(), s.qdot0.copy(), 2)
    o.set_state(*states[1])
    st, E, g = o.energy_grad_hess(states[2][0].reshape(-1), project=False)
    H = o.dense_hessian()
    assert np.linalg.eigvalsh(H).min() > 0


def _contact_scene():
    B = scenes._Builder("adjoint", 0)
    gv, gt = scenes.box_mesh(2.0, 2.0, 0.4)
    B.add(gv, gt, p=(0.0, 0.0, -0.2), static=True)
    cv, ct = scenes.cube_mesh(0.2)
    B.add(cv, ct, R=scenes.small_rotation(np.random.default_rng(1), 2.0), p=(0.0, 0.0, 0.1 + 0.0012),
          v=(0.4, -0.2, 0.05), kappa=1e6)
    B.add(cv, ct, p=(0.35, 0.0, 0.1 + 0.0012), v=(-0.3, 0.1, 0.0), kappa=2e6)
    return B.build(dict(mu=0.0))


def backward_projected(o, s, states, gq, gqd):
    """the same chain with the PSD-projected Hessian (the one Newton uses)
    in place of the true one: lam = H_proj^-1 rhs by numpy, M lam by the
    oracle's mass matrices"""
    dt = s.params["dt"]
    dyn = np.nonzero(s.is_static == 0)[0]
    idx = np.concatenate([np.arange(12 * b, 12 * b + 12) for b in dyn])
    for t in range(len(states) - 2, -1, -1):
        (qt, qdt), (qn, _) = states[t], states[t + 1]
        o.set_state(qt, qdt)
        st, _, _ = o.energy_grad_hess(qn.reshape(-1), project=True)
        assert st == 0
        H = o.dense_hessian()
        rhs = (gq + gqd / dt).reshape(-1)
        lam = np.zeros(12 * s.nb)
        lam[idx] = np.linalg.solve(H[np.ix_(idx, idx)], rhs[idx])
        Mlam = np.zeros_like(gq)
        for b in dyn:
            Mlam[b] = o.mass_matrix(b) @ lam[12 * b:12 * b + 12]
        gq, gqd = Mlam - gqd / dt, dt * Mlam
    gqd[s.is_static == 1] = 0.0
    return gq, gqd


def test_projected_hessian_adjoint_differs_from_the_implicit_function_one():
    """The implicit-function theorem needs the true Hessian of the IP at the
    converged step; the Newton loop uses its PSD projection.  Through an
    active contact the two chains give different gradients: the unprojected
    one matches central differences of the loss, the projected one is off
    by more (its mismatch is the difference the adjoint would carry if it
    reused Newton's Hessian)."""
    s = _contact_scene()
    target = np.array([0.3, -0.1, 0.2])
    n = 4
    o = O.Oracle(s, newton_rel=1e-14, newton_max=200)
    states = rollout(o, s.q0.copy(), s.qdot0.copy(), n)
    g0 = _dloss(states, s, target)
    _, gqd_true, _ = backward(o, s, states, g0, np.zeros_like(s.q0))
    _, gqd_proj = backward_projected(o, s, states, g0, np.zeros_like(s.q0))

    def loss_at(qd0):
        o2 = O.Oracle(s, newton_rel=1e-14, newton_max=200)
        return _loss(rollout(o2, s.q0.copy(), qd0, n), s, target)

    h = 1e-6
    err_true, err_proj = [], []
    for b, k in ((1, 0), (1, 2), (2, 0), (2, 1)):
        e = np.zeros_like(s.qdot0)
        e[b, k] = h
        fd = (loss_at(s.qdot0 + e) - loss_at(s.qdot0 - e)) / (2 * h)
        scale = max(abs(fd), 1e-9 * np.abs(gqd_true).max())
        err_true.append(abs(gqd_true[b, k] - fd) / scale)
        err_proj.append(abs(gqd_proj[b, k] - fd) / scale)
    rel_diff = np.abs(gqd_true - gqd_proj).max() / np.abs(gqd_true).max()
    print(f"adjoint through contact: unprojected vs central differences {max(err_true):.2e}, "
          f"projected {max(err_proj):.2e}; projected vs unprojected gradient {rel_diff:.2e}")
    assert max(err_true) <= 2e-4
    assert rel_diff > 10 * max(err_true)
    assert max(err_proj) > max(err_true)


def test_ldl_solve_matches_library_solve_on_indefinite_systems():
    """the adjoint's dense factorisation A = L D L^T (no pivoting) against
    numpy's LU solve: symmetric matrices with eigenvalues of both signs
    (where Cholesky does not exist), an SPD matrix, and a zero leading
    pivot reported as a failure"""
    rng = np.random.default_rng(11)
    for n, neg in ((12, 1), (48, 5), (97, 30)):
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
        lam = rng.uniform(0.5, 4.0, n)
        lam[:neg] *= -1.0
        A = (Q * lam) @ Q.T
        A = 0.5 * (A + A.T)
        with pytest.raises(np.linalg.LinAlgError):
            np.linalg.cholesky(A)
        b = rng.standard_normal(n)
        r, x = O.ldl_solve(A, b)
        assert r == 0
        ref = np.linalg.solve(A, b)
        assert np.abs(x - ref).max() <= 1e-10 * np.abs(ref).max()
        assert np.abs(A @ x - b).max() <= 1e-12 * np.abs(A).max() * np.abs(x).max() * n
    B = rng.standard_normal((30, 30))
    A = B @ B.T + 30 * np.eye(30)
    b = rng.standard_normal(30)
    r, x = O.ldl_solve(A, b)
    assert r == 0 and np.allclose(x, np.linalg.solve(A, b), rtol=1e-12, atol=0)
    r, _ = O.ldl_solve(np.array([[0.0, 1.0], [1.0, 0.0]]), np.ones(2))
    assert r == -1


def test_adjoint_at_an_indefinite_converged_state():
    """the throw-into-stack workload at its first contact step: Newton's
    stationary point is not a minimiser of the IP there (the unprojected
    Hessian has a negative eigenvalue), yet nonsingular, so the implicit
    function theorem applies; the oracle's adjoint solves with that exact
    Hessian (M lam with lam = H^-1 rhs by numpy's LU on the oracle's own
    unprojected matrix)"""
    s = scenes.throw_stack(seed=4)
    o = O.Oracle(s, newton_max=300)
    states = rollout(o, s.q0.copy(), s.qdot0.copy(), 3)
    (qt, qdt), (qn, _) = states[2], states[3]
    o.set_state(qt, qdt)
    st, _, _ = o.energy_grad_hess(qn.reshape(-1), project=False)
    assert st == 0
    dyn = np.nonzero(s.is_static == 0)[0]
    idx = np.concatenate([np.arange(12 * b, 12 * b + 12) for b in dyn])
    H = o.dense_hessian()[np.ix_(idx, idx)]
    ev = np.linalg.eigvalsh(H)
    assert ev.min() < 0.0 < ev.max()
    assert np.abs(ev).min() > 1e-12 * ev.max()
    rhs = np.zeros_like(s.q0)
    rhs[dyn, :3] = np.random.default_rng(2).standard_normal((dyn.size, 3))
    st, Mlam, _ = o.adjoint_step(qt, qdt, qn, rhs)
    assert st == 0, O.ERRORS[st]
    lam = np.zeros(12 * s.nb)
    lam[idx] = np.linalg.solve(H, rhs.reshape(-1)[idx])
    ref = np.zeros_like(s.q0)
    for b in dyn:
        ref[b] = o.mass_matrix(b) @ lam[12 * b:12 * b + 12]
    # cond(H) = 5e5 / 0.027 ~ 2e7: eps * cond ~ 4e-9 bounds the difference of
    # two backward-stable solves
    assert np.abs(Mlam - ref).max() <= 1e-8 * np.abs(ref).max()


def test_throw_stack_adjoint_golden_is_the_oracles():
    """the stored 20-step throw-into-stack adjoint (the GPU test's expected
    values) is the oracle's: the chain's inputs are the next step's outputs,
    exactly one step's unprojected Hessian is indefinite (the first contact,
    numpy's eigenvalues of the oracle's matrix), and the last step's adjoint
    recomputed now from the stored states equals the stored one"""
    import os
    G = np.load(os.path.join(os.path.dirname(__file__), "golden", "throw_stack_adjoint.npz"))
    n = G["q"].shape[0] - 1
    for t in range(n - 1):
        assert np.array_equal(G["gq_in"][t], G["gq_out"][t + 1])
        assert np.array_equal(G["gqd_in"][t], G["gqd_out"][t + 1])
    assert (G["hess_eig"][:, 0] < 0).sum() == 1
    s = scenes.throw_stack(seed=int(G["seed"]))
    o = O.Oracle(s, newton_max=300)
    dt = s.params["dt"]
    t = n - 1
    gq, gqd = G["gq_in"][t], G["gqd_in"][t]
    st, Mlam, gk = o.adjoint_step(G["q"][t], G["qdot"][t], G["q"][t + 1], gq + gqd / dt)
    assert st == 0, O.ERRORS[st]
    dyn = s.is_static == 0
    out = Mlam - gqd / dt
    out[~dyn] = 0.0
    scale = np.abs(G["gq_out"][t]).max()
    assert np.abs(out - G["gq_out"][t]).max() <= 1e-12 * scale
    assert np.abs(gk - G["gk_out"][t]).max() <= 1e-12 * max(np.abs(G["gk_out"][t]).max(), 1e-300)
