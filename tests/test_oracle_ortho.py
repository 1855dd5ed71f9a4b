"""Pins of the oracle's orthogonality potential (Sec. 3.2, Eq. orthogonality,
Eq. ortho-energy, Eq. ortho-poly) and of the per-body IP term (Sec. 4)."""
import numpy as np
import pytest

import oracle as O
from paper_2201_10022_gb300 import scenes


def _q(A, p=(0.0, 0.0, 0.0)):
    return np.concatenate([np.asarray(p, float), np.asarray(A, float).reshape(-1)])


def test_zero_on_rotations():
    rng = np.random.default_rng(1)
    for _ in range(5):
        R = scenes.random_rotation(rng)
        V, g, H = O.ortho(_q(R, rng.normal(size=3)), 1e8, 0.3)
        assert abs(V) < 1e-20
        assert np.abs(g).max() < 1e-6  # kappa*nu*|grad| ~ 1e8 * eps
        assert np.abs(g).max() / (1e8 * 0.3) < 1e-14


def test_energy_is_frobenius_definition():
    rng = np.random.default_rng(2)
    A = rng.normal(size=(3, 3))
    V, _, _ = O.ortho(_q(A), 2.0, 0.5)
    assert V == pytest.approx(2.0 * 0.5 * np.linalg.norm(A @ A.T - np.eye(3)) ** 2, rel=1e-13)


def _fd(f, x, h):
    g = np.zeros_like(x)
    for i in range(len(x)):
        e = np.zeros_like(x)
        e[i] = h
        g[i] = (f(x + e) - f(x - e)) / (2 * h)
    return g


def test_gradient_and_hessian_finite_differences():
    rng = np.random.default_rng(3)
    for _ in range(3):
        q = _q(scenes.random_rotation(rng) + 0.05 * rng.normal(size=(3, 3)), rng.normal(size=3))
        V, g, H = O.ortho(q, 1.0, 1.0)
        gfd = _fd(lambda x: O.ortho(x, 1.0, 1.0)[0], q, 1e-6)
        np.testing.assert_allclose(g, gfd, rtol=1e-6, atol=1e-9)
        Hfd = np.stack([_fd(lambda x, i=i: O.ortho(x, 1.0, 1.0)[1][i], q, 1e-6) for i in range(12)])
        np.testing.assert_allclose(H, Hfd, rtol=1e-6, atol=1e-8)
        np.testing.assert_allclose(H, H.T, atol=1e-14)


def test_paper_gradient_and_diagonal_block_forms():
    """Eq. ortho-poly read with the sums over j != i:
    dV/da_i = 2 kappa nu (2(a_i.a_i - 1) a_i + 2 sum_{j!=i} (a_j a_j^T) a_i),
    d2V/da_i^2 = 2 kappa nu (4 a_i a_i^T + 2(|a_i|^2 - 1) I + 2 sum_{j!=i} a_j a_j^T);
    the off-diagonal blocks the paper omits are 4 kappa nu (a_j a_i^T + (a_i.a_j) I)."""
    rng = np.random.default_rng(4)
    A = rng.normal(size=(3, 3))
    k, nu = 3.0, 0.7
    V, g, H = O.ortho(_q(A), k, nu)
    for i in range(3):
        ai = A[i]
        s = sum(np.outer(A[j], A[j]) for j in range(3) if j != i)
        gi = 2 * k * nu * (2 * (ai @ ai - 1) * ai + 2 * s @ ai)
        np.testing.assert_allclose(g[3 + 3 * i:6 + 3 * i], gi, rtol=1e-12)
        Hii = 2 * k * nu * (4 * np.outer(ai, ai) + 2 * (ai @ ai - 1) * np.eye(3) + 2 * s)
        np.testing.assert_allclose(H[3 + 3 * i:6 + 3 * i, 3 + 3 * i:6 + 3 * i], Hii, rtol=1e-12, atol=1e-12)
        for j in range(3):
            if j == i:
                continue
            Hij = 4 * k * nu * (np.outer(A[j], ai) + (ai @ A[j]) * np.eye(3))
            np.testing.assert_allclose(H[3 + 3 * i:6 + 3 * i, 3 + 3 * j:6 + 3 * j], Hij, rtol=1e-12, atol=1e-12)
    assert np.abs(g[:3]).max() == 0 and np.abs(H[:3]).max() == 0


def test_hessian_at_identity_has_six_zero_modes():
    """At A = I the 9x9 block is PSD with exactly three zero eigenvalues (the
    skew-symmetric directions); with p the 12x12 Hessian has six."""
    V, g, H = O.ortho(_q(np.eye(3)), 1.0, 1.0)
    w = np.linalg.eigvalsh(H)
    assert (np.abs(w) < 1e-12).sum() == 6
    assert w.min() > -1e-12
    w9 = np.linalg.eigvalsh(H[3:, 3:])
    assert (np.abs(w9) < 1e-12).sum() == 3


def test_hessian_matches_hand_derived_closed_form():
    """d2V/da_k da_l = 4 kappa nu [(a_k.a_l - delta_kl) I + delta_kl A^T A + a_l a_k^T],
    derived by hand from V = kappa nu sum_ij (a_i.a_j - delta_ij)^2 (rows a_i of A),
    against the oracle's jets"""
    rng = np.random.default_rng(11)
    for _ in range(10):
        q = rng.normal(size=12)
        kap, vol = 1e3 * rng.uniform(1, 2), rng.uniform(0.1, 1.0)
        _, _, H = O.ortho(q, kap, vol)
        A = q[3:].reshape(3, 3)
        G, ATA = A @ A.T, A.T @ A
        Hc = np.zeros((12, 12))
        for k in range(3):
            for l in range(3):
                blk = (G[k, l] - (k == l)) * np.eye(3) + (k == l) * ATA + np.outer(A[l], A[k])
                Hc[3 + 3 * k:6 + 3 * k, 3 + 3 * l:6 + 3 * l] = 4 * kap * vol * blk
        np.testing.assert_allclose(H, Hc, rtol=0, atol=1e-13 * np.abs(H).max())


def test_body_block_is_unprojected_when_positive_definite():
    """the body block of the assembled Hessian is M + dt^2 hess V exactly when
    that block is positive definite (it is projected only when Cholesky fails)"""
    s = scenes.cube_stack(n=2)
    o = O.Oracle(s)
    q = s.q0.reshape(-1).copy()
    for b in range(s.nb):
        if not s.is_static[b]:
            # slight compression: the rotation modes of hess V turn negative
            # (4 kappa nu (s^2 - 1) < 0) while M still dominates them
            q[12 * b + 3:12 * b + 12] *= 1.0 - 1e-5
    st, E, g = o.energy_grad_hess(q)
    diag, _, _ = o.hessian()
    dt = s.params["dt"]
    for b in range(s.nb):
        if s.is_static[b]:
            continue
        vol = o.moments(b)[0]
        _, _, Hv = O.ortho(q[12 * b:12 * b + 12], s.kappa_body[b], vol)
        assert np.linalg.eigvalsh(Hv[3:, 3:]).min() < 0  # the 9x9 part alone is indefinite
        B = o.mass_matrix(b) + dt * dt * Hv
        assert np.linalg.eigvalsh(B).min() > 0
        np.testing.assert_allclose(diag[b], B, rtol=0, atol=1e-12 * np.abs(B).max())


def test_body_block_is_projected_when_indefinite():
    """strong compression makes M + dt^2 hess V indefinite: the assembled body
    block is then M + dt^2 H+, where H+ is hess V (the oracle's jets) with
    its residual-curvature part 4 kappa nu C (x) I (C = A A^T - I, over the
    rows of A) replaced by the eigenvalue clamp of C (numpy's eigh); the block
    is positive definite"""
    s = scenes.cube_stack(n=2)
    o = O.Oracle(s)
    q = s.q0.reshape(-1).copy()
    for b in range(s.nb):
        if not s.is_static[b]:
            q[12 * b + 3:12 * b + 12] *= 0.95
    o.energy_grad_hess(q)
    diag, _, _ = o.hessian()
    dt = s.params["dt"]
    n_proj = 0
    for b in range(s.nb):
        if s.is_static[b]:
            continue
        vol = o.moments(b)[0]
        qb = q[12 * b:12 * b + 12]
        _, _, Hv = O.ortho(qb, s.kappa_body[b], vol)
        M = o.mass_matrix(b)
        B = M + dt * dt * Hv
        if np.linalg.eigvalsh(B).min() > 0:
            continue
        n_proj += 1
        A = qb[3:].reshape(3, 3)
        C = A @ A.T - np.eye(3)
        w, V = np.linalg.eigh(C)
        Cp = (V * np.maximum(w, 0)) @ V.T
        Hp = Hv.copy()
        Hp[3:, 3:] += 4 * s.kappa_body[b] * vol * np.kron(Cp - C, np.eye(3))
        assert np.linalg.eigvalsh(Hp).min() >= -1e-12 * np.abs(Hp).max()
        np.testing.assert_allclose(diag[b], M + dt * dt * Hp, rtol=0, atol=1e-10 * np.abs(B).max())
        assert np.linalg.eigvalsh(diag[b]).min() > 0
    assert n_proj > 0

