"""Pins of the oracle's kinematics, mass properties and predictor against
closed forms (Sec. 3 Eq. kinematic, Sec. 3.1 Eq. mass, Sec. 4 predictor)."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2201_10022_gb300 import scenes


def _single_body_scene(verts, tris, q=None, qdot=None, density=1000.0, **params):
    B = scenes._Builder("one", 0)
    B.add(verts, tris, density=density)
    s = B.build(params)
    if q is not None:
        s.q0[0] = q
    if qdot is not None:
        s.qdot0[0] = qdot
    return s


def test_unit_cube_moments_closed_form():
    v, t = scenes.cube_mesh(1.0)
    o = O.Oracle(_single_body_scene(v, t))
    vol, m1, S = o.moments(0)
    assert vol == pytest.approx(1.0, rel=1e-14)
    assert np.abs(m1).max() < 1e-15
    np.testing.assert_allclose(S, np.eye(3) / 12.0, rtol=1e-13, atol=1e-15)


def test_box_second_moment_closed_form():
    a, b, c = 1.0, 0.2, 0.3
    v, t = scenes.box_mesh(a, b, c)
    o = O.Oracle(_single_body_scene(v, t))
    vol, m1, S = o.moments(0)
    assert vol == pytest.approx(a * b * c, rel=1e-13)
    np.testing.assert_allclose(S, np.diag([a * a, b * b, c * c]) * a * b * c / 12.0, rtol=1e-12, atol=1e-17)


def test_icosahedron_volume_closed_form_and_isotropy():
    r = 0.7
    v, t = scenes.icosphere_mesh(0, r)
    o = O.Oracle(_single_body_scene(v, t))
    vol, m1, S = o.moments(0)
    edge = r / math.sin(2.0 * math.pi / 5.0)
    assert vol == pytest.approx(5.0 / 12.0 * (3.0 + math.sqrt(5.0)) * edge ** 3, rel=1e-13)
    # the icosahedron's second moment is isotropic
    np.testing.assert_allclose(S, np.eye(3) * S[0, 0], atol=1e-14 * S[0, 0])


def test_moments_parallel_axis_theorem():
    v, t = scenes.icosphere_mesh(1, 0.3)
    shift = np.array([0.4, -1.3, 2.2])
    o0 = O.Oracle(_single_body_scene(v, t))
    o1 = O.Oracle(_single_body_scene(v + shift, t))
    vol0, m10, S0 = o0.moments(0)
    vol1, m11, S1 = o1.moments(0)
    assert vol1 == pytest.approx(vol0, rel=1e-12)
    np.testing.assert_allclose(m11, vol0 * shift, rtol=1e-12)
    np.testing.assert_allclose(S1, S0 + vol0 * np.outer(shift, shift), rtol=1e-11, atol=1e-13)


def test_mass_matrix_kinetic_energy_by_quadrature():
    """1/2 qdot^T M qdot equals the volume integral of 1/2 rho |xdot|^2,
    evaluated here by a midpoint rule over an off-centre box."""
    a, b, c = 0.6, 0.4, 0.3
    v, t = scenes.box_mesh(a, b, c)
    off = np.array([0.3, -0.2, 0.5])
    rho = 700.0
    o = O.Oracle(_single_body_scene(v + off, t, density=rho))
    M = o.mass_matrix(0)
    rng = np.random.default_rng(5)
    qd = rng.normal(size=12)
    n = 40
    gx = (np.arange(n) + 0.5) / n
    X, Y, Z = np.meshgrid(off[0] + (gx - 0.5) * a, off[1] + (gx - 0.5) * b, off[2] + (gx - 0.5) * c, indexing="ij")
    P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    Adot = qd[3:].reshape(3, 3)
    xdot = P @ Adot.T + qd[:3]
    ke_quad = 0.5 * rho * (xdot ** 2).sum() * (a * b * c) / len(P)
    # midpoint rule is exact for the constant and linear terms; the quadratic
    # term carries an O(1/n^2) error
    assert 0.5 * qd @ M @ qd == pytest.approx(ke_quad, rel=2e-3)
    # exact check of the structure: M (g,0,0,0) = rho (vol g, m1 g_c)
    vol, m1, S = o.moments(0)
    assert M[0, 0] == pytest.approx(rho * vol)
    np.testing.assert_allclose(M[0, 3:6], rho * m1, rtol=1e-12)
    np.testing.assert_allclose(M[3:6, 3:6], rho * S, rtol=1e-12)
    np.testing.assert_allclose(M, M.T, atol=0)


def test_vertex_map_rotation_and_translation():
    v, t = scenes.cube_mesh(1.0)
    R = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])  # 90 deg about z
    q = np.concatenate([[1.0, 2.0, 3.0], R.reshape(-1)])
    o = O.Oracle(_single_body_scene(v, t, q=q))
    x = o.vertices(q)
    exp = np.stack([-v[:, 1] + 1.0, v[:, 0] + 2.0, v[:, 2] + 3.0], axis=1)
    np.testing.assert_array_equal(x, exp)


def test_free_fall_implicit_euler_closed_form():
    """p^n = p^0 + n dt v^0 + dt^2 g n(n+1)/2 and A^n = A^0 for a body that
    touches nothing; holds for a spinning body too (V does not depend on p
    and M is block diagonal for a centred body)."""
    v, t = scenes.icosphere_mesh(1, 0.2)
    rng = np.random.default_rng(0)
    R = scenes.random_rotation(rng)
    v0 = np.array([0.3, -0.2, 1.5])
    q = np.concatenate([[0.0, 0.0, 5.0], R.reshape(-1)])
    qd = np.concatenate([v0, np.zeros(9)])
    s = _single_body_scene(v, t, q=q, qdot=qd)
    o = O.Oracle(s)
    dt, g = s.params["dt"], np.array(s.params["gravity"])
    n = 12
    r, st = o.step(n)
    assert r == 0
    qn, qdn = o.get_state()
    p_exp = q[:3] + n * dt * v0 + dt * dt * g * n * (n + 1) / 2
    np.testing.assert_allclose(qn[0, :3], p_exp, rtol=0, atol=1e-13)
    np.testing.assert_allclose(qn[0, 3:], q[3:], rtol=0, atol=1e-13)
    # spinning: translation still follows the closed form
    W = np.array([[0, -2.0, 1.0], [2.0, 0, -0.5], [-1.0, 0.5, 0]])
    qd2 = np.concatenate([v0, (W @ R).reshape(-1)])
    o2 = O.Oracle(_single_body_scene(v, t, q=q, qdot=qd2))
    r, st = o2.step(n)
    assert r == 0
    qn2, _ = o2.get_state()
    np.testing.assert_allclose(qn2[0, :3], p_exp, rtol=0, atol=1e-11)


def test_predictor_gravity_term():
    """qtilde = q + dt qdot + dt^2 M^-1 f with f = int rho J^T g; for any body
    M^-1 f = (g, 0, 0, 0) since M (g,0,0,0) = f."""
    v, t = scenes.box_mesh(0.5, 0.3, 0.2)
    rng = np.random.default_rng(2)
    q = np.concatenate([[0.1, 0.2, 0.3], scenes.random_rotation(rng).reshape(-1)])
    qd = rng.normal(size=12)
    s = _single_body_scene(v + np.array([0.2, 0.1, -0.3]), t, q=q, qdot=qd)
    o = O.Oracle(s)
    dt = s.params["dt"]
    g = np.array(s.params["gravity"])
    exp = q + dt * qd + dt * dt * np.concatenate([g, np.zeros(9)])
    np.testing.assert_allclose(o.qtilde()[0], exp, rtol=1e-14, atol=1e-15)
