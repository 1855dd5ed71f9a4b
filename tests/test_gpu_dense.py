"""Dense direct solve of small systems (dense_max_dofs > 0): the solution of
the GPU's own assembled matrix against numpy's, trajectories against the
oracle (whose solve is a dense Cholesky too), the adjoint against the
oracle's, and a 10-cube stack where the block-Jacobi PCG needs many
iterations."""
import numpy as np
import pytest

import oracle as O
from paper_2201_10022_gb300 import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def abd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_10022_gb300 import abd as A
    A.load()
    return A


def _dense_matrix(s, diag, bp, blocks):
    dyn = np.nonzero(s.is_static == 0)[0]
    idx = {b: k for k, b in enumerate(dyn)}
    n = 12 * len(dyn)
    H = np.zeros((n, n))
    for b in dyn:
        H[12 * idx[b]:12 * idx[b] + 12, 12 * idx[b]:12 * idx[b] + 12] = diag[b]
    for (a, b), B in zip(bp.tolist(), blocks):
        if a in idx and b in idx:
            H[12 * idx[a]:12 * idx[a] + 12, 12 * idx[b]:12 * idx[b] + 12] = B
            H[12 * idx[b]:12 * idx[b] + 12, 12 * idx[a]:12 * idx[a] + 12] = B.T
    return H, dyn


@pytest.mark.parametrize("name", ["stack", "packed", "tower"])
def test_dense_solve_matches_numpy(abd, name):
    if name == "stack":
        s = scenes.cube_stack(seed=1, gap=0.0004)
    elif name == "packed":
        s = scenes.packed_cubes(nx=3, ny=3, nz=3)  # 28 bodies: several 32-wide tiles, a ragged last one
    else:
        s = scenes.throw_stack(n_throw=8)
    gpu = abd.AbdScene(s, dense_max_dofs=3072)
    E, g, cnt = gpu.energy_grad_hess(torch.tensor(s.q0))
    H, dyn = _dense_matrix(s, *gpu.hessian())
    dq, st = gpu.solve(-g)
    b = -g.cpu().numpy()[dyn].reshape(-1)
    ref = np.linalg.solve(H, b)
    got = dq.cpu().numpy()[dyn].reshape(-1)
    cond = np.linalg.cond(H)
    assert np.abs(got - ref).max() <= 1e-15 * cond * np.abs(ref).max(), (name, cond)
    assert np.linalg.norm(H @ got - b) <= 1e-12 * np.linalg.norm(H, 2) * np.linalg.norm(got)
    assert st["iterations"] == 0
    assert np.abs(dq.cpu().numpy()[s.is_static == 1]).max(initial=0.0) == 0.0


def test_dense_trajectory_cube_stack(abd):
    s = scenes.cube_stack(seed=1)
    orc = O.Oracle(s)
    gpu = abd.AbdScene(s, newton_tol=orc.newton_tol, dense_max_dofs=3072)
    worst = 0.0
    for _ in range(40):
        gpu.step(1)
        r, _ = orc.step(1)
        assert r == 0, O.ERRORS[r]
        xg = orc.vertices(gpu.get_state()[0].cpu().numpy().reshape(-1))
        xo = orc.vertices(orc.get_state()[0].reshape(-1))
        worst = max(worst, np.abs(xg - xo).max())
    assert worst <= 1e-8 * orc.l_bbox


def test_dense_adjoint_matches_oracle(abd):
    B = scenes._Builder("adjoint", 0)
    gv, gt = scenes.box_mesh(2.0, 2.0, 0.4)
    B.add(gv, gt, p=(0.0, 0.0, -0.2), static=True)
    cv, ct = scenes.cube_mesh(0.2)
    B.add(cv, ct, R=scenes.small_rotation(np.random.default_rng(1), 2.0), p=(0.0, 0.0, 0.1 + 0.0012),
          v=(0.4, -0.2, 0.05), kappa=1e6)
    B.add(cv, ct, p=(0.35, 0.0, 0.1 + 0.0012), v=(-0.3, 0.1, 0.0), kappa=2e6)
    s = B.build(dict(mu=0.0))
    o = O.Oracle(s, newton_rel=1e-14, newton_max=200)
    o.set_state(s.q0, s.qdot0)
    r, _ = o.step(1)
    assert r == 0
    qn, _ = o.get_state()
    rng = np.random.default_rng(3)
    gq0 = rng.normal(size=s.q0.shape)
    gq0[s.is_static == 1] = 0.0
    st, Mlam, gk = o.adjoint_step(s.q0, s.qdot0, qn, gq0)
    assert st == 0
    gpu = abd.AbdScene(s, dense_max_dofs=3072)
    dev = gpu.device
    gq = torch.tensor(gq0, device=dev)
    gqd = torch.zeros_like(gq)
    gkt = torch.zeros(s.nb, dtype=torch.float64, device=dev)
    gpu.adjoint_step(s.q0, s.qdot0, qn, gq, gqd, gkt)
    dt = s.params["dt"]
    np.testing.assert_allclose(gqd.cpu().numpy(), dt * Mlam, rtol=0, atol=1e-9 * np.abs(dt * Mlam).max())
    np.testing.assert_allclose(gkt.cpu().numpy(), gk, rtol=0, atol=1e-9 * np.abs(gk).max())


def test_dense_steps_the_tower(abd):
    """the 10-cube stack settling (8 thrown cubes still in flight): the
    direct solve takes every Newton step without iterations, and the end
    state agrees with the PCG path's within the inexact-Newton tolerances"""
    s = scenes.throw_stack(n_throw=8)
    d = abd.AbdScene(s, dense_max_dofs=3072)
    p = abd.AbdScene(s, pcg_max=20000)
    sd = d.step(8)
    sp = p.step(8)
    print(f"tower, 8 steps: Newton {sd['newton_iters']} (dense) / {sp['newton_iters']} (PCG), "
          f"PCG iterations {sp['pcg_iters']}")
    assert sd["pcg_iters"] == 0 and sd["n_active"] > 0
    qd, qp = d.get_state()[0].cpu().numpy(), p.get_state()[0].cpu().numpy()
    assert np.abs(qd - qp).max() < 1e-4
