"""CUDA implicit-function adjoint (abd_adjoint_step, the Rollout autograd
function) against the oracle's adjoint and against central finite
differences of the CUDA forward map, on a frictionless contact scene."""
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


def contact_scene():
    B = scenes._Builder("adjoint", 0)
    gv, gt = scenes.box_mesh(2.0, 2.0, 0.4)
    B.add(gv, gt, p=(0.0, 0.0, -0.2), static=True)
    cv, ct = scenes.cube_mesh(0.2)
    B.add(cv, ct, R=scenes.small_rotation(np.random.default_rng(1), 2.0), p=(0.0, 0.0, 0.1 + 0.0012),
          v=(0.4, -0.2, 0.05), kappa=1e6)
    B.add(cv, ct, p=(0.35, 0.0, 0.1 + 0.0012), v=(-0.3, 0.1, 0.0), kappa=2e6)
    return B.build(dict(mu=0.0))


TARGET = np.array([0.3, -0.1, 0.2])
NSTEPS = 4


def oracle_states(s):
    o = O.Oracle(s, newton_rel=1e-14, newton_max=200)
    o.set_state(s.q0, s.qdot0)
    states = [(s.q0.copy(), s.qdot0.copy())]
    for _ in range(NSTEPS):
        r, _ = o.step(1)
        assert r == 0, O.ERRORS[r]
        q, qd = o.get_state()
        states.append((q.copy(), qd.copy()))
    return o, states


def dloss(s, qK):
    dyn = s.is_static == 0
    g = np.zeros_like(qK)
    g[dyn, :3] = 2.0 * (qK[dyn, :3].mean(axis=0) - TARGET) / dyn.sum()
    return g


def oracle_backward(o, s, states, gq, gqd):
    dt = s.params["dt"]
    gk = np.zeros(s.nb)
    for t in range(len(states) - 2, -1, -1):
        (qt, qdt), (qn, _) = states[t], states[t + 1]
        st, Mlam, gkt = o.adjoint_step(qt, qdt, qn, gq + gqd / dt)
        assert st == 0, O.ERRORS[st]
        gq, gqd = Mlam - gqd / dt, dt * Mlam
        gk += gkt
    gq[s.is_static == 1] = 0.0
    gqd[s.is_static == 1] = 0.0
    return gq, gqd, gk


def test_adjoint_steps_match_oracle(abd):
    s = contact_scene()
    o, states = oracle_states(s)
    gq0, gqd0, gk0 = oracle_backward(o, s, states, dloss(s, states[-1][0]), np.zeros_like(s.q0))
    gpu = abd.AbdScene(s)
    dev = gpu.device
    gq = torch.tensor(dloss(s, states[-1][0]), device=dev)
    gqd = torch.zeros_like(gq)
    gk = torch.zeros(s.nb, dtype=torch.float64, device=dev)
    for t in range(NSTEPS - 1, -1, -1):
        (qt, qdt), (qn, _) = states[t], states[t + 1]
        st = gpu.adjoint_step(qt, qdt, qn, gq, gqd, gk)
        assert st["rel_residual"] <= 1e-11
    scale = np.abs(gqd0).max()
    np.testing.assert_allclose(gqd.cpu().numpy(), gqd0, rtol=0, atol=1e-9 * scale)
    np.testing.assert_allclose(gq.cpu().numpy(), gq0, rtol=0, atol=1e-9 * np.abs(gq0).max())
    np.testing.assert_allclose(gk.cpu().numpy(), gk0, rtol=0, atol=1e-9 * np.abs(gk0).max())


def _rollout_grads(abd, s):
    from paper_2201_10022_gb300.autograd import Rollout
    orc = O.Oracle(s)
    # a tight Newton and linear tolerance: the finite differences below see
    # the forward map's solver noise
    gpu = abd.AbdScene(s, newton_tol=1e-5 * orc.newton_tol, pcg_rel_tol=1e-12)
    dev = gpu.device
    q0 = torch.tensor(s.q0, device=dev, requires_grad=True)
    qd0 = torch.tensor(s.qdot0, device=dev, requires_grad=True)
    kb = torch.tensor(s.kappa_body, device=dev, requires_grad=True)
    qK, _ = Rollout.apply(gpu, NSTEPS, q0, qd0, kb)
    dyn = torch.tensor(s.is_static == 0, device=dev)
    loss = ((qK[dyn, :3].mean(dim=0) - torch.tensor(TARGET, device=dev)) ** 2).sum()
    loss.backward()
    return gpu, loss.item(), qd0.grad.cpu().numpy(), kb.grad.cpu().numpy()


def test_rollout_gradient_matches_oracle(abd):
    s = contact_scene()
    o, states = oracle_states(s)
    _, gqd0, gk0 = oracle_backward(o, s, states, dloss(s, states[-1][0]), np.zeros_like(s.q0))
    _, _, gqd, gk = _rollout_grads(abd, s)
    np.testing.assert_allclose(gqd, gqd0, rtol=0, atol=1e-7 * np.abs(gqd0).max())
    np.testing.assert_allclose(gk, gk0, rtol=0, atol=1e-7 * np.abs(gk0).max())


def test_rollout_gradient_matches_central_differences(abd):
    s = contact_scene()
    gpu, _, gqd, gk = _rollout_grads(abd, s)
    dyn = s.is_static == 0

    def loss(qd0):
        gpu.set_state(torch.tensor(s.q0), torch.tensor(qd0))
        gpu.step(NSTEPS)
        qK = gpu.get_state()[0].cpu().numpy()
        return float(np.sum((qK[dyn, :3].mean(axis=0) - TARGET) ** 2))

    h = 1e-6
    for b in (1, 2):
        for k in (0, 1, 2, 4, 9):
            e = np.zeros_like(s.qdot0)
            e[b, k] = h
            fd = (loss(s.qdot0 + e) - loss(s.qdot0 - e)) / (2 * h)
            # absolute floor: the finite-difference noise of the loss (~1e-15)
            # over 2h, against components down to 1e-9 of the largest
            assert gqd[b, k] == pytest.approx(fd, rel=2e-4, abs=2e-7 * np.abs(gqd).max()), (b, k)


def test_adjoint_steps_match_oracle_on_the_throw_stack(abd):
    """the adjoint workload itself (64 cubes thrown at a 10-cube stack, 74
    dynamic bodies): five steps forward by the oracle, then the adjoint of
    the last two (the stack's cubes in contact, 60 and 68 active pairs) on
    the GPU (PCG with the cluster preconditioner) against the oracle's (dense
    Cholesky), for a loss on the mean translation of every dynamic body.
    (At the third step, the first with contact, the unprojected Hessian of
    the converged state has an eigenvalue of -0.05 against 5e5: there the
    implicit-function Jacobian is not defined by a Cholesky solve, on either
    side.)"""
    s = scenes.throw_stack(seed=4)
    nsteps, nback = 5, 2
    dyn = s.is_static == 0
    o = O.Oracle(s, newton_max=300)
    o.set_state(s.q0, s.qdot0)
    states = [(s.q0.copy(), s.qdot0.copy())]
    for _ in range(nsteps):
        r, _ = o.step(1)
        assert r == 0, O.ERRORS[r]
        q, qd = o.get_state()
        states.append((q.copy(), qd.copy()))
    assert o.pairs(1)["kind"].size > 0  # contact at the last state
    states = states[-(nback + 1):]
    g = np.zeros_like(s.q0)
    g[dyn, :3] = 2.0 * (states[-1][0][dyn, :3].mean(axis=0) - np.array([-0.5, 0.0, 0.25])) / dyn.sum()
    gq0, gqd0, gk0 = oracle_backward(o, s, states, g.copy(), np.zeros_like(s.q0))
    gpu = abd.AbdScene(s)
    dev = gpu.device
    gq = torch.tensor(g, device=dev)
    gqd = torch.zeros_like(gq)
    gk = torch.zeros(s.nb, dtype=torch.float64, device=dev)
    for t in range(nback - 1, -1, -1):
        (qt, qdt), (qn, _) = states[t], states[t + 1]
        st = gpu.adjoint_step(qt, qdt, qn, gq, gqd, gk)
        assert st["rel_residual"] <= 1e-11
    np.testing.assert_allclose(gqd.cpu().numpy(), gqd0, rtol=0, atol=1e-9 * np.abs(gqd0).max())
    np.testing.assert_allclose(gq.cpu().numpy(), gq0, rtol=0, atol=1e-9 * np.abs(gq0).max())
    np.testing.assert_allclose(gk.cpu().numpy(), gk0, rtol=0, atol=1e-9 * max(np.abs(gk0).max(), 1e-300))


def test_adjoint_matches_oracle_over_20_steps_of_the_throw_stack(abd):
    """the adjoint workload over a 20-step horizon (the thrown block in
    flight, the stack settling, the first impacts), with the benchmark's
    solver setting (dense direct solves): every step's GPU adjoint from the
    oracle's inputs against the oracle's outputs (states, inputs and outputs
    from tests/golden/throw_stack_adjoint.npz, written by the oracle alone),
    then the whole chain on the GPU against the oracle's chain.  Steps whose
    converged state is a saddle of the IP (unprojected Hessian with a
    negative eigenvalue) are solved by the signed dense factorisation on the
    GPU and by LDL^T in the oracle."""
    import os
    G = np.load(os.path.join(os.path.dirname(__file__), "golden", "throw_stack_adjoint.npz"))
    s = scenes.throw_stack(seed=int(G["seed"]))
    q, qd = G["q"], G["qdot"]
    n = q.shape[0] - 1
    assert (G["hess_eig"][:, 0] < 0).any()  # the horizon holds an indefinite step
    gpu = abd.AbdScene(s, dense_max_dofs=3072)
    dev = gpu.device

    def t64(a):
        return torch.tensor(np.ascontiguousarray(a), device=dev)

    # the kappa gradient of a step with no contact and rigid bodies is
    # rounding noise (1e-49 here): it is compared on the scale of the largest
    # step's kappa gradient
    gk_scale = np.abs(G["gk_out"]).max()
    for t in range(n):
        gq, gqd = t64(G["gq_in"][t]), t64(G["gqd_in"][t])
        gk = torch.zeros(s.nb, dtype=torch.float64, device=dev)
        gpu.adjoint_step(q[t], qd[t], q[t + 1], gq, gqd, gk)
        for got, ref, scale in ((gq, G["gq_out"][t], np.abs(G["gq_out"][t]).max()),
                                (gqd, G["gqd_out"][t], np.abs(G["gqd_out"][t]).max()),
                                (gk, G["gk_out"][t], gk_scale)):
            np.testing.assert_allclose(got.cpu().numpy(), ref, rtol=0, atol=1e-9 * scale, err_msg=f"step {t}")
    gq, gqd = t64(G["gq_in"][n - 1]), t64(G["gqd_in"][n - 1])
    gk = torch.zeros(s.nb, dtype=torch.float64, device=dev)
    for t in range(n - 1, -1, -1):
        gpu.adjoint_step(q[t], qd[t], q[t + 1], gq, gqd, gk)
    gk0 = G["gk_out"].sum(axis=0)
    np.testing.assert_allclose(gq.cpu().numpy(), G["gq_out"][0], rtol=0, atol=1e-8 * np.abs(G["gq_out"][0]).max())
    np.testing.assert_allclose(gqd.cpu().numpy(), G["gqd_out"][0], rtol=0, atol=1e-8 * np.abs(G["gqd_out"][0]).max())
    np.testing.assert_allclose(gk.cpu().numpy(), gk0, rtol=0, atol=1e-8 * np.abs(gk0).max())
