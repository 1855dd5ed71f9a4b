"""Mixed-precision mode (precision = 1: the barrier Hessian's PSD projection
from an FP32 eigenbasis, everything else FP64) against the FP64 oracle: pair
sets bit-exact, energies and gradients within 1e-10 (they are FP64), Hessian
blocks within FP32 accuracy, and trajectories with their error stated."""
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


def _pairset(d):
    return set(zip(d["kind"].tolist(), d["i"].tolist(), d["j"].tolist(), d["type"].tolist()))


def _scenes():
    out = []
    for seed, kinds in [(1, ("cube", "ico1")), (3, ("box", "cube"))]:
        out.append((f"pair{seed}", scenes.random_pair(seed, kinds=kinds, sep=0.0003)))
    out.append(("stack", scenes.cube_stack(seed=1, gap=0.0004)))
    out.append(("packed", scenes.packed_cubes(nx=2, ny=2, nz=2)))
    return out


@pytest.mark.parametrize("name,s", _scenes(), ids=[n for n, _ in _scenes()])
def test_mixed_energy_gradient_exact_hessian_fp32(abd, name, s):
    gpu = abd.AbdScene(s, precision=1)
    orc = O.Oracle(s)
    E, g, _ = gpu.energy_grad_hess(torch.tensor(s.q0))
    st, Eo, go = orc.energy_grad_hess(s.q0.reshape(-1))
    assert st == 0
    assert _pairset(gpu.pairs(1)) == _pairset(orc.pairs(1))
    np.testing.assert_allclose(E, Eo, rtol=1e-10, atol=1e-14)
    gg = g.cpu().numpy()
    assert np.abs(gg - go).max() <= 1e-10 * np.abs(go).max()
    diag, bp, blocks = gpu.hessian()
    od, obp, oblk = orc.hessian()
    hs = max(np.abs(od).max(), np.abs(oblk).max() if len(oblk) else 0)
    # FP32 eigenbasis: entries within a few FP32 units of the largest entry
    np.testing.assert_allclose(diag, od, atol=2e-6 * hs, rtol=0)
    gb = {tuple(k): B for k, B in zip(bp.tolist(), blocks)}
    for k, B in zip(obp.tolist(), oblk):
        np.testing.assert_allclose(gb[tuple(k)], B, atol=2e-6 * hs, rtol=0)


def _trajectory(abd, s, nsteps, **kw):
    """accumulated deviation of a free run, and the per-step deviation when
    every GPU step starts from the oracle's state (no accumulation)"""
    orc = O.Oracle(s)
    gpu = abd.AbdScene(s, newton_tol=orc.newton_tol, **kw)
    one = abd.AbdScene(s, newton_tol=orc.newton_tol, **kw)
    worst, per_step = 0.0, 0.0
    for _ in range(nsteps):
        qo0, qdo0 = orc.get_state()
        one.set_state(torch.tensor(qo0.reshape(s.nb, 12)), torch.tensor(qdo0.reshape(s.nb, 12)))
        one.step(1)
        gpu.step(1)
        r, _ = orc.step(1)
        assert r == 0, O.ERRORS[r]
        qo, _ = orc.get_state()
        xo = orc.vertices(qo.reshape(-1))
        worst = max(worst, np.abs(orc.vertices(gpu.get_state()[0].cpu().numpy().reshape(-1)) - xo).max())
        per_step = max(per_step, np.abs(orc.vertices(one.get_state()[0].cpu().numpy().reshape(-1)) - xo).max())
    return worst, per_step, orc.l_bbox


def test_mixed_trajectory_cube_stack(abd, record_property):
    s = scenes.cube_stack(seed=1)
    worst, per_step, L = _trajectory(abd, s, 40, precision=1)
    record_property("max_vertex_deviation_over_lbbox", worst / L)
    print(f"mixed cube stack, 40 steps: max vertex deviation {worst / L:.3e} L_bbox, per step {per_step / L:.3e}")
    assert per_step <= 1e-8 * L, (per_step, L)
    assert worst <= 1e-7 * L, (worst, L)


def test_mixed_trajectory_friction_slide(abd, record_property):
    """A cube sliding on 4-6 marginal contacts amplifies any difference in the
    converged point (x200 a step at first): the FP64 path stays within 1e-8 of
    the oracle only because it takes the oracle's Newton iterates.  The mixed
    path converges to the same tolerance along other iterates; its per-step
    error is bounded like the FP64 path's, its accumulated error is stated."""
    B = scenes._Builder("slide", 0)
    gv, gt = scenes.box_mesh(10.0, 10.0, 1.0)
    B.add(gv, gt, p=(0.0, 0.0, -0.5), static=True)
    cv, ct = scenes.cube_mesh(0.2)
    B.add(cv, ct, p=(0.0, 0.0, 0.1 + 0.0015), v=(2.0, 0.3, 0.0))
    s = B.build(dict(mu=0.3))
    worst, per_step, L = _trajectory(abd, s, 25, precision=1)
    record_property("max_vertex_deviation_over_lbbox", worst / L)
    record_property("max_per_step_deviation_over_lbbox", per_step / L)
    print(f"mixed friction slide, 25 steps: max vertex deviation {worst / L:.3e} L_bbox, per step {per_step / L:.3e}")
    assert per_step <= 1e-8 * L, (per_step, L)
    assert worst <= 1e-4 * L, (worst, L)
