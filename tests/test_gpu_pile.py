"""CUDA path (through the C ABI) against the CPU oracle on the benchmark's own
recipe with friction: the lattice pile (cubes, subdivision-1 icospheres and
1 x 0.2 x 0.2 m boxes, mu = 0.3) on a 6x6x3 sub-lattice of 109 bodies, from
oracle-written snapshots (tests/golden/pile_snapshots.npz: free fall, first
ground impacts, resting and sliding contacts, second layer landing), and a
small scene whose friction couples two dynamic bodies through point-face,
point-edge, edge-edge (line-line and point-edge) contacts.

At each state: candidate, active and lagged friction pair sets with distance
types bit-exact; the friction records (mu lambda, closest-point weights,
normal, lagged offset) to rounding; E, g (1e-10) and Hessian blocks (1e-9 of
the largest entry), off-diagonal friction blocks included, at a point inside
the step; one time step from the snapshot within 1e-8 of the box diagonal at
the oracle's Newton tolerance (Sec. 4: lagged friction V_F, barrier V_C,
Sec. 4.3 assembly)."""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2201_10022_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))
SNAP = np.load(os.path.join(HERE, "golden", "pile_snapshots.npz"))
STEPS = [int(k) for k in SNAP["steps"]]


@pytest.fixture(scope="module")
def abd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_10022_gb300 import abd as A
    A.load()
    return A


def pile_scene():
    d = SNAP["dims"]
    return scenes.lattice_pile(seed=3, nx=int(d[0]), ny=int(d[1]), nz=int(d[2]))


def _rot(axis, deg):
    a = np.asarray(axis, float)
    a /= np.linalg.norm(a)
    t = math.radians(deg)
    return scenes.quat_to_mat(math.cos(t / 2), *(math.sin(t / 2) * a))


def friction_pair_scene(g=0.0006, overhang=True):
    """two dynamic stacks on a static ground, every contact within d-hat at
    the start: a cube lying on one edge across a sliding cube's top face
    (turned 23 degrees; with overhang, one end of its edge just past the
    lower cube's top edge: point-face, point-edge, line-line and point-edge
    edge-edge pairs), and a box lying across another box (line-line
    crossings)"""
    B = scenes._Builder("friction_pair", 0)
    gv, gt = scenes.box_mesh(6.0, 6.0, 1.0)
    B.add(gv, gt, p=(0.0, 0.0, -0.5), static=True)
    cv, ct = scenes.cube_mesh(0.2)
    B.add(cv, ct, p=(0.0, 0.0, 0.1 + g), v=(0.4, 0.1, 0.0))
    R = _rot((0, 0, 1), 23.0) @ _rot((1, 0, 0), 45.0)
    xv = (R @ cv.T).T
    px = 0.1 + 0.0003 - 0.1 * math.cos(math.radians(23.0)) if overhang else 0.035
    B.add(cv, ct, R=R, p=(px, -0.02, 0.2 + 2 * g - xv[:, 2].min()), v=(-0.3, 0.2, 0.0))
    bv, bt = scenes.box_mesh(1.0, 0.2, 0.2)
    B.add(bv, bt, p=(1.2, 0.0, 0.1 + g), v=(0.0, 0.3, 0.0))
    R2 = _rot((0, 0, 1), 71.0) @ _rot((1, 0, 0), 3.0)
    xv = (R2 @ bv.T).T
    B.add(bv, bt, R=R2, p=(1.3, 0.05, 0.2 + 2 * g - xv[:, 2].min()), v=(0.2, -0.2, 0.0))
    return B.build(dict(mu=0.3))


def _key(d, k):
    return (int(d["kind"][k]), int(d["i"][k]), int(d["j"][k]))


def _pair_bodies(s, kind, i, j):
    if kind == 0:
        return s.vbody[i], s.vbody[s.tri[j][0]]
    return s.vbody[s.edge[i][0]], s.vbody[s.edge[j][0]]


def check_friction_records(gpu, orc):
    """lagged friction sets bit-exact (kind, i, j, type); mu lambda, weights,
    normal and offset to rounding; returns the oracle's set"""
    fg, fo = gpu.pairs(2), orc.pairs(2)
    kg = {_key(fg, k): k for k in range(len(fg["kind"]))}
    ko = {_key(fo, k): k for k in range(len(fo["kind"]))}
    # the GPU keeps a record for every active pair; the oracle drops pairs
    # whose normal force is zero (an exactly parallel edge pair, mollifier
    # m = 0): those extra records must carry mu lambda = 0 exactly
    extra = set(kg) - set(ko)
    assert all(fg["val"][kg[key]] == 0.0 for key in extra), [(key, fg["val"][kg[key]]) for key in extra]
    kg = {key: m for key, m in kg.items() if key not in extra}
    assert set(kg) == set(ko)
    ga, na, ra = gpu.friction_records()
    oa, on, orr = orc.friction_records()
    for key, k in ko.items():
        m = kg[key]
        assert fg["type"][m] == fo["type"][k], key
        assert abs(fg["val"][m] - fo["val"][k]) <= 1e-10 * abs(fo["val"][k]), key
        assert np.abs(ga[m] - oa[k]).max() <= 1e-11, (key, ga[m], oa[k])
        assert np.abs(na[m] - on[k]).max() <= 1e-9, (key, na[m], on[k])
        assert np.abs(ra[m] - orr[k]).max() <= 1e-12 * max(1.0, np.abs(orr[k]).max()), key
    return fo


def check_system(gpu, orc, s, q):
    """pair sets, energies, gradient and Hessian blocks at q (friction lagged
    at the current state of both sides)"""
    E, g, cnt = gpu.energy_grad_hess(torch.tensor(q))
    st, Eo, go = orc.energy_grad_hess(q.reshape(-1))
    assert st == 0
    for which in (0, 1):
        pg, po = gpu.pairs(which), orc.pairs(which)
        sg = set(zip(pg["kind"].tolist(), pg["i"].tolist(), pg["j"].tolist(),
                     (pg["type"] if which else 0 * pg["kind"]).tolist()))
        so = set(zip(po["kind"].tolist(), po["i"].tolist(), po["j"].tolist(),
                     (po["type"] if which else 0 * po["kind"]).tolist()))
        assert sg == so, (which, len(sg), len(so))
    np.testing.assert_allclose(E, Eo, rtol=1e-10, atol=1e-12)
    gg = g.cpu().numpy()
    scale = np.abs(go).max()
    assert np.abs(gg - go).max() <= 1e-10 * scale, (np.abs(gg - go).max(), scale)
    diag, bp, blocks = gpu.hessian()
    od, obp, oblk = orc.hessian()
    hs = max(np.abs(od).max(), np.abs(oblk).max() if len(oblk) else 0.0)
    np.testing.assert_allclose(diag, od, atol=1e-9 * hs, rtol=0)
    gb = {tuple(k): B for k, B in zip(bp.tolist(), blocks)}
    for k, B in zip(obp.tolist(), oblk):
        assert tuple(k) in gb, k
        np.testing.assert_allclose(gb[tuple(k)], B, atol=1e-9 * hs, rtol=0)
    return obp, oblk, E


def _inside_step(orc, s, q0, qd0):
    """a state inside the step: halfway from the snapshot to the oracle's
    converged next state (the oracle is left at the snapshot)"""
    orc.set_state(q0, qd0)
    r, _ = orc.step(1)
    assert r == 0, O.ERRORS[r]
    q1, _ = orc.get_state()
    orc.set_state(q0, qd0)
    return q0 + 0.5 * (q1 - q0), q1


@pytest.fixture(scope="module")
def pile():
    s = pile_scene()
    return s, O.Oracle(s, newton_max=500)


@pytest.mark.parametrize("step", STEPS)
def test_pile_snapshot_system_and_step(abd, pile, step):
    s, orc = pile
    q0, qd0 = SNAP[f"q_{step}"], SNAP[f"qdot_{step}"]
    qmid, q1 = _inside_step(orc, s, q0, qd0)
    gpu = abd.AbdScene(s, newton_tol=orc.newton_tol)
    gpu.set_state(q0, qd0)
    fo = check_friction_records(gpu, orc)
    obp, oblk, E = check_system(gpu, orc, s, qmid)
    if step >= 35:
        assert len(fo["kind"]) > 0 and E[4] > 0.0   # friction at work
    # one step from the snapshot
    gpu.set_state(q0, qd0)
    gpu.step(1)
    qg, _ = gpu.get_state()
    xg = orc.vertices(qg.cpu().numpy().reshape(-1))
    xo = orc.vertices(q1.reshape(-1))
    assert np.abs(xg - xo).max() <= 1e-8 * orc.l_bbox, (np.abs(xg - xo).max(), orc.l_bbox)


def test_friction_between_dynamic_bodies(abd):
    """friction records and off-diagonal friction blocks between two dynamic
    bodies, every pair type of the scene, at the start and at a tangentially
    moved state (the friction terms' displacement u nonzero)"""
    s = friction_pair_scene()
    orc = O.Oracle(s)
    gpu = abd.AbdScene(s, newton_tol=orc.newton_tol)
    fo = check_friction_records(gpu, orc)
    dd_types = set()
    for k in range(len(fo["kind"])):
        a, b = _pair_bodies(s, *_key(fo, k))
        if not s.is_static[a] and not s.is_static[b]:
            dd_types.add((int(fo["kind"][k]), int(fo["type"][k])))
    # point-face, point-edge, edge-edge line-line and point-edge, all between dynamic bodies
    assert {(0, 6), (0, 4), (1, 8)} <= dd_types and any(k == 1 and 4 <= t <= 7 for k, t in dd_types), dd_types
    rng = np.random.default_rng(2)
    dyn = s.is_static == 0
    for trial in range(2):
        q = s.q0.copy()
        q[dyn, :2] += rng.normal(size=(dyn.sum(), 2)) * 2e-5   # tangential slide
        q[dyn, 3:] += rng.normal(size=(dyn.sum(), 9)) * 2e-6
        obp, oblk, E = check_system(gpu, orc, s, q)
        assert E[4] > 0.0
        # off-diagonal blocks of dynamic body pairs carry friction
        assert any(not s.is_static[a] and not s.is_static[b] and np.abs(B).max() > 0
                   for (a, b), B in zip(obp.tolist(), oblk))


def test_friction_scene_steps(abd):
    """steps of the scene with the edge-on cube fully on the lower face
    (friction between dynamic bodies through point-face and line-line
    pairs), GPU against oracle within 1e-8 of the box diagonal after each.
    With the overhang the oracle's Newton loop does not reach its tolerance
    within its cap (the contact switches between point-face and point-edge
    types), so the step comparison uses this placement."""
    s = friction_pair_scene(overhang=False)
    orc = O.Oracle(s)
    gpu = abd.AbdScene(s, newton_tol=orc.newton_tol)
    dyn_fric = 0
    for k in range(4):
        fo = orc.pairs(2)
        dyn_fric += sum(1 for m in range(len(fo["kind"]))
                        if not any(s.is_static[b] for b in _pair_bodies(s, *_key(fo, m))))
        gpu.step(1)
        r, _ = orc.step(1)
        assert r == 0, O.ERRORS[r]
        qg, _ = gpu.get_state()
        qo, _ = orc.get_state()
        dx = np.abs(orc.vertices(qg.cpu().numpy().reshape(-1)) - orc.vertices(qo.reshape(-1))).max()
        assert dx <= 1e-8 * orc.l_bbox, (k, dx, orc.l_bbox)
    assert dyn_fric > 0
