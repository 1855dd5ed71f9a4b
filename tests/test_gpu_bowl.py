"""CUDA path (through the C ABI) against the CPU oracle on the 512-icosphere
bowl at full size (subdivision-2 icospheres dropped into a static bowl,
83,281 vertices), from oracle-written snapshots
(tests/golden/bowl_snapshots.npz, written by make_bowl_snapshots.py from the
oracle alone: the initial state and step 1, the first contacts): at each
snapshot the candidate and active pair sets with
their distance types bit-exact, the incremental potential's energies and
gradient to 1e-10, and one time step from the snapshot within 1e-8 of the
box diagonal of the oracle's step at the oracle's Newton tolerance (Sec. 4,
Sec. 4.1, Sec. 4.3)."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2201_10022_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))
SNAP = np.load(os.path.join(HERE, "golden", "bowl_snapshots.npz"))
STEPS = [int(k) for k in SNAP["steps"]]


@pytest.fixture(scope="module")
def abd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_10022_gb300 import abd as A
    A.load()
    return A


@pytest.fixture(scope="module")
def bowl():
    s = scenes.ico_bowl(seed=2)
    return s, O.Oracle(s, newton_max=300)


@pytest.mark.parametrize("step", STEPS)
def test_bowl_snapshot_system_and_step(abd, bowl, step):
    s, orc = bowl
    q0, qd0, q1 = SNAP[f"q_{step}"], SNAP[f"qdot_{step}"], SNAP[f"q1_{step}"]
    assert abs(orc.l_bbox - float(SNAP["l_bbox"])) <= 1e-12 * orc.l_bbox
    orc.set_state(q0, qd0)
    gpu = abd.AbdScene(s, newton_tol=orc.newton_tol)
    gpu.set_state(q0, qd0)
    E, g, cnt = gpu.energy_grad_hess(torch.tensor(q0))
    st, Eo, go = orc.energy_grad_hess(q0.reshape(-1))
    assert st == 0
    for which in (0, 1):
        pg, po = gpu.pairs(which), orc.pairs(which)
        sg = set(zip(pg["kind"].tolist(), pg["i"].tolist(), pg["j"].tolist(),
                     (pg["type"] if which else 0 * pg["kind"]).tolist()))
        so = set(zip(po["kind"].tolist(), po["i"].tolist(), po["j"].tolist(),
                     (po["type"] if which else 0 * po["kind"]).tolist()))
        assert sg == so, (which, len(sg), len(so))
    assert int(SNAP[f"active_{step}"]) > 0  # contact within the step
    np.testing.assert_allclose(E, Eo, rtol=1e-10, atol=1e-12)
    gg = g.cpu().numpy()
    assert np.abs(gg - go).max() <= 1e-10 * np.abs(go).max()
    gpu.set_state(q0, qd0)
    gpu.step(1)
    qg, _ = gpu.get_state()
    xg = orc.vertices(qg.cpu().numpy().reshape(-1))
    xo = orc.vertices(q1.reshape(-1))
    assert np.abs(xg - xo).max() <= 1e-8 * orc.l_bbox, (np.abs(xg - xo).max(), orc.l_bbox)
