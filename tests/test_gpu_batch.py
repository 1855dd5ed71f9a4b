"""Many-scene form (abd_step_batch, SceneBatch): every scene of a batch is
bit-identical to the same scene stepped alone, whatever the worker count and
grid divisor; the autotuner restores the state it tunes from; and a batched
scene stays on the oracle's trajectory."""
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


def _small_batch(n=6):
    # a 1.2 m pitch would keep these apart for a long time: pack them so that
    # contacts form within the few steps run here
    return scenes.scene_batch(n_scenes=n, nmin=8, nmax=48, vel_sigma=2.0)


def _alone(abd, S, nsteps, **kw):
    out = []
    for s in S:
        g = abd.AbdScene(s, **kw)
        g.step(nsteps)
        out.append(tuple(t.clone() for t in g.get_state()))
        g.close()
    return out


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_scenes_bit_identical_to_alone(abd, precision):
    from paper_2201_10022_gb300.batch import SceneBatch
    S = _small_batch()
    nsteps = 6
    ref = _alone(abd, S, nsteps, precision=precision)
    for nw, gd in ((3, 4), (6, 1), (1, 16), (4, "by_size")):
        B = SceneBatch(S, precision=precision)
        B.nworkers = nw
        B.set_grid_policy(gd)
        stats = B.step(nsteps)
        assert sum(st["n_active"] for st in stats) >= 0
        for k, (q, qd) in enumerate(B.get_states()):
            assert torch.equal(q, ref[k][0]) and torch.equal(qd, ref[k][1]), (nw, gd, k)
        B.close()


def test_contacts_form_in_the_small_batch(abd):
    from paper_2201_10022_gb300.batch import SceneBatch
    B = SceneBatch(_small_batch())
    stats = B.step(6)
    assert max(st["n_active"] for st in stats) > 0
    B.close()


def test_tune_restores_state_and_caches(abd, tmp_path, monkeypatch):
    from paper_2201_10022_gb300.batch import SceneBatch
    monkeypatch.setenv("ABD_TUNE_CACHE", str(tmp_path / "tune.json"))
    B = SceneBatch(_small_batch(4))
    B.step(2)
    before = [(q.clone(), qd.clone()) for q, qd in B.get_states()]
    res = B.tune(trial_steps=1)
    assert not res["cached"] and res["grid_div"] in ("by_size", 1, 4, 16) and res["nworkers"] >= 1
    for (q0, qd0), (q1, qd1) in zip(before, B.get_states()):
        assert torch.equal(q0, q1) and torch.equal(qd0, qd1)
    again = B.tune()
    assert again["cached"] and again["grid_div"] == res["grid_div"]
    B.close()


def test_batched_scene_follows_the_oracle(abd):
    from paper_2201_10022_gb300.batch import SceneBatch
    S = scenes.scene_batch(n_scenes=3, nmin=8, nmax=16, vel_sigma=2.0, types=("cube",))
    orcs = [O.Oracle(s, newton_max=500) for s in S]
    B = SceneBatch(S, params_list=[{"newton_tol": o.newton_tol} for o in orcs])
    active = 0
    for _ in range(10):
        B.step(1)
        for o, g, s in zip(orcs, B.scenes, S):
            r, st = o.step(1)
            assert r == 0, O.ERRORS[r]
            active += st["n_active"]
            qo, _ = o.get_state()
            xo = o.vertices(qo.reshape(-1))
            xg = o.vertices(g.get_state()[0].cpu().numpy().reshape(-1))
            assert np.abs(xg - xo).max() <= 1e-8 * o.l_bbox
    assert active > 0
    B.close()
