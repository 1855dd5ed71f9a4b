"""Write oracle_regression.json: the oracle's energy, gradient and one-step
state for a small two-body contact scene (a regression fixture; calls only
the oracle and the scene generator)."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2201_10022_gb300 import scenes  # noqa: E402


def scene():
    s = scenes.random_pair(3, kinds=("cube", "ico1"), sep=0.0004)
    s.qdot0[1, :3] = [0.0, 0.0, -0.3]
    return s


def compute():
    s = scene()
    o = O.Oracle(s)
    st, E, g = o.energy_grad_hess(s.q0.reshape(-1))
    assert st == 0
    n_active = int(o.pairs(1)["kind"].size)
    o.set_state(s.q0, s.qdot0)
    r, stats = o.step(1)
    assert r == 0
    q, qd = o.get_state()
    return {"energy": [float(e) for e in E], "gradient": [float(x) for x in g.reshape(-1)],
            "q1": [float(x) for x in q.reshape(-1)], "qdot1": [float(x) for x in qd.reshape(-1)],
            "n_active": n_active}


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as f:
        json.dump(compute(), f, indent=1)
