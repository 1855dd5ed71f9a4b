"""Write bowl_snapshots.npz: the 512-icosphere bowl (subdivision-2
icospheres of radius 0.05..0.15 m dropped into a static bowl, seed 2,
mu = 0), advanced by the oracle at its own Newton tolerance (1e-9 x the
dynamic bodies' box diagonal) with its block-Jacobi PCG.

Snapshots: the states at steps 0 and 1 (the first contacts: one active
pair after the first step, 22 after the second, which takes the oracle 149
Newton iterations; its global line search reaches the 300-iteration cap on
the third), each with the oracle's state one step later, so the GPU test compares one step from the same state without
running the oracle for it.  Calls only the oracle and the scene
generator."""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2201_10022_gb300 import scenes  # noqa: E402

STEPS = (0, 1)
NEWTON_MAX = 300


def scene():
    return scenes.ico_bowl(seed=2)


def compute(verbose=True):
    s = scene()
    o = O.Oracle(s, newton_max=NEWTON_MAX)
    out = {"steps": np.array(STEPS), "l_bbox": np.array(o.l_bbox)}
    t0 = time.time()
    k = 0
    for target in STEPS:
        while k < target:
            r, st = o.step(1)
            if r:
                raise RuntimeError(f"oracle failed at step {k}: {O.ERRORS[r]}")
            k += 1
            if verbose:
                print(f"step {k} newton {st['newton_iters']} active {st['n_active']} {time.time() - t0:.0f}s",
                      flush=True)
        q, qd = o.get_state()
        out[f"q_{target}"] = q
        out[f"qdot_{target}"] = qd
        r, st = o.step(1)
        if r:
            raise RuntimeError(f"oracle failed at step {k}: {O.ERRORS[r]}")
        out[f"q1_{target}"] = o.get_state()[0]
        out[f"active_{target}"] = np.array(st["n_active"])
        o.set_state(q, qd)
    return out


if __name__ == "__main__":
    data = compute()
    np.savez_compressed(os.path.join(HERE, "bowl_snapshots.npz"), **data)
