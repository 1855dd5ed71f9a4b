"""Write pile_snapshots.npz: states of the lattice-pile recipe on a 6x6x3
sub-lattice (109 bodies, mu = 0.3, the benchmark's recipe at a size the
oracle steps in seconds), advanced by the oracle at its own Newton tolerance
(1e-9 x the dynamic bodies' box diagonal, at most 500 iterations) with a
dense direct solve.

Snapshots (step index -> what the pile is doing there):
  10  free fall, no contact
  16  first ground impacts of the bottom layer
  35  bottom layer on the ground: resting and sliding contacts with friction
  52  second layer landing on the first: body-body contacts and stacking
Calls only the oracle and the scene generator; the GPU tests start both
sides from these states."""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2201_10022_gb300 import scenes  # noqa: E402

DIMS = (6, 6, 3)
NEWTON_MAX = 500   # the landing steps need more than the oracle's default cap of 100
STEPS = (10, 16, 35, 52)


def scene():
    return scenes.lattice_pile(seed=3, nx=DIMS[0], ny=DIMS[1], nz=DIMS[2])


def compute(verbose=True):
    s = scene()
    o = O.Oracle(s, newton_max=NEWTON_MAX)
    out = {"dims": np.array(DIMS), "steps": np.array(STEPS), "l_bbox": np.array(o.l_bbox)}
    t0 = time.time()
    k = 0
    for target in STEPS:
        while k < target:
            r, st = o.step(1)
            if r:
                raise RuntimeError(f"oracle failed at step {k}: {O.ERRORS[r]}")
            k += 1
            if verbose:
                print(f"step {k} newton {st['newton_iters']} active {st['n_active']} "
                      f"friction {st['n_friction']} {time.time() - t0:.0f}s", flush=True)
        q, qd = o.get_state()
        out[f"q_{target}"] = q
        out[f"qdot_{target}"] = qd
    return out


if __name__ == "__main__":
    data = compute()
    np.savez_compressed(os.path.join(HERE, "pile_snapshots.npz"), **data)
