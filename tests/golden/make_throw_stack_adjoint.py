"""Write throw_stack_adjoint.npz: the throw-into-stack adjoint workload (64
cubes thrown at a 10-cube stack, 74 dynamic bodies, FP64, mu = 0) over a
20-step horizon, forward and backward by the oracle alone.

Forward: 20 oracle steps from the scene's initial state (at most 300 Newton
iterations a step, the oracle's own tolerance, dense direct solves).
Backward: the implicit-function adjoint of every step (Sec. 6: the step is
differentiable through its optimality condition), chained from the last step
to the first for the loss |mean translation of the dynamic bodies - TARGET|^2
on the final state.  For every step t the file keeps the adjoint's inputs
(dL/dq^{t+1}, dL/dqdot^{t+1}) and outputs (dL/dq^t, dL/dqdot^t, the step's
dL/dkappa), so the GPU test compares step by step from the same inputs, and
the smallest, smallest-magnitude and largest eigenvalue of the step's
unprojected Hessian (numpy, on the oracle's dense matrix).

Calls only the oracle and the scene generator."""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2201_10022_gb300 import scenes  # noqa: E402

SEED = 4
NSTEPS = 20
NEWTON_MAX = 300
TARGET = np.array([-0.5, 0.0, 0.25])


def scene():
    return scenes.throw_stack(seed=SEED)


def compute(verbose=True):
    s = scene()
    dyn = s.is_static == 0
    dt = s.params["dt"]
    o = O.Oracle(s, newton_max=NEWTON_MAX, dense_max_dof=12 * s.nb)
    o.set_state(s.q0, s.qdot0)
    q = [s.q0.copy()]
    qd = [s.qdot0.copy()]
    npairs = [0]
    t0 = time.time()
    for t in range(NSTEPS):
        r, _ = o.step(1)
        assert r == 0, (t, O.ERRORS[r])
        a, b = o.get_state()
        q.append(a.copy())
        qd.append(b.copy())
        npairs.append(int(o.pairs(1)["kind"].size))
        if verbose:
            print(f"forward step {t + 1}: {npairs[-1]} active pairs, {time.time() - t0:.0f} s", flush=True)
    # extreme eigenvalues of each step's unprojected Hessian over the dynamic
    # bodies' DOFs at the converged state (a negative minimum: a stationary
    # point that is not a minimiser, solved by the adjoint's LDL^T)
    idx = np.concatenate([np.arange(12 * b, 12 * b + 12) for b in np.nonzero(dyn)[0]])
    eig = []
    for t in range(NSTEPS):
        o.set_state(q[t], qd[t])
        st, _, _ = o.energy_grad_hess(q[t + 1].reshape(-1), project=False)
        assert st == 0
        ev = np.linalg.eigvalsh(o.dense_hessian()[np.ix_(idx, idx)])
        eig.append((ev.min(), np.abs(ev).min(), ev.max()))
    gq = np.zeros_like(s.q0)
    gq[dyn, :3] = 2.0 * (q[-1][dyn, :3].mean(axis=0) - TARGET) / dyn.sum()
    gqd = np.zeros_like(s.q0)
    gq_in, gqd_in, gq_out, gqd_out, gk_out = [], [], [], [], []
    for t in range(NSTEPS - 1, -1, -1):
        gq_in.append(gq.copy())
        gqd_in.append(gqd.copy())
        st, Mlam, gk = o.adjoint_step(q[t], qd[t], q[t + 1], gq + gqd / dt)
        assert st == 0, (t, O.ERRORS[st])
        gq, gqd = Mlam - gqd / dt, dt * Mlam
        gq[~dyn] = 0.0
        gqd[~dyn] = 0.0
        gq_out.append(gq.copy())
        gqd_out.append(gqd.copy())
        gk_out.append(gk.copy())
        if verbose:
            print(f"adjoint step {t}: {time.time() - t0:.0f} s", flush=True)
    rev = lambda a: np.array(a[::-1])  # noqa: E731  (index by step t)
    return {"seed": np.array(SEED), "target": TARGET, "q": np.array(q), "qdot": np.array(qd),
            "n_active": np.array(npairs), "hess_eig": np.array(eig), "gq_in": rev(gq_in), "gqd_in": rev(gqd_in),
            "gq_out": rev(gq_out), "gqd_out": rev(gqd_out), "gk_out": rev(gk_out)}


if __name__ == "__main__":
    out = compute()
    np.savez_compressed(os.path.join(HERE, "throw_stack_adjoint.npz"), **out)
