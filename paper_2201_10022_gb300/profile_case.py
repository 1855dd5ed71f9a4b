"""Run the contact path of one synthetic scene a bounded number of times on
cuda:0 (for profilers: a small, self-terminating case).

    python -m paper_2201_10022_gb300.profile_case packed 10 10 10 --evals 2
    python -m paper_2201_10022_gb300.profile_case lattice 25 20 20 --steps 3
    python -m paper_2201_10022_gb300.profile_case throw 4 10 0 --steps 20 --dense --newton-rel 1e-9 --prof
    python -m paper_2201_10022_gb300.profile_case packed 22 22 21 --solves 2 --pcg-max 200
    python -m paper_2201_10022_gb300.profile_case lattice 25 20 20 --steps 70 --save-state S.npz
    python -m paper_2201_10022_gb300.profile_case lattice 25 20 20 --load-state S.npz --steps 1 --timed --direct

This module is the profiling entry point of the commands recorded under
profiles/: each run is bounded (a fixed number of evaluations, steps or
linear solves), so a profiler capture of it ends by itself.

--save-state writes (q, qdot) after the steps to an .npz file; --load-state
starts from such a state instead of the scene's initial one (the lattice
pile at step 70 without advancing it under a profiler).  --timed wraps the
steps in an NVTX range "timed" (for ncu --nvtx-include "timed/");
--direct launches every kernel directly (the library's profiling mode: no
CUDA graphs, the line search's rounds from the host), so that a launch list
shows every kernel.

`packed` evaluates energy, gradient and Hessian of a contact-dense block of
cubes (every face pair within d-hat), and with --solves runs that many
linear solves of its Newton system (abd_solve, at most --pcg-max
iterations each, at --precision); `lattice` advances the lattice pile;
`throw` advances the throw-into-stack scene (dims: cubes per side of the
thrown block, stack height, unused).
"""
import argparse

import torch

from . import scenes
from .abd import AbdScene


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("scene", choices=["packed", "lattice", "throw"])
    ap.add_argument("dims", type=int, nargs=3)
    ap.add_argument("--evals", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0)
    ap.add_argument("--prof", action="store_true", help="print per-slot kernel times (CUDA events)")
    ap.add_argument("--dense", action="store_true", help="dense direct solves (dense_max_dofs 3072)")
    ap.add_argument("--solves", type=int, default=0, help="linear solves of the evaluated Newton system")
    ap.add_argument("--pcg-max", type=int, default=200, help="PCG iteration cap of those solves")
    ap.add_argument("--pcg-tol", type=float, default=1e-8, help="PCG relative tolerance of those solves")
    ap.add_argument("--precision", type=int, default=0, help="0 FP64, 1 mixed")
    ap.add_argument("--newton-rel", type=float, default=0.0,
                    help="Newton tolerance relative to the dynamic bodies' box diagonal (0: library default)")
    ap.add_argument("--save-state", default="", help="write (q, qdot) after the steps to this .npz file")
    ap.add_argument("--load-state", default="", help="start from (q, qdot) of this .npz file")
    ap.add_argument("--timed", action="store_true", help='wrap the steps in the NVTX range "timed"')
    ap.add_argument("--direct", action="store_true", help="direct launches (no graphs) during the steps")
    a = ap.parse_args()
    nx, ny, nz = a.dims
    if a.scene == "packed":
        s = scenes.packed_cubes(nx=nx, ny=ny, nz=nz)
    elif a.scene == "lattice":
        s = scenes.lattice_pile(nx=nx, ny=ny, nz=nz)
    else:
        s = scenes.throw_stack(n_throw=nx ** 3, n_stack=ny)
    kw = {"precision": a.precision}
    if a.solves:
        kw.update(pcg_max=a.pcg_max, pcg_rel_tol=a.pcg_tol)
    if a.dense:
        kw["dense_max_dofs"] = 3072
    if a.newton_rel > 0:
        import numpy as np
        q = s.q0
        Am = q[s.vbody, 3:].reshape(-1, 3, 3)
        x = np.einsum("vij,vj->vi", Am, s.xbar) + q[s.vbody, :3]
        x = x[s.is_static[s.vbody] == 0]
        kw["newton_tol"] = a.newton_rel * float(np.linalg.norm(x.max(axis=0) - x.min(axis=0)))
    g = AbdScene(s, **kw)
    if a.load_state:
        import numpy as np
        d = np.load(a.load_state)
        g.set_state(torch.tensor(d["q"]), torch.tensor(d["qdot"]))
    q = g.get_state()[0]
    E, grad, cnt = g.energy_grad_hess(q)  # warm-up (buffer growth)
    if a.prof:
        g.set_profiling(True)
    for _ in range(a.evals):
        E, grad, cnt = g.energy_grad_hess(q)
    solves = []
    for _ in range(a.solves):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        try:
            _, sst = g.solve(-grad)
        except Exception as e:  # the iteration cap is an outcome here, not a failure
            sst = {"error": str(e).split(":")[0]}
        e1.record()
        torch.cuda.synchronize()
        solves.append(dict(sst, ms=round(e0.elapsed_time(e1), 3)))
    st = None
    if a.steps:
        if a.direct:
            g.set_profiling(True)
        torch.cuda.synchronize()
        if a.timed:
            torch.cuda.nvtx.range_push("timed")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st = g.step(a.steps)
        e1.record()
        torch.cuda.synchronize()
        if a.timed:
            torch.cuda.nvtx.range_pop()
        st = dict(st, ms_per_step=e0.elapsed_time(e1) / a.steps)
    if a.save_state:
        import numpy as np
        qs, qds = g.get_state()
        np.savez(a.save_state, q=qs.cpu().numpy(), qdot=qds.cpu().numpy())
    torch.cuda.synchronize()
    out = {"bodies": s.nb, "active": cnt["n_active"], "candidates": cnt["n_candidates"], "energy": float(E[0])}
    if solves:
        out["solves"] = solves
    if st:
        out["steps"] = {k: st[k] for k in ("ms_per_step", "newton_iters", "pcg_iters", "ls_halvings", "n_active",
                                           "kernel_launches")}
    if a.prof:
        out["kernels"] = {k: {"launches": v["launches"], "ms": round(v["total_ms"], 4),
                              "tflops": round(v["flops"] / (v["total_ms"] * 1e-3) / 1e12, 4) if v["total_ms"] > 0 and v["flops"] else None}
                          for k, v in g.profile().items() if v["launches"]}
        out["counters"] = g.counters()
    print(out)


if __name__ == "__main__":
    main()
