"""Run the contact path of one synthetic scene a bounded number of times on
cuda:0 (for profilers: a small, self-terminating case).

    python -m paper_2201_10022_gb300.profile_case packed 10 10 10 --evals 2
    python -m paper_2201_10022_gb300.profile_case lattice 25 20 20 --steps 3

`packed` evaluates energy, gradient and Hessian of a contact-dense block of
cubes (every face pair within d-hat); `lattice` advances the lattice pile.
"""
import argparse

import torch

from . import scenes
from .abd import AbdScene


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("scene", choices=["packed", "lattice"])
    ap.add_argument("dims", type=int, nargs=3)
    ap.add_argument("--evals", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0)
    ap.add_argument("--prof", action="store_true", help="print per-slot kernel times (CUDA events)")
    a = ap.parse_args()
    nx, ny, nz = a.dims
    s = scenes.packed_cubes(nx=nx, ny=ny, nz=nz) if a.scene == "packed" else scenes.lattice_pile(nx=nx, ny=ny, nz=nz)
    g = AbdScene(s)
    q = torch.tensor(s.q0)
    E, grad, cnt = g.energy_grad_hess(q)  # warm-up (buffer growth)
    if a.prof:
        g.set_profiling(True)
    for _ in range(a.evals):
        E, grad, cnt = g.energy_grad_hess(q)
    if a.steps:
        g.step(a.steps)
    torch.cuda.synchronize()
    out = {"bodies": s.nb, "active": cnt["n_active"], "candidates": cnt["n_candidates"], "energy": float(E[0])}
    if a.prof:
        out["kernels"] = {k: {"launches": v["launches"], "ms": round(v["total_ms"], 4),
                              "tflops": round(v["flops"] / (v["total_ms"] * 1e-3) / 1e12, 4) if v["total_ms"] > 0 and v["flops"] else None}
                          for k, v in g.profile().items() if v["launches"]}
        out["counters"] = g.counters()
    print(out)


if __name__ == "__main__":
    main()
