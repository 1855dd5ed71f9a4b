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
    a = ap.parse_args()
    nx, ny, nz = a.dims
    s = scenes.packed_cubes(nx=nx, ny=ny, nz=nz) if a.scene == "packed" else scenes.lattice_pile(nx=nx, ny=ny, nz=nz)
    g = AbdScene(s)
    q = torch.tensor(s.q0)
    for _ in range(a.evals):
        E, grad, cnt = g.energy_grad_hess(q)
    if a.steps:
        g.step(a.steps)
    torch.cuda.synchronize()
    print({"bodies": s.nb, "active": cnt["n_active"], "candidates": cnt["n_candidates"], "energy": float(E[0])})


if __name__ == "__main__":
    main()
