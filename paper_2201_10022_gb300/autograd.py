"""Differentiable multi-step rollout of a scene (implicit-function adjoint).

``Rollout.apply(scene, nsteps, q0, qdot0, kappa_body)`` advances ``scene``
(an :class:`~paper_2201_10022_gb300.abd.AbdScene`) ``nsteps`` time steps from
``(q0, qdot0)`` and returns the end state ``(q, qdot)``.  The state of every
step is checkpointed on the device; the backward pass walks the steps in
reverse through ``abd_adjoint_step`` (the unprojected Hessian of each step's
incremental potential at its end state, a PCG solve and the chain through
q~ = q + dt qdot + dt^2 g and qdot_next = (q_next - q) / dt), and returns the
gradients with respect to ``q0``, ``qdot0`` and the per-body orthogonality
stiffness ``kappa_body``.  The lagged friction quantities of each step are
held fixed.  ``kappa_body`` must hold the scene's values (the scene is built
with them); it is an input only so that its gradient can be returned.  The
adjoint solves run to ``scene.adjoint_rel_tol`` (default 1e-12) within the
scene's PCG iteration cap.
"""
from __future__ import annotations

import numpy as np
import torch


class Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, scene, nsteps, q0, qdot0, kappa_body):
        kb = np.asarray(scene.scene.kappa_body, dtype=np.float64)
        if not np.array_equal(kappa_body.detach().cpu().numpy(), kb):
            raise ValueError("kappa_body must equal the scene's per-body stiffness")
        scene.set_state(q0.detach(), qdot0.detach())
        qs = [q0.detach().to(scene.device, torch.float64).clone()]
        qds = [qdot0.detach().to(scene.device, torch.float64).clone()]
        for _ in range(int(nsteps)):
            scene.step(1)
            q, qd = scene.get_state()
            qs.append(q.clone())
            qds.append(qd.clone())
        ctx.scene = scene
        ctx.save_for_backward(torch.stack(qs), torch.stack(qds))
        return qs[-1].clone(), qds[-1].clone()

    @staticmethod
    def backward(ctx, gq_out, gqd_out):
        scene = ctx.scene
        qs, qds = ctx.saved_tensors
        dev = scene.device
        gq = (gq_out if gq_out is not None else torch.zeros_like(qs[0])).to(dev, torch.float64).contiguous().clone()
        gqd = (gqd_out if gqd_out is not None else torch.zeros_like(qs[0])).to(dev, torch.float64).contiguous().clone()
        gk = torch.zeros(scene.nb, dtype=torch.float64, device=dev)
        rel_tol = getattr(scene, "adjoint_rel_tol", 1e-12)
        for t in range(qs.shape[0] - 2, -1, -1):
            scene.adjoint_step(qs[t], qds[t], qs[t + 1], gq, gqd, gk, rel_tol=rel_tol)
        return None, None, gq, gqd, gk
