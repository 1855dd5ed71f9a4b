#!/usr/bin/env python
"""Benchmark of the affine-body time step on GB300.

Metric: milliseconds per time step of the 10,001-body lattice pile (25x20x20
jittered lattice of cubes, subdivision-1 icospheres and 1x0.2x0.2 m boxes
collapsing onto a static ground, friction mu = 0.3, FP64), with contact-pair
evaluations per second beside it.  The pile's first steps are free fall; the
timed window starts `--start-step` steps into the run (advanced untimed on
the GPU), after `--warmup` further untimed steps, and covers `--steps` steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl abd|reference]

Prints one JSON line.  Under torchrun (N > 1) every rank steps its own
replica of the scene; rank 0 prints the line with the maximum time over
ranks.  The reference arm times the CPU oracle on a bounded sample of the
same workload (see `cpu_baseline`).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2201_10022_gb300 import scenes  # noqa: E402

WORKLOAD = dict(name="lattice_pile", nx=25, ny=20, nz=20, seed=3)
METRIC = "ms/timestep, 10k-body lattice pile (FP64, friction)"


def workload_scene(nx=None, ny=None, nz=None):
    return scenes.lattice_pile(seed=WORKLOAD["seed"], nx=nx or WORKLOAD["nx"], ny=ny or WORKLOAD["ny"],
                               nz=nz or WORKLOAD["nz"])


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.rows, self.proc, self.uuid = [], None, uuid

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ---------------------------------------------------------------------------
# CPU oracle: bounded sample of the same workload
# ---------------------------------------------------------------------------
def oracle_sample(start_step, warmup, steps, dims=(6, 6, 3)):
    """Time the CPU oracle on a sub-lattice of the workload's recipe over the
    same step window; ms/step is scaled to the full body count."""
    import oracle as O
    s = workload_scene(*dims)
    full = workload_scene()
    # the library's Newton rule: |dx|_inf <= 1e-5 * bbox diagonal * dt
    o = O.Oracle(s, newton_rel=1e-5 * s.params["dt"], newton_max=500, cg_tol=1e-4)
    r, _ = o.step(start_step + warmup)
    if r:
        raise RuntimeError(f"oracle failed while advancing: {O.ERRORS[r]}")
    steps = min(steps, 5)
    t0 = time.perf_counter()
    r, st = o.step(steps)
    dt = time.perf_counter() - t0
    if r:
        raise RuntimeError(f"oracle failed: {O.ERRORS[r]}")
    scale = full.nb / s.nb
    return {"value": 1e3 * dt / steps * scale, "unit": "ms/step", "cores": 1, "kind": "oracle",
            "sample": (f"oracle (1 thread) on a {dims[0]}x{dims[1]}x{dims[2]} sub-lattice ({s.nb} bodies) of the "
                       f"same recipe, steps {start_step + warmup}..{start_step + warmup + steps - 1}, "
                       f"{1e3 * dt / steps:.1f} ms/step scaled by bodies x{scale:.1f}"),
            "seconds": dt}


_T0 = time.perf_counter()

# DRAM bytes (read + write) of one k_barrier launch on this workload, from one
# full ncu capture of the kernel as it stands (a Newton iteration near step
# 20 of the lattice pile: 139,264 B read, 0 B written; the terms' inputs and
# outputs stay in the 129 MB L2).  Re-capture when the kernel changes.
BARRIER_DRAM_BYTES = 139264


def log(msg):
    """progress on stderr (the JSON line goes to stdout)"""
    print(f"[bench {time.perf_counter() - _T0:7.1f}s] {msg}", file=sys.stderr, flush=True)


def max_over_ranks(x, world, device):
    """the largest value of x over the ranks of the job (the slowest rank's
    time); x itself on a single rank"""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def aggregate_ms_per_step(total_ms, steps, world):
    """replicas: every rank steps its own copy of the scene, so the job
    advances steps * world scene-steps in the slowest rank's time"""
    return total_ms / (steps * world)


def vertices(s, q):
    """world vertex positions x = A xbar + p for body states q (nb, 12)"""
    q = np.asarray(q).reshape(-1, 12)
    A = q[s.vbody, 3:].reshape(-1, 3, 3)
    return np.einsum("vij,vj->vi", A, s.xbar) + q[s.vbody, :3]


def bbox_diag(x):
    return float(np.linalg.norm(x.max(axis=0) - x.min(axis=0)))


def adjoint_run(dev, nsteps=100, seed=4, budget_s=120.0):
    """Throw into a stack (64 thrown cubes, 10-cube stack, FP64): forward and
    implicit-function backward through nsteps steps; loss = squared distance
    of the thrown cubes' mean final translation to a seeded target; gradients
    with respect to their initial velocities and the per-body kappa.  Every
    linear solve (Newton steps and adjoint) is the dense direct solve (900
    DOFs; the stack's chain of stiff contacts stalls the block-Jacobi PCG);
    Newton stops at 1e-9 of the dynamic bodies' box diagonal, so the forward
    map is smooth enough for central differences with h = 1e-6, which check
    two velocity components while the run stays within budget_s."""
    import torch
    from paper_2201_10022_gb300 import scenes
    from paper_2201_10022_gb300.abd import AbdError, AbdScene
    from paper_2201_10022_gb300.autograd import Rollout

    s = scenes.throw_stack(seed=seed)
    thrown = np.arange(s.nb - 64, s.nb)
    target = np.random.default_rng(seed).uniform([-1.0, -0.5, 0.0], [0.0, 0.5, 0.5])
    dyn_v = s.is_static[s.vbody] == 0
    L = bbox_diag(vertices(s, s.q0)[dyn_v])
    g = AbdScene(s, device=dev, dense_max_dofs=3072, newton_tol=1e-9 * L)
    tgt = torch.tensor(target, device=dev)
    idx = torch.tensor(thrown, device=dev)
    out = {"workload": f"throw_stack seed {seed}: 64 thrown + 10 stacked 0.2 m cubes, {nsteps} steps, FP64, mu 0, "
                       f"dense direct solves, Newton tol 1e-9 L_bbox"}

    def loss_of(qK):
        return ((qK[idx, :3].mean(dim=0) - tgt) ** 2).sum()

    t_start = time.perf_counter()
    try:
        q0 = torch.tensor(s.q0, device=dev, requires_grad=True)
        qd0 = torch.tensor(s.qdot0, device=dev, requires_grad=True)
        kb = torch.tensor(s.kappa_body, device=dev, requires_grad=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        qK, _ = Rollout.apply(g, nsteps, q0, qd0, kb)
        loss = loss_of(qK)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        loss.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
    except AbdError as e:
        out["error"] = str(e)
        g.close()
        return out
    gv = qd0.grad[idx, :3].cpu().numpy()
    log(f"adjoint: forward {t1 - t0:.1f} s, backward {t2 - t1:.1f} s")
    out.update({"forward_ms_per_step": 1e3 * (t1 - t0) / nsteps, "backward_ms_per_step": 1e3 * (t2 - t1) / nsteps,
                "loss": loss.item(), "grad_v0_norm": float(np.linalg.norm(gv)),
                "grad_kappa_norm": float(kb.grad.norm().item())})
    checks = []
    h = 1e-6

    def fd_check(T, b, k, adj):
        vals = []
        for sgn in (1.0, -1.0):
            qd = s.qdot0.copy()
            qd[b, k] += sgn * h
            g.set_state(torch.tensor(s.q0), torch.tensor(qd))
            g.step(T)
            vals.append(loss_of(g.get_state()[0]).item())
        fd = (vals[0] - vals[1]) / (2 * h)
        return {"horizon": T, "body": b, "component": k, "adjoint": adj, "central_difference": fd,
                "rel_mismatch": abs(adj - fd) / max(abs(fd), 1e-300)}

    # a short horizon first (the thrown block in flight, its cubes touching
    # one another, the stack settling): the loss is a smooth function of the
    # initial velocities there; then the full horizon, whose 64-body
    # collisions make the loss chaotic (the central difference and the
    # adjoint derivative need not agree at any practical h; reported)
    T = 20
    q0s = torch.tensor(s.q0, device=dev, requires_grad=True)
    qd0s = torch.tensor(s.qdot0, device=dev, requires_grad=True)
    kbs = torch.tensor(s.kappa_body, device=dev, requires_grad=True)
    qKs, _ = Rollout.apply(g, T, q0s, qd0s, kbs)
    loss_of(qKs).backward()
    for b, k in ((int(thrown[0]), 0), (int(thrown[-1]), 2)):
        if time.perf_counter() - t_start > budget_s:
            break
        checks.append(fd_check(T, b, k, float(qd0s.grad[b, k].item())))
    for b, k in ((int(thrown[0]), 0),):
        if time.perf_counter() - t_start > budget_s:
            break
        checks.append(fd_check(nsteps, b, k, float(qd0.grad[b, k].item())))
    out["fd_checks"] = checks
    g.close()
    return out


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def batched_run(dev, steps=2, pre_steps=10, seed=5, n_scenes=256):
    """Many independent scenes (log-uniform 16..2048 bodies of 0.2 m cubes and
    radius-0.1 m icosphere-2s per scene, lattice-pile layouts, seeded
    velocities, frictionless), advanced pre_steps steps, then timed over
    `steps` steps from one saved state three ways: the plain FP64 path one
    scene after another (one host worker, full-device grids); the FP64 batch
    (autotuned workers and grid divisor: bit-identical results); and the
    mixed-precision batch.  Wall-clock around each batch call, which returns
    once every scene's stream has drained."""
    import torch
    from paper_2201_10022_gb300 import scenes
    from paper_2201_10022_gb300.abd import AbdError
    from paper_2201_10022_gb300.batch import SceneBatch

    t0 = time.perf_counter()
    S = scenes.scene_batch(seed=seed, n_scenes=n_scenes)
    nb = np.array([s.nb - 1 for s in S])
    B = SceneBatch(S, device=dev)
    log(f"batch: {n_scenes} scenes created ({int(nb.sum())} bodies)")
    B.step(pre_steps)
    log(f"batch: {pre_steps} pre-steps done")
    saved = [(q.clone(), qd.clone()) for q, qd in B.get_states()]
    setup_s = time.perf_counter() - t0

    def timed(batch, warm=True):
        batch.set_states(saved)
        if warm:  # capture of the launch sequences at this shape
            batch.step(1)
            batch.set_states(saved)
        return batch.time_steps(steps)

    # the plain path one scene after another at full-device grids (the
    # pre-steps captured its launch sequences)
    B.nworkers = 1
    B.set_grid_policy(1)
    ms_seq, st_seq = timed(B, warm=False)
    log(f"batch: sequential {ms_seq / steps:.1f} ms/step")
    tune = B.tune(trial_steps=1, use_cache=False, write_cache=False, log=log)
    ms_b, st_b = timed(B)
    log(f"batch: batched {ms_b / steps:.1f} ms/step")
    q_b = [q.clone() for q, _ in B.get_states()]
    B.close()
    mixed = None
    try:
        Bm = SceneBatch(S, device=dev, precision=1)
        Bm.nworkers = tune["nworkers"]
        Bm.set_grid_policy(tune["grid_div"])  # the FP64 batch's launch shape
        ms_m, st_m = timed(Bm)
        dev_max = 0.0
        for s, qb, (qm, _) in zip(S, q_b, Bm.get_states()):
            x0 = vertices(s, qb.cpu().numpy())
            dev_max = max(dev_max, float(np.abs(vertices(s, qm.cpu().numpy()) - x0).max() / bbox_diag(x0)))
        mixed = {"ms_per_step": ms_m / steps, "max_vertex_deviation_vs_fp64_over_scene_lbbox": dev_max}
        Bm.close()
    except AbdError as e:
        mixed = {"error": str(e)}
    log("batch: mixed done")
    newton = sum(st["newton_iters"] for st in st_b)
    return {
        "workload": f"{n_scenes} scenes seed {seed}: {int(nb.sum())} bodies (per scene {int(nb.min())}..{int(nb.max())}, "
                    f"median {int(np.median(nb))}), {sum(s.nv for s in S)} vertices, steps {pre_steps + 1}.."
                    f"{pre_steps + steps} timed, mu 0",
        "steps": steps,
        "sequential_fp64_ms_per_step": ms_seq / steps,
        "batched_fp64_ms_per_step": ms_b / steps,
        "batched_mixed": mixed,
        "speedup_batched_fp64_vs_sequential": ms_seq / ms_b,
        "scene_steps_per_s_batched_fp64": n_scenes * steps / (ms_b * 1e-3),
        "newton_iters_per_s_batched_fp64": newton / (ms_b * 1e-3),
        "newton_iters_per_scene_step": newton / (n_scenes * steps),
        "pcg_iters_per_newton": sum(st["pcg_iters"] for st in st_b) / max(newton, 1),
        "tuning": {"nworkers": tune["nworkers"], "grid_div": tune["grid_div"],
                   "trials": [(t["nworkers"], t["grid_div"], round(t["ms"], 1)) for t in tune["trials"]]},
        "gpu_launches": sum(st["kernel_launches"] for st in st_b),
        "setup_s": setup_s,
        "timing": "wall clock around abd_step_batch (returns after every scene's stream drained)",
    }


def run_abd(args, rank, world):
    import torch
    from paper_2201_10022_gb300.abd import AbdScene, abd_get_state, abd_set_state, abd_step, abd_step_stats
    import ctypes as C

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    s = workload_scene()
    g = AbdScene(s, device=dev)
    if args.start_step:
        g.step(args.start_step)
    log(f"workload: {args.start_step} pre-roll steps done")
    g.step(args.warmup)
    torch.cuda.synchronize()
    q0, qd0 = g.get_state()
    q0, qd0 = q0.clone(), qd0.clone()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2

    # ---- device-timed region: inputs resident in HBM ----------------------
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = None
    clk = ClockSampler(uuid)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk.start()
    torch.cuda.nvtx.range_push("timed")
    ms, stats = [], []
    for k in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st = g.step(1)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        stats.append(st)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = clk.stop()

    # ---- per-kernel-class device times: the same steps again from the same
    # state with the library's event profiling on (kept out of the timed run)
    g.set_state(q0, qd0)
    g.set_profiling(True)
    for k in range(args.steps):
        flush.zero_()
        g.step(1)
    torch.cuda.synchronize()
    prof = g.profile()
    g.set_profiling(False)
    cnt = g.counters()
    total_ms = max_over_ranks(sum(ms), world, dev)

    # ---- end to end through the C ABI with host buffers -------------------
    qh = torch.empty((s.nb, 12), dtype=torch.float64).pin_memory()
    qdh = torch.empty_like(qh).pin_memory()
    qh.copy_(q0.cpu())
    qdh.copy_(qd0.cpu())
    torch.cuda.synchronize()
    sst = abd_step_stats()
    t0 = time.perf_counter()
    for k in range(args.steps):
        r = abd_set_state(g.h, qh.data_ptr(), qdh.data_ptr(), 0)
        r = r or abd_step(g.h, 1, C.byref(sst))
        r = r or abd_get_state(g.h, qh.data_ptr(), qdh.data_ptr(), 0)
        if r:
            raise RuntimeError(f"e2e step failed: {r}")
    e2e_ms = max_over_ranks(1e3 * (time.perf_counter() - t0), world, dev)

    # ---- mixed precision (precision = 1): the same steps from the same state;
    # the end state is compared with the FP64 run's (the e2e pass above)
    mixed = None
    if not args.no_mixed:
        gm = AbdScene(s, device=dev, precision=1)
        gm.set_state(q0, qd0)
        gm.step(1)  # buffer growth outside the timed steps
        gm.set_state(q0, qd0)
        torch.cuda.synchronize()
        ms_m, st_m = [], []
        for k in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st_m.append(gm.step(1))
            e1.record()
            torch.cuda.synchronize()
            ms_m.append(e0.elapsed_time(e1))
        qm, _ = gm.get_state()
        xm = vertices(s, qm.cpu().numpy())
        x64 = vertices(s, qh.numpy())
        L = bbox_diag(vertices(s, q0.cpu().numpy()))
        mixed = {"value": sum(ms_m) / len(ms_m), "unit": "ms/step",
                 "newton_iters_per_step": sum(st["newton_iters"] for st in st_m) / len(st_m),
                 "max_vertex_deviation_vs_fp64_over_lbbox": float(np.abs(xm - x64).max() / L),
                 "precision": "FP32 eigenbasis for the barrier Hessian projection; distances, barrier, "
                              "energies, gradients, CCD, Newton test and line search FP64"}
        gm.close()

    log("timed, profiled, e2e and mixed runs done")
    # the adjoint and the many-scene batch are single-GPU figures: under
    # torchrun (N > 1) the replicas time the headline step only
    adjoint = None
    if not args.no_adjoint and world == 1:
        try:
            adjoint = adjoint_run(dev)
        except Exception as e:  # reported in the line, not fatal to the headline measurement
            adjoint = {"error": f"{type(e).__name__}: {e}"}
    batched = None
    if not args.no_batched and world == 1:
        try:
            batched = batched_run(dev)
        except Exception as e:  # reported in the line, not fatal to the headline measurement
            batched = {"error": f"{type(e).__name__}: {e}"}
    log("batched run done")

    steps_total = args.steps * world
    ms_per_step = aggregate_ms_per_step(total_ms, args.steps, world)
    newton = sum(st["newton_iters"] for st in stats)
    cand = sum(st["candidates_tested"] for st in stats)
    act = sum(st["active_evaluated"] for st in stats)
    launches = sum(st["kernel_launches"] for st in stats)
    pk, src = peaks()
    # roofline of the kernel class with an algorithmic flop or byte model
    # that took the most device time
    modelled = [kv for kv in prof.items() if kv[1]["flops"] > 0 or kv[1]["bytes"] > 0]
    roof = None
    name, p = max(modelled or prof.items(), key=lambda kv: kv[1]["total_ms"])
    if p["launches"] and p["total_ms"] > 0:
        t_s = p["total_ms"] * 1e-3
        if p["flops"] > 0:
            # FP64 SIMT peak: 152 SMs x 2 FP64 FMA/clk x 2 flop x clock
            clk = (clocks.get("sm_mhz") or 2070.0) * 1e6
            peak = 152 * 2 * 2 * clk / 1e12
            achieved = p["flops"] / t_s / 1e12
            roof = {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": BARRIER_DRAM_BYTES if name == "barrier_terms" else None,
                    "peak_source": "derived (FP64 FMA units x clock)",
                    "launches": p["launches"], "avg_launch_ms": p["total_ms"] / p["launches"]}
        elif p["bytes"] > 0:
            achieved = p["bytes"] / t_s / 1e9
            roof = {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / pk["hbm_gbs"], "traffic": None, "peak_source": src,
                    "launches": p["launches"], "avg_launch_ms": p["total_ms"] / p["launches"]}
    out = {
        "metric": METRIC, "value": ms_per_step, "unit": "ms/step", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"lattice_pile {WORKLOAD['nx']}x{WORKLOAD['ny']}x{WORKLOAD['nz']} seed "
                               f"{WORKLOAD['seed']}, {s.nb} bodies ({s.nv} vertices, {s.nt} triangles, {s.ne} edges), "
                               f"mu 0.3, kappa 1e8, dt 0.01, dhat 1e-3",
                   "timed_steps": f"{args.start_step + args.warmup}..{args.start_step + args.warmup + args.steps - 1}",
                   "l2": "256 MB buffer written between timed steps",
                   "newton_tol": "1e-5 * bbox diagonal * dt", "pcg_rel_tol": 1e-4, "parallelism": f"replicas x{world}"},
        "steps_per_s": 1e3 / ms_per_step,
        "newton_iters_per_s": newton / (total_ms * 1e-3),
        "contact_evals_per_s": cand / (total_ms * 1e-3),
        "active_evals_per_s": act / (total_ms * 1e-3),
        "newton_iters_per_step": newton / args.steps,
        "pcg_iters_per_newton": sum(st["pcg_iters"] for st in stats) / max(newton, 1),
        "e2e": {"value": e2e_ms / steps_total, "unit": "ms/step", "h2d_bytes_per_step": 2 * 12 * 8 * s.nb,
                "d2h_bytes_per_step": 2 * 12 * 8 * s.nb},
        "gpu_launches": launches,
        "roofline": roof,
        "kernel_ms": {k: round(v["total_ms"], 3) for k, v in prof.items()},
        "barrier_counters": {k: cnt[k] for k in ("barrier_terms", "sweeps_fp32", "sweeps_fp64", "capped_fp64")},
        "culling": {"prim_pairs_of_body_pairs": cnt["prim_pairs_body"],
                    "prim_pairs_after_iaabb": cnt["prim_pairs_iaabb"],
                    "candidates": cnt["prim_pairs_cand"],
                    "iaabb_kept_frac": cnt["prim_pairs_iaabb"] / max(cnt["prim_pairs_body"], 1),
                    "candidates_frac_of_iaabb": cnt["prim_pairs_cand"] / max(cnt["prim_pairs_iaabb"], 1),
                    "scope": "every enumeration since the scene was created (pre-roll, warm-up, timed and "
                             "profiled steps)"},
        "mixed": mixed,
        "adjoint": adjoint,
        "batched": batched,
        "clocks": clocks,
    }
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--start-step", type=int, default=20)
    ap.add_argument("--impl", default="abd", choices=["abd", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision run")
    ap.add_argument("--no-batched", action="store_true", help="skip the 256-scene batch run")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the throw-into-stack adjoint run")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.warmup < 3:
        args.warmup = 3

    if args.impl == "reference":
        if rank != 0:
            return
        cb = oracle_sample(args.start_step, args.warmup, args.steps)
        line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "ms/step", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": cb["value"], "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "same recipe, sub-lattice sample (see cpu_baseline.sample)"},
                "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
                "e2e": {"value": cb["value"], "unit": "ms/step", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    out = run_abd(args, rank, world)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            cb = oracle_sample(args.start_step, args.warmup, args.steps)
            out["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
        else:
            out["cpu_baseline"] = None
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
