#!/usr/bin/env python
"""Benchmark of the affine-body time step on GB300.

Metric: milliseconds per time step of the 10,001-body lattice pile (25x20x20
jittered lattice of cubes, subdivision-1 icospheres and 1x0.2x0.2 m boxes
collapsing onto a static ground, friction mu = 0.3, FP64), with contact-pair
evaluations per second beside it.  The timed steps lie in windows of the
pile's own trajectory (`--windows`, default first impacts at step 10, ground
contact at 30, the second layer landing at 50): the scene is advanced
untimed on the GPU to each window, `--warmup` further untimed steps, then
its share of the `--steps` timed steps; `value` is the mean over all of
them, and every window is also reported on its own.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--windows a,b,c]
                    [--impl abd|reference]

Prints one JSON line.  Under torchrun (N > 1) every rank steps its own
replica of the scene; rank 0 prints the line with the maximum time over
ranks.  The reference arm times the CPU oracle on the same full pile over
the first steps of the first window (see `cpu_baseline`).
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
def host_cpu():
    """the host's core count and CPU model (the CPU baseline's machine)"""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "model": model}


def oracle_sample(first_step, budget_s=20.0, max_steps=3):
    """Time the CPU oracle (single thread, -O3) on the full workload -- the
    same 10,001-body pile, the library's Newton rule and PCG tolerance, its
    block-Jacobi CG solve -- over the first steps of the first timed window:
    the oracle advances the pile from step 0 to first_step itself (untimed),
    then times whole steps until budget_s has passed or max_steps are done."""
    import oracle as O
    s = workload_scene()
    # the library's Newton rule: |dx|_inf <= 1e-5 * bbox diagonal * dt
    o = O.Oracle(s, newton_rel=1e-5 * s.params["dt"], newton_max=500, cg_tol=1e-4, dense_max_dof=0)
    r, _ = o.step(first_step)
    if r:
        raise RuntimeError(f"oracle failed while advancing: {O.ERRORS[r]}")
    t0 = time.perf_counter()
    n = 0
    while n < max_steps and (n == 0 or time.perf_counter() - t0 < budget_s):
        r, st = o.step(1)
        if r:
            raise RuntimeError(f"oracle failed: {O.ERRORS[r]}")
        n += 1
    dt = time.perf_counter() - t0
    cpu = host_cpu()
    return {"value": 1e3 * dt / n, "unit": "ms/step", "cores": 1, "kind": "oracle",
            "sample": (f"oracle (1 thread, gcc -O3) on the full {s.nb}-body pile, steps {first_step}.."
                       f"{first_step + n - 1} (the first timed window's first steps; the oracle advanced the "
                       f"pile from step 0 itself); host {cpu['nproc']} cores, {cpu['model']}"),
            "seconds": dt, "host": cpu}


_T0 = time.perf_counter()

# DRAM bytes (read + write) of one k_barrier launch on this workload, from one
# full ncu capture of the kernel as it stands (the first Newton iteration of
# step 30 of the lattice pile: 187,136 B read, 0 B written; the terms' inputs
# and outputs stay in the 129 MB L2).  Re-capture when the kernel changes.
BARRIER_DRAM_BYTES = 187136
# DRAM bytes (read + write) per iteration of the PCG solve kernel, from an ncu
# capture (None until captured for the kernel as it stands)
PCG_DRAM_BYTES_PER_ITER = None
# first steps of the default timed windows: first ground impacts of the
# bottom layer, bottom layer on the ground with friction, second layer
# landing, third layer landing
DEFAULT_WINDOWS = "10,30,50,70"


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
        loss.backward(retain_graph=True)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        # the same backward again: the first one also pays one-off costs
        # (first launches of the unprojected path's kernels, buffer growth)
        g_first = qd0.grad.clone()
        qd0.grad = None
        q0.grad = None
        kb.grad = None
        loss.backward()
        torch.cuda.synchronize()
        t3 = time.perf_counter()
    except AbdError as e:
        out["error"] = str(e)
        g.close()
        return out
    gv = qd0.grad[idx, :3].cpu().numpy()
    log(f"adjoint: forward {t1 - t0:.1f} s, backward {t2 - t1:.1f} s, again {t3 - t2:.1f} s")
    out.update({"forward_ms_per_step": 1e3 * (t1 - t0) / nsteps, "backward_ms_per_step": 1e3 * (t2 - t1) / nsteps,
                "backward_again_ms_per_step": 1e3 * (t3 - t2) / nsteps,
                "backward_again_identical": bool(torch.equal(g_first, qd0.grad)),
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


def plain_hash_tests(s, q, dhat, h=None):
    """Box tests a plain primitive-level uniform hash would run at state q
    (the culling the paper's i-AABB is set against, Sec. 4.2), on the host:
    every primitive's box (triangles and edges dilated by dhat, points as
    points) in each cell it covers, cell edge h (default: the median box
    extent of the dynamic bodies' triangles); per cell, point-triangle tests
    between different bodies and edge-edge tests between different bodies,
    a pair sharing k cells counted k times."""
    x = vertices(s, q)
    tri, edge, vb = s.tri, s.edge, s.vbody
    tlo, thi = x[tri].min(axis=1) - dhat, x[tri].max(axis=1) + dhat
    elo, ehi = x[edge].min(axis=1) - dhat, x[edge].max(axis=1) + dhat
    if h is None:
        dyn_t = s.is_static[vb[tri[:, 0]]] == 0
        h = float(np.median((thi - tlo)[dyn_t].max(axis=1)))

    def cells(lo, hi):
        a = np.floor(lo / h).astype(np.int64)
        b = np.floor(hi / h).astype(np.int64)
        ext = b - a + 1
        n = np.prod(ext, axis=1)
        idx = np.repeat(np.arange(len(lo)), n)
        off = np.arange(int(n.sum())) - np.repeat(np.cumsum(n) - n, n)
        e = ext[idx]
        c = a[idx] + np.stack([off % e[:, 0], (off // e[:, 0]) % e[:, 1], off // (e[:, 0] * e[:, 1])], axis=1)
        return idx, ((c[:, 0] + (1 << 20)) << 42) + ((c[:, 1] + (1 << 20)) << 21) + (c[:, 2] + (1 << 20))

    pi, pk = cells(x, x)
    ti, tk = cells(tlo, thi)
    ei, ek = cells(elo, ehi)
    keys, inv = np.unique(np.concatenate([pk, tk, ek]), return_inverse=True)
    n_p, n_t = len(pk), len(tk)
    parts = [(inv[:n_p], vb[pi]), (inv[n_p:n_p + n_t], vb[tri[ti, 0]]), (inv[n_p + n_t:], vb[edge[ei, 0]])]
    cnt = [np.bincount(iv, minlength=len(keys)).astype(np.float64) for iv, _ in parts]
    per_body = []
    for iv, bodies in parts:
        u, c = np.unique(iv.astype(np.int64) * s.nb + bodies, return_counts=True)
        per_body.append((u, c.astype(np.float64)))
    _, ip, it = np.intersect1d(per_body[0][0], per_body[1][0], return_indices=True)
    pt = float((cnt[0] * cnt[1]).sum() - (per_body[0][1][ip] * per_body[1][1][it]).sum())
    ce, cee = cnt[2], per_body[2][1]
    ee = float(((ce * ce - ce) / 2).sum() - ((cee * cee - cee) / 2).sum())
    return {"cell_edge_m": h, "box_tests": pt + ee, "point_triangle": pt, "edge_edge": ee}


def culling_at_state(g, s):
    """the library's culling counts for one enumeration at the scene's
    current state (abd_energy_grad_hess at q), beside a plain primitive
    hash's at the same state"""
    q, _ = g.get_state()
    c0 = g.counters()
    g.energy_grad_hess(q)
    c1 = g.counters()
    lib = {k: c1[k] - c0[k] for k in ("prim_pairs_body", "prim_pairs_iaabb", "prim_pairs_cand")}
    plain = plain_hash_tests(s, q.cpu().numpy(), s.params["dhat"])
    return {"primitive_pairs_of_overlapping_body_pairs": lib["prim_pairs_body"],
            "box_tests_after_iaabb": lib["prim_pairs_iaabb"], "candidates": lib["prim_pairs_cand"],
            "plain_primitive_hash": plain,
            "iaabb_tests_per_plain_hash_test": lib["prim_pairs_iaabb"] / max(plain["box_tests"], 1.0)}


def window_splits(windows, steps):
    """timed steps per window: `steps` split as evenly as possible, the
    remainder to the last windows"""
    n = len(windows)
    base = [steps // n] * n
    for k in range(steps % n):
        base[n - 1 - k] += 1
    return base


def step_summary(stats, ms):
    """per-window figures from the per-step statistics and device times"""
    newton = sum(st["newton_iters"] for st in stats)
    total_s = sum(ms) * 1e-3
    hist = [sum(st["toi_hist"][k] for st in stats) for k in range(6)]
    return {
        "ms_per_step": sum(ms) / len(ms),
        "newton_iters_per_step": newton / len(stats),
        "pcg_iters_per_newton": sum(st["pcg_iters"] for st in stats) / max(newton, 1),
        "ls_rounds_per_newton": sum(st["ls_halvings"] for st in stats) / max(newton, 1),
        "ccd_limited_frac": sum(st["ccd_limited"] for st in stats) / max(newton, 1),
        "toi_hist": {"1": hist[0], "[0.1,1)": hist[1], "[0.01,0.1)": hist[2], "[1e-3,0.01)": hist[3],
                     "[1e-4,1e-3)": hist[4], "<1e-4": hist[5]},
        "toi_min": min(st["toi_min"] for st in stats),
        "max_island_halvings": max(st["ls_island_halvings_max"] for st in stats),
        "islands_last": stats[-1]["n_islands"],
        "active_pairs_last": stats[-1]["n_active"],
        "candidates_last": stats[-1]["n_candidates"],
        "contact_evals_per_s": sum(st["candidates_tested"] for st in stats) / total_s,
        "active_evals_per_s": sum(st["active_evaluated"] for st in stats) / total_s,
        "newton_iters_per_s": newton / total_s,
        "kernel_launches": sum(st["kernel_launches"] for st in stats),
    }


def run_abd(args, rank, world):
    import torch
    from paper_2201_10022_gb300.abd import (AbdError, AbdScene, abd_get_state, abd_set_state, abd_step,
                                            abd_step_stats)
    import ctypes as C

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    s = workload_scene()
    g = AbdScene(s, device=dev)
    gm = None if args.no_mixed else AbdScene(s, device=dev, precision=1)
    windows = [int(w) for w in args.windows.split(",")]
    splits = window_splits(windows, args.steps)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = None
    qh = torch.empty((s.nb, 12), dtype=torch.float64).pin_memory()
    qdh = torch.empty_like(qh).pin_memory()
    sst = abd_step_stats()
    L0 = bbox_diag(vertices(s, s.q0))

    all_ms, all_stats, mixed_ms = [], [], []
    prof_tot = {}
    per_window = []
    clocks_rows = []
    state = {"at": 0, "e2e_s": 0.0}  # steps the scene has advanced; e2e seconds

    def run_window(w, start, nsteps):
        """advance to the window, warm up, then the timed, profiled, e2e and
        mixed passes over its steps"""
        at = state["at"]
        first = max(start - args.warmup, at)
        if first > at:
            g.step(first - at)  # advance untimed (device), the pile's own trajectory
            at = first
        g.step(args.warmup)
        at += args.warmup
        state["at"] = at
        torch.cuda.synchronize()
        log(f"window {w}: warm at step {at}")
        q0, qd0 = g.get_state()
        q0, qd0 = q0.clone(), qd0.clone()

        # ---- device-timed region: inputs resident in HBM ------------------
        clk = ClockSampler(uuid)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clk.start()
        torch.cuda.nvtx.range_push("timed")
        ms, stats = [], []
        for k in range(nsteps):
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
        clocks_rows.append(clk.stop())
        all_ms.extend(ms)
        all_stats.extend(stats)

        # ---- per-kernel-class device times: the same steps again from the
        # same state with the library's event profiling on
        g.set_state(q0, qd0)
        g.set_profiling(True)
        for k in range(nsteps):
            flush.zero_()
            g.step(1)
        torch.cuda.synchronize()
        for name, v in g.profile().items():
            t = prof_tot.setdefault(name, {"launches": 0, "total_ms": 0.0, "bytes": 0.0, "flops": 0.0})
            for key in t:
                t[key] += v[key]
        g.set_profiling(False)

        # ---- end to end through the C ABI with host buffers ----------------
        qh.copy_(q0.cpu())
        qdh.copy_(qd0.cpu())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(nsteps):
            r = abd_set_state(g.h, qh.data_ptr(), qdh.data_ptr(), 0)
            r = r or abd_step(g.h, 1, C.byref(sst))
            r = r or abd_get_state(g.h, qh.data_ptr(), qdh.data_ptr(), 0)
            if r:
                raise RuntimeError(f"e2e step failed: {r}")
        state["e2e_s"] += time.perf_counter() - t0
        at = start_end = at + nsteps  # the scene is at the timed window's end state again
        state["at"] = at

        # ---- mixed precision (precision = 1): the same steps from the same
        # state; its end state against the FP64 run's
        mixed = None
        if gm is not None:
            try:
                gm.set_state(q0, qd0)
                gm.step(1)  # buffer growth outside the timed steps
                gm.set_state(q0, qd0)
                torch.cuda.synchronize()
                ms_m, st_m = [], []
                for k in range(nsteps):
                    flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    st_m.append(gm.step(1))
                    e1.record()
                    torch.cuda.synchronize()
                    ms_m.append(e0.elapsed_time(e1))
                mixed_ms.extend(ms_m)
                qm, _ = gm.get_state()
                mixed = step_summary(st_m, ms_m)
                mixed["max_vertex_deviation_vs_fp64_over_lbbox"] = float(
                    np.abs(vertices(s, qm.cpu().numpy()) - vertices(s, qh.numpy())).max() / L0)
            except AbdError as e:  # reported in the window, not fatal to the FP64 measurement
                mixed = {"error": str(e)}
        summ = step_summary(stats, ms)
        summ["steps"] = f"{start_end - nsteps}..{start_end - 1}"
        summ["mixed"] = mixed
        per_window.append(summ)
        log(f"window {w}: steps {summ['steps']} {summ['ms_per_step']:.1f} ms/step, "
            f"{summ['newton_iters_per_step']:.1f} Newton/step, {summ['pcg_iters_per_newton']:.1f} PCG/Newton")

    failed = None
    for w, (start, nsteps) in enumerate(zip(windows, splits)):
        if nsteps <= 0 or failed:
            continue
        try:
            run_window(w, start, nsteps)
        except (AbdError, RuntimeError) as e:  # the step is transactional: report it and stop here
            failed = {"window_start": start, "error": str(e)}
            log(f"window {w}: {e}")
    if gm is not None:
        gm.close()
    culling_state = None
    if per_window and world == 1:
        try:
            culling_state = culling_at_state(g, s)
            culling_state["state"] = f"end of the last timed window (step {state['at']})"
        except Exception as e:  # reported in the line, not fatal to the headline measurement
            culling_state = {"error": f"{type(e).__name__}: {e}"}
        log("culling counts at the last state done")
    if not all_ms:
        raise RuntimeError(f"no timed window completed: {failed}")
    total_ms = max_over_ranks(sum(all_ms), world, dev)
    e2e_ms = max_over_ranks(1e3 * state["e2e_s"], world, dev)
    cnt = g.counters()
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

    nsteps_all = len(all_ms)
    steps_total = nsteps_all * world
    ms_per_step = aggregate_ms_per_step(total_ms, nsteps_all, world)
    summ_all = step_summary(all_stats, all_ms)
    pk, src = peaks()
    clocks = {"sm_mhz": statistics.median([c["sm_mhz"] for c in clocks_rows if c["sm_mhz"]] or [0]) or None,
              "sm_max_mhz": max([c["sm_max_mhz"] or 0 for c in clocks_rows] or [0]) or None,
              "reasons": sorted({r for c in clocks_rows for r in c["reasons"]}),
              "samples": sum(c["samples"] for c in clocks_rows)}
    # roofline of the kernel class with an algorithmic flop or byte model
    # that took the most device time
    modelled = [kv for kv in prof_tot.items() if kv[1]["flops"] > 0 or kv[1]["bytes"] > 0]
    roof = None
    name, p = max(modelled or prof_tot.items(), key=lambda kv: kv[1]["total_ms"])
    if p["launches"] and p["total_ms"] > 0:
        t_s = p["total_ms"] * 1e-3
        clk_hz = (clocks.get("sm_mhz") or 2070.0) * 1e6
        fp64_peak = 152 * 2 * 2 * clk_hz / 1e12  # 152 SMs x 2 FP64 FMA/clk x 2 flop x clock
        if name == "pcg_solve":
            # FP64 block products on this part are bound by the FP64 pipe, not by HBM
            achieved = p["flops"] / t_s / 1e12
            roof = {"kernel": name, "bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                    "frac": achieved / fp64_peak, "traffic": PCG_DRAM_BYTES_PER_ITER,
                    "peak_source": "derived (152 SMs x 2 FP64 FMA/clk x clock)",
                    "hbm_achieved_gbs": p["bytes"] / t_s / 1e9, "hbm_peak_gbs": pk["hbm_gbs"],
                    "hbm_frac": p["bytes"] / t_s / 1e9 / pk["hbm_gbs"], "hbm_peak_source": src,
                    "launches": p["launches"], "avg_launch_ms": p["total_ms"] / p["launches"]}
        elif p["flops"] > 0:
            achieved = p["flops"] / t_s / 1e12
            roof = {"kernel": name, "bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                    "frac": achieved / fp64_peak, "traffic": BARRIER_DRAM_BYTES if name == "barrier_terms" else None,
                    "peak_source": "derived (152 SMs x 2 FP64 FMA/clk x clock)",
                    "launches": p["launches"], "avg_launch_ms": p["total_ms"] / p["launches"]}
        elif p["bytes"] > 0:
            achieved = p["bytes"] / t_s / 1e9
            roof = {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / pk["hbm_gbs"], "traffic": None, "peak_source": src,
                    "launches": p["launches"], "avg_launch_ms": p["total_ms"] / p["launches"]}
    win_desc = ", ".join(w["steps"] for w in per_window)
    out = {
        "metric": METRIC, "value": ms_per_step, "unit": "ms/step", "n_gpus": world, "steps": nsteps_all,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"lattice_pile {WORKLOAD['nx']}x{WORKLOAD['ny']}x{WORKLOAD['nz']} seed "
                               f"{WORKLOAD['seed']}, {s.nb} bodies ({s.nv} vertices, {s.nt} triangles, {s.ne} edges), "
                               f"mu 0.3, kappa 1e8, dt 0.01, dhat 1e-3; timed steps in windows {win_desc} of the "
                               f"pile's own trajectory (first impacts, ground contact, second layer landing); "
                               f"value = mean ms/step over every timed step",
                   "timed_steps": win_desc,
                   "l2": "256 MB buffer written between timed steps",
                   "newton_tol": "1e-5 * bbox diagonal * dt", "pcg_rel_tol": 1e-4, "parallelism": f"replicas x{world}"},
        "steps_per_s": 1e3 / ms_per_step,
        "newton_iters_per_s": summ_all["newton_iters_per_s"],
        "contact_evals_per_s": summ_all["contact_evals_per_s"],
        "active_evals_per_s": summ_all["active_evals_per_s"],
        "newton_iters_per_step": summ_all["newton_iters_per_step"],
        "pcg_iters_per_newton": summ_all["pcg_iters_per_newton"],
        "windows": per_window,
        "windows_failed": failed,
        "e2e": {"value": e2e_ms / steps_total, "unit": "ms/step", "h2d_bytes_per_step": 2 * 12 * 8 * s.nb,
                "d2h_bytes_per_step": 2 * 12 * 8 * s.nb},
        "gpu_launches": summ_all["kernel_launches"],
        "roofline": roof,
        "kernel_ms": {k: round(v["total_ms"], 3) for k, v in prof_tot.items()},
        "barrier_counters": {k: cnt[k] for k in ("barrier_terms", "sweeps_fp32", "sweeps_fp64", "capped_fp64")},
        "culling": {"prim_pairs_of_body_pairs": cnt["prim_pairs_body"],
                    "prim_pairs_after_iaabb": cnt["prim_pairs_iaabb"],
                    "candidates": cnt["prim_pairs_cand"],
                    "iaabb_kept_frac": cnt["prim_pairs_iaabb"] / max(cnt["prim_pairs_body"], 1),
                    "candidates_frac_of_iaabb": cnt["prim_pairs_cand"] / max(cnt["prim_pairs_iaabb"], 1),
                    "scope": "every enumeration since the scene was created (advance, warm-up, timed, profiled "
                             "and e2e steps)",
                    "at_one_state": culling_state},
        "mixed": None if gm is None or not mixed_ms else {
            "value": sum(mixed_ms) / len(mixed_ms), "unit": "ms/step",
            "precision": "FP32-stored Hessian blocks and FP32 inner PCG iterations with FP64 iterative refinement of "
                         "the linear residual; FP32 eigenbasis for the barrier Hessian projection; distances, "
                         "barrier values, energies, gradients, CCD, Newton test and line search FP64",
            "per_window": "windows[k].mixed"},
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
    ap.add_argument("--windows", default=DEFAULT_WINDOWS,
                    help="first steps of the timed windows (comma-separated); --steps is split over them")
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
        cb = oracle_sample(int(args.windows.split(",")[0]))
        line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "ms/step", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": cb["value"], "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "the same pile, first steps of the first timed window (see "
                                       "cpu_baseline.sample)"},
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
            cb = oracle_sample(int(args.windows.split(",")[0]))
            out["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
        else:
            out["cpu_baseline"] = None
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
