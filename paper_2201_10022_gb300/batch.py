"""Many independent scenes stepped together (the many-scene form of the
time step of Sec. 4), with an autotuner for the launch shape.

``SceneBatch(scenes, ...)`` creates one library scene per
:class:`~paper_2201_10022_gb300.scenes.Scene`, each on its own CUDA stream,
and ``step(n)`` advances all of them through ``abd_step_batch``: a pool of
host threads drives the scenes' Newton loops (each with its own captured
launch sequences) so that the kernels of many small scenes share the GPU.
Every scene keeps its own Newton iteration, line search and convergence test,
so its result is bit-identical to stepping it alone.

``tune()`` picks the two knobs of the batch (host workers, i.e. scenes in
flight, and the grid divisor of the device-sized kernels: one value for all
scenes or a divisor per scene by its size) by timing short runs from the
current state, restores the state afterwards, and caches the choice per
(GPU, size class) in a JSON file.
"""
from __future__ import annotations

import ctypes as C
import json
import os
import time

import numpy as np

from . import abd as A

_GRID_DIVS = (1, 4, 16)
_WORKERS = (1, 2, 4, 8, 16, 32, 64)


def _cache_path() -> str:
    p = os.environ.get("ABD_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_2201_10022_gb300", "tune.json")


class SceneBatch:
    def __init__(self, scenes, device="cuda:0", params_list=None, **params):
        """params: abd_params overrides for every scene; params_list: one
        dict of further overrides per scene (e.g. a per-scene newton_tol)"""
        import torch
        self.torch = torch
        self.device = torch.device(device)
        extra = params_list or [{}] * len(scenes)
        self.scenes = [A.AbdScene(s, device=self.device, stream=torch.cuda.Stream(self.device), **{**params, **e})
                       for s, e in zip(scenes, extra)]
        self.params = params
        self.nworkers = min(16, os.cpu_count() or 1, max(1, len(self.scenes)))
        self.grid_div = 1

    def __len__(self):
        return len(self.scenes)

    @property
    def bodies(self):
        return [s.nb for s in self.scenes]

    # state ----------------------------------------------------------------
    def get_states(self):
        return [s.get_state() for s in self.scenes]

    def set_states(self, states):
        for s, (q, qd) in zip(self.scenes, states):
            s.set_state(q, qd)

    # stepping ---------------------------------------------------------------
    def set_tuning(self, nworkers=None, grid_div=None):
        if nworkers is not None:
            self.nworkers = int(nworkers)
        if grid_div is not None:
            self.grid_div = int(grid_div)
            for s in self.scenes:
                s.set_tuning(grid_div=self.grid_div)

    def step(self, n=1, nworkers=None):
        """advance every scene n steps; returns the per-scene abd_step_stats
        dicts; raises AbdError naming the failing scenes"""
        k = len(self.scenes)
        status = (C.c_int * k)()
        stats = (A.abd_step_stats * k)()
        self.torch.cuda.synchronize(self.device)
        with self.torch.cuda.device(self.device):
            r = A.abd_step_batch([s.h for s in self.scenes], n, nworkers or self.nworkers, status, stats)
        if r != 0:
            bad = [(i, A.STATUS.get(status[i], status[i]), A.abd_last_error(self.scenes[i].h))
                   for i in range(k) if status[i] != 0]
            raise A.AbdError(r, f"{len(bad)} scene(s) failed, first: {bad[:3]}")
        return [A._as_dict(stats[i]) for i in range(k)]

    def time_steps(self, n=1, nworkers=None):
        """wall-clock ms of n batch steps (the call returns after every
        scene's stream has drained)"""
        self.torch.cuda.synchronize(self.device)
        t0 = time.perf_counter()
        st = self.step(n, nworkers)
        self.torch.cuda.synchronize(self.device)
        return 1e3 * (time.perf_counter() - t0), st

    # autotuner --------------------------------------------------------------
    def size_class(self) -> str:
        b = np.array(self.bodies)
        prec = int(self.params.get("precision", 0))
        return (f"scenes{int(2 ** np.round(np.log2(max(len(b), 1))))}"
                f"_median{int(2 ** np.round(np.log2(max(np.median(b), 1))))}"
                f"_max{int(2 ** np.ceil(np.log2(max(b.max(), 1))))}_prec{prec}")

    def _key(self) -> str:
        name = self.torch.cuda.get_device_name(self.device)
        return f"{name}|{self.size_class()}"

    def set_grid_policy(self, policy):
        """grid divisor per scene: an int for every scene, or "by_size"
        (2^round(log2(4096 / bodies)), clamped to 1..64: small scenes leave
        most SMs to the others)"""
        if policy == "by_size":
            for s in self.scenes:
                g = int(2 ** np.round(np.log2(4096.0 / max(s.nb, 1))))
                s.set_tuning(grid_div=min(64, max(1, g)))
            self.grid_div = "by_size"
        else:
            self.set_tuning(grid_div=int(policy))

    def tune(self, trial_steps=1, use_cache=True, write_cache=True, log=None, workers=None, policies=None):
        """choose (nworkers, grid policy): the worker count first at the
        by-size grid policy, then the policy at that worker count; every trial
        runs one untimed step (re-capture of the launch sequences) and
        trial_steps timed steps from the same saved state, which is restored
        at the end"""
        key = self._key()
        path = _cache_path()
        cache = {}
        if os.path.exists(path):
            try:
                with open(path) as f:
                    cache = json.load(f)
            except (OSError, ValueError):
                cache = {}
        if use_cache and key in cache:
            c = cache[key]
            self.nworkers = c["nworkers"]
            self.set_grid_policy(c["grid_div"])
            return dict(c, cached=True)
        saved = [(q.clone(), qd.clone()) for q, qd in self.get_states()]
        cpus = os.cpu_count() or 1
        trials = []

        memo = {}

        def run(nw, gp):
            if (nw, gp) in memo:
                return memo[(nw, gp)]
            self.nworkers = nw
            self.set_grid_policy(gp)
            self.set_states(saved)
            self.step(1)
            self.set_states(saved)
            ms, _ = self.time_steps(trial_steps)
            trials.append({"nworkers": nw, "grid_div": gp, "ms": ms})
            if log:
                log(f"tune: workers {nw} grid {gp}: {ms:.1f} ms")
            memo[(nw, gp)] = ms
            return ms

        # a worker waits on its scene's stream by polling: no more workers
        # than cores; one or two workers only for small batches
        if workers is None:
            lo = 1 if len(self.scenes) < 32 else 4
            workers = [w for w in _WORKERS if lo <= w <= max(1, min(len(self.scenes), cpus))] or [1]
        policies = policies or ["by_size", *_GRID_DIVS]
        best_nw = min(workers, key=lambda nw: run(nw, policies[0]))
        best_gp = min(policies, key=lambda gp: run(best_nw, gp))
        self.nworkers = best_nw
        self.set_grid_policy(best_gp)
        self.set_states(saved)
        res = {"nworkers": best_nw, "grid_div": best_gp, "trial_steps": trial_steps, "trials": trials}
        if write_cache:
            cache[key] = res
            try:
                os.makedirs(os.path.dirname(path), exist_ok=True)
                with open(path, "w") as f:
                    json.dump(cache, f, indent=1)
            except OSError:
                pass
        return dict(res, cached=False)

    def close(self):
        for s in self.scenes:
            s.close()
        self.scenes = []
