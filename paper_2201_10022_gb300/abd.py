"""Python binding of libabd.so (include/abd.h): argument marshalling only.

Every function named ``abd_*`` here calls the C function of the same name;
all compute runs in the library's CUDA kernels.  PyTorch provides device
memory (through the ``abd_allocator`` callbacks backed by its caching
allocator) and the CUDA stream.  There is no CPU fallback: loading fails
loudly when the library cannot be built or loaded.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

# ---------------------------------------------------------------------------
# C structures (mirror include/abd.h)
# ---------------------------------------------------------------------------
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)

STATUS = {0: "ABD_OK", 1: "ABD_ERR_INVALID_ARG", 2: "ABD_ERR_CUDA", 3: "ABD_ERR_OOM", 4: "ABD_ERR_CAPACITY",
          5: "ABD_ERR_INITIAL_INTERSECTION", 6: "ABD_ERR_NONFINITE", 7: "ABD_ERR_NEWTON_MAXITER",
          8: "ABD_ERR_LINESEARCH", 9: "ABD_ERR_PCG_BREAKDOWN", 10: "ABD_ERR_PCG_MAXITER", 11: "ABD_ERR_CCD_MAXITER"}


class abd_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class abd_params(C.Structure):
    _fields_ = [("dt", C.c_double), ("dhat", C.c_double), ("kappa", C.c_double), ("gravity", C.c_double * 3),
                ("mu", C.c_double), ("eps_v", C.c_double), ("newton_tol", C.c_double), ("pcg_rel_tol", C.c_double),
                ("ls_slack_rel", C.c_double), ("ccd_s", C.c_double), ("newton_max", C.c_int), ("pcg_max", C.c_int),
                ("ls_max", C.c_int), ("ccd_max", C.c_int), ("precision", C.c_int), ("dense_max_dofs", C.c_int)]


class abd_scene_desc(C.Structure):
    _fields_ = [("nb", C.c_int), ("nv", C.c_int), ("nt", C.c_int), ("ne", C.c_int),
                ("xbar", C.c_void_p), ("tri", C.c_void_p), ("edge", C.c_void_p), ("vbody", C.c_void_p),
                ("q0", C.c_void_p), ("qdot0", C.c_void_p), ("density", C.c_void_p), ("kappa_body", C.c_void_p),
                ("is_static", C.c_void_p)]


class abd_pair_counts(C.Structure):
    _fields_ = [("n_candidates", C.c_long), ("n_active", C.c_long), ("n_friction", C.c_long),
                ("n_body_pairs", C.c_long)]


class abd_solve_stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("rel_residual", C.c_double)]


class abd_step_stats(C.Structure):
    _fields_ = [("newton_iters", C.c_int), ("pcg_iters", C.c_int), ("ls_halvings", C.c_int),
                ("n_candidates", C.c_long), ("n_active", C.c_long), ("n_swept", C.c_long),
                ("toi_min", C.c_double), ("last_step", C.c_double), ("kernel_launches", C.c_long),
                ("candidates_tested", C.c_long), ("active_evaluated", C.c_long), ("ccd_limited", C.c_int),
                ("toi_hist", C.c_int * 6), ("n_islands", C.c_int), ("ls_island_halvings_max", C.c_int)]


class abd_kernel_profile(C.Structure):
    _fields_ = [("name", C.c_char_p), ("launches", C.c_long), ("total_ms", C.c_double), ("bytes", C.c_double),
                ("flops", C.c_double)]


class abd_counters(C.Structure):
    _fields_ = [("barrier_terms", C.c_ulonglong * 4), ("sweeps_fp32", C.c_ulonglong),
                ("sweeps_fp64", C.c_ulonglong), ("capped_fp64", C.c_ulonglong),
                ("prim_pairs_body", C.c_ulonglong), ("prim_pairs_iaabb", C.c_ulonglong),
                ("prim_pairs_cand", C.c_ulonglong)]


class abd_tuning(C.Structure):
    _fields_ = [("grid_div", C.c_int), ("cluster_max", C.c_int), ("reserved", C.c_int * 6)]


def _as_dict(st):
    return {k: (list(getattr(st, k)) if isinstance(getattr(st, k), C.Array) else getattr(st, k))
            for k, _ in st._fields_}


_lib = None
EXPORTS = ["abd_default_params", "abd_create_scene", "abd_destroy", "abd_set_state", "abd_get_state",
           "abd_energy_grad_hess", "abd_get_hessian", "abd_get_pairs", "abd_get_friction", "abd_solve",
           "abd_ccd_toi", "abd_step",
           "abd_set_profiling", "abd_get_profile", "abd_get_counters", "abd_adjoint_step",
           "abd_ccd_toi_pairs_noalloc", "abd_set_tuning", "abd_get_tuning", "abd_step_batch", "abd_last_error"]


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libabd.so (compiling it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libabd.so not found at {path}: build it with paper_2201_10022_gb300.build.build()")
    L = C.CDLL(path)
    vp, i, l, d = C.c_void_p, C.c_int, C.c_long, C.c_double
    sig = {
        "abd_default_params": (None, [vp]),
        "abd_create_scene": (i, [vp, vp, vp, vp, vp]),
        "abd_destroy": (None, [vp]),
        "abd_set_state": (i, [vp, vp, vp, i]),
        "abd_get_state": (i, [vp, vp, vp, i]),
        "abd_energy_grad_hess": (i, [vp, vp, vp, vp, vp]),
        "abd_get_hessian": (i, [vp, vp, vp, vp, vp, l, vp]),
        "abd_get_pairs": (i, [vp, i, vp, vp, vp, vp, vp, l, vp]),
        "abd_get_friction": (i, [vp, vp, vp, vp, l, vp]),
        "abd_solve": (i, [vp, vp, vp, vp]),
        "abd_ccd_toi": (i, [vp, vp, vp, vp]),
        "abd_step": (i, [vp, i, vp]),
        "abd_set_profiling": (i, [vp, i]),
        "abd_get_profile": (i, [vp, vp, i, vp]),
        "abd_get_counters": (i, [vp, vp]),
        "abd_adjoint_step": (i, [vp, vp, vp, vp, vp, vp, vp, d, vp]),
        "abd_ccd_toi_pairs_noalloc": (i, [vp, vp, i, vp, vp, l, d, i, vp, vp]),
        "abd_set_tuning": (i, [vp, vp]),
        "abd_get_tuning": (i, [vp, vp]),
        "abd_step_batch": (i, [vp, i, i, i, vp, vp]),
        "abd_last_error": (C.c_char_p, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


class AbdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


# ---------------------------------------------------------------------------
# C-ABI functions, same names
# ---------------------------------------------------------------------------

def abd_default_params() -> abd_params:
    p = abd_params()
    load().abd_default_params(C.byref(p))
    return p


def abd_create_scene(desc: abd_scene_desc, params: abd_params, alloc, stream: int):
    h = C.c_void_p()
    r = load().abd_create_scene(C.byref(desc), C.byref(params), C.byref(alloc) if alloc is not None else None,
                                C.c_void_p(stream), C.byref(h))
    return r, h


def abd_destroy(h):
    load().abd_destroy(h)


def abd_set_state(h, q_ptr, qdot_ptr, on_device):
    return load().abd_set_state(h, C.c_void_p(q_ptr), C.c_void_p(qdot_ptr), int(on_device))


def abd_get_state(h, q_ptr, qdot_ptr, on_device):
    return load().abd_get_state(h, C.c_void_p(q_ptr), C.c_void_p(qdot_ptr), int(on_device))


def abd_energy_grad_hess(h, q_ptr, E_host, g_ptr, counts):
    return load().abd_energy_grad_hess(h, C.c_void_p(q_ptr), E_host, C.c_void_p(g_ptr), counts)


def abd_get_hessian(h, diag, bi, bj, blocks, cap, nblocks):
    return load().abd_get_hessian(h, diag, bi, bj, blocks, cap, nblocks)


def abd_get_pairs(h, which, kind, i, j, type_, d2, cap, n):
    return load().abd_get_pairs(h, which, kind, i, j, type_, d2, cap, n)


def abd_get_friction(h, gamma, normal, offset, cap, n):
    return load().abd_get_friction(h, gamma, normal, offset, cap, n)


def abd_solve(h, rhs_ptr, dq_ptr, stats):
    return load().abd_solve(h, C.c_void_p(rhs_ptr), C.c_void_p(dq_ptr), stats)


def abd_ccd_toi(h, q_ptr, dq_ptr, toi):
    return load().abd_ccd_toi(h, C.c_void_p(q_ptr), C.c_void_p(dq_ptr), toi)


def abd_step(h, nsteps, stats):
    return load().abd_step(h, int(nsteps), stats)


def abd_set_profiling(h, on):
    return load().abd_set_profiling(h, int(on))


def abd_get_profile(h, out, cap, n):
    return load().abd_get_profile(h, out, cap, n)


def abd_get_counters(h, out):
    return load().abd_get_counters(h, out)


def abd_adjoint_step(h, q_t, qdot_t, q_next, gq, gqdot, gkappa, rel_tol, stats):
    return load().abd_adjoint_step(h, C.c_void_p(q_t), C.c_void_p(qdot_t), C.c_void_p(q_next), C.c_void_p(gq),
                                   C.c_void_p(gqdot), C.c_void_p(gkappa), float(rel_tol), stats)


def abd_ccd_toi_pairs_noalloc(x_ptr, dx_ptr, nv, verts_ptr, kind_ptr, npairs, ccd_s, ccd_max, stream, toi):
    """Allocation-free CCD bound over caller-given pairs (see include/abd.h)."""
    return load().abd_ccd_toi_pairs_noalloc(C.c_void_p(x_ptr), C.c_void_p(dx_ptr), int(nv), C.c_void_p(verts_ptr),
                                            C.c_void_p(kind_ptr), int(npairs), float(ccd_s), int(ccd_max),
                                            C.c_void_p(stream), toi)


def abd_set_tuning(h, tuning):
    return load().abd_set_tuning(h, C.byref(tuning))


def abd_get_tuning(h, tuning):
    return load().abd_get_tuning(h, C.byref(tuning))


def abd_step_batch(handles, nsteps, nworkers, status, stats):
    """handles: sequence of scene handles; status: (c_int * n) or None;
    stats: (abd_step_stats * n) or None"""
    arr = (C.c_void_p * len(handles))(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    return load().abd_step_batch(arr, len(handles), int(nsteps), int(nworkers), status, stats)


def abd_last_error(h) -> str:
    s = load().abd_last_error(h)
    return s.decode() if s else ""


# ---------------------------------------------------------------------------
# convenience wrapper over one scene (torch tensors in, numpy / torch out)
# ---------------------------------------------------------------------------

def _np_ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class TorchAllocator:
    """abd_allocator backed by PyTorch's caching allocator."""

    def __init__(self, device):
        import torch
        self._torch = torch
        self.device = torch.device(device)

        def _alloc(nbytes, stream, ctx):
            try:
                return self._torch.cuda.caching_allocator_alloc(int(nbytes), self.device.index, stream)
            except Exception:  # out of memory: report NULL to the library
                return None

        def _free(ptr, stream, ctx):
            self._torch.cuda.caching_allocator_delete(ptr)

        self._alloc_cb = ALLOC_FN(_alloc)
        self._free_cb = FREE_FN(_free)
        self.struct = abd_allocator(self._alloc_cb, self._free_cb, None)


class AbdScene:
    """A scene of the CUDA library (one GPU, one stream).

    ``scene`` is a :class:`paper_2201_10022_gb300.scenes.Scene`; keyword
    arguments override fields of :func:`abd_default_params`."""

    def __init__(self, scene, device="cuda:0", stream=None, torch_alloc=True, **params):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.scene = scene
        self.nb = scene.nb
        p = abd_default_params()
        prm = dict(scene.params)
        prm.update(params)
        for k, v in prm.items():
            if k == "gravity":
                p.gravity[:] = list(v)
            elif hasattr(p, k):
                setattr(p, k, v)
        self.params = p
        self._keep = [np.ascontiguousarray(scene.xbar, dtype=np.float64),
                      np.ascontiguousarray(scene.tri, dtype=np.int32),
                      np.ascontiguousarray(scene.edge, dtype=np.int32),
                      np.ascontiguousarray(scene.vbody, dtype=np.int32),
                      np.ascontiguousarray(scene.q0, dtype=np.float64),
                      np.ascontiguousarray(scene.qdot0, dtype=np.float64),
                      np.ascontiguousarray(scene.density, dtype=np.float64),
                      np.ascontiguousarray(scene.kappa_body, dtype=np.float64),
                      np.ascontiguousarray(scene.is_static, dtype=np.uint8)]
        d = abd_scene_desc(scene.nb, scene.nv, scene.nt, scene.ne, *[_np_ptr(a) for a in self._keep])
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.alloc = TorchAllocator(self.device) if torch_alloc else None
            r, h = abd_create_scene(d, p, self.alloc.struct if self.alloc else None, self.stream.cuda_stream)
        if r != 0:
            raise AbdError(r, "abd_create_scene failed")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            with self.torch.cuda.device(self.device):
                abd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, r):
        if r != 0:
            raise AbdError(r, abd_last_error(self.h))

    def _dev(self, t):
        t = self.torch.as_tensor(t, dtype=self.torch.float64, device=self.device).contiguous()
        return t

    # state -----------------------------------------------------------------
    def set_state(self, q, qdot):
        q, qd = self._dev(q), self._dev(qdot)
        with self.torch.cuda.device(self.device):
            self._check(abd_set_state(self.h, q.data_ptr(), qd.data_ptr(), 1))

    def get_state(self):
        q = self.torch.empty((self.nb, 12), dtype=self.torch.float64, device=self.device)
        qd = self.torch.empty_like(q)
        with self.torch.cuda.device(self.device):
            self._check(abd_get_state(self.h, q.data_ptr(), qd.data_ptr(), 1))
        return q, qd

    # parity entry points ------------------------------------------------------
    def energy_grad_hess(self, q):
        q = self._dev(q)
        g = self.torch.empty((self.nb, 12), dtype=self.torch.float64, device=self.device)
        E = (C.c_double * 5)()
        cnt = abd_pair_counts()
        with self.torch.cuda.device(self.device):
            self._check(abd_energy_grad_hess(self.h, q.data_ptr(), E, g.data_ptr(), C.byref(cnt)))
        return np.array(E[:]), g, _as_dict(cnt)

    def hessian(self):
        n = C.c_long()
        self._check(abd_get_hessian(self.h, None, None, None, None, 0, C.byref(n)))
        m = max(n.value, 1)
        diag = np.zeros((self.nb, 12, 12))
        bi = np.zeros(m, np.int32)
        bj = np.zeros(m, np.int32)
        blocks = np.zeros((m, 12, 12))
        self._check(abd_get_hessian(self.h, _np_ptr(diag), _np_ptr(bi), _np_ptr(bj), _np_ptr(blocks), m,
                                    C.byref(n)))
        k = n.value
        return diag, np.stack([bi[:k], bj[:k]], axis=1), blocks[:k]

    def pairs(self, which=1):
        n = C.c_long()
        self._check(abd_get_pairs(self.h, which, None, None, None, None, None, 0, C.byref(n)))
        m = max(n.value, 1)
        kind, pi, pj, ty = (np.zeros(m, np.int32) for _ in range(4))
        d2 = np.zeros(m)
        self._check(abd_get_pairs(self.h, which, _np_ptr(kind), _np_ptr(pi), _np_ptr(pj), _np_ptr(ty), _np_ptr(d2),
                                  m, C.byref(n)))
        k = n.value
        return dict(kind=kind[:k], i=pi[:k], j=pj[:k], type=ty[:k], val=d2[:k])

    def friction_records(self):
        """lagged friction records (order of pairs(2)): gamma (n x 4), unit
        normal (n x 3), lagged offset (n x 3)"""
        n = C.c_long()
        self._check(abd_get_friction(self.h, None, None, None, 0, C.byref(n)))
        m = max(n.value, 1)
        ga, nn, rr = np.zeros((m, 4)), np.zeros((m, 3)), np.zeros((m, 3))
        self._check(abd_get_friction(self.h, _np_ptr(ga), _np_ptr(nn), _np_ptr(rr), m, C.byref(n)))
        k = n.value
        return ga[:k], nn[:k], rr[:k]

    def solve(self, rhs):
        rhs = self._dev(rhs)
        dq = self.torch.empty_like(rhs)
        st = abd_solve_stats()
        with self.torch.cuda.device(self.device):
            r = abd_solve(self.h, rhs.data_ptr(), dq.data_ptr(), C.byref(st))
        self._check(r)
        return dq, _as_dict(st)

    def ccd_toi(self, q, dq):
        q, dq = self._dev(q), self._dev(dq)
        t = C.c_double()
        with self.torch.cuda.device(self.device):
            self._check(abd_ccd_toi(self.h, q.data_ptr(), dq.data_ptr(), C.byref(t)))
        return t.value

    def step(self, n=1):
        st = abd_step_stats()
        with self.torch.cuda.device(self.device):
            self._check(abd_step(self.h, n, C.byref(st)))
        return _as_dict(st)

    def set_profiling(self, on):
        self._check(abd_set_profiling(self.h, on))

    def profile(self):
        arr = (abd_kernel_profile * 16)()
        n = C.c_int()
        self._check(abd_get_profile(self.h, arr, 16, C.byref(n)))
        return {arr[k].name.decode(): dict(launches=arr[k].launches, total_ms=arr[k].total_ms, bytes=arr[k].bytes,
                                           flops=arr[k].flops)
                for k in range(min(n.value, 16))}

    def adjoint_step(self, q_t, qdot_t, q_next, gq, gqdot, gkappa, rel_tol=1e-12):
        """one step backwards (see abd_adjoint_step): gq, gqdot (nb x 12) hold
        dL/dq_next, dL/dqdot_next and receive dL/dq_t, dL/dqdot_t; gkappa (nb)
        accumulates dL/dkappa_body.  All float64 tensors on the scene's device."""
        st = abd_solve_stats()
        args = [self._dev(t) for t in (q_t, qdot_t, q_next)]
        for t in (gq, gqdot, gkappa):
            if t.device != self.device or t.dtype != self.torch.float64 or not t.is_contiguous():
                raise ValueError("gq, gqdot, gkappa: contiguous float64 tensors on the scene's device")
        with self.torch.cuda.device(self.device):
            self._check(abd_adjoint_step(self.h, *[a.data_ptr() for a in args], gq.data_ptr(), gqdot.data_ptr(),
                                         gkappa.data_ptr(), rel_tol, C.byref(st)))
        return _as_dict(st)

    def set_tuning(self, grid_div=1, cluster_max=0):
        """grid_div: divisor of the device-sized grids (1..64); cluster_max:
        bodies per preconditioner cluster (1..16, 0 = the default 12)"""
        t = abd_tuning()
        t.grid_div = int(grid_div)
        t.cluster_max = int(cluster_max)
        self._check(abd_set_tuning(self.h, t))

    def tuning(self):
        t = abd_tuning()
        self._check(abd_get_tuning(self.h, t))
        return {"grid_div": t.grid_div, "cluster_max": t.cluster_max}

    def counters(self):
        c = abd_counters()
        self._check(abd_get_counters(self.h, C.byref(c)))
        return _as_dict(c)
