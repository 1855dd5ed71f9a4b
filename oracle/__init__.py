"""CPU oracle for the affine-body implicit time step.

TEST INFRASTRUCTURE ONLY.  A plain, slow FP64 C implementation written from
the paper (Lan et al., Affine Body Dynamics, 2022), loaded through ctypes.
Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import it; the CUDA library shares no code with it.

Parity status of each oracle function (what pins it) is listed in the test
files ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = ["ip.c", "geometry.c", "jet.c"]
_LIB_PATH = os.path.join(_HERE, "_build", "liborc.so")
_lib = None

ORC_PT, ORC_EE = 0, 1
ERRORS = {0: "ok", 1: "newton cap", 2: "line search cap", 3: "ccd cap", 4: "solve failed",
          5: "intersection", 6: "bad argument"}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (contraction off: the canonical evaluation
    order relies on it)."""
    srcs = [os.path.join(_HERE, s) for s in _SRC + ["abd_oracle.h", "jet.h"]]
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(s) for s in srcs)):
        return _LIB_PATH
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp] + [os.path.join(_HERE, s) for s in _SRC] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Scene(C.Structure):
    _fields_ = [("nb", C.c_int), ("nv", C.c_int), ("nt", C.c_int), ("ne", C.c_int),
                ("xbar", C.c_void_p), ("tri", C.c_void_p), ("edge", C.c_void_p), ("vbody", C.c_void_p),
                ("density", C.c_void_p), ("kappa_body", C.c_void_p), ("is_static", C.c_void_p),
                ("dt", C.c_double), ("dhat", C.c_double), ("kappa", C.c_double),
                ("gravity", C.c_double * 3), ("mu", C.c_double), ("eps_v", C.c_double),
                ("newton_tol", C.c_double), ("ls_slack_rel", C.c_double), ("cg_tol", C.c_double),
                ("ccd_s", C.c_double),
                ("newton_max", C.c_int), ("ls_max", C.c_int), ("ccd_max", C.c_int), ("cg_max", C.c_int),
                ("dense_max_dof", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("newton_iters", C.c_int), ("ls_halvings", C.c_int), ("solve_iters", C.c_int),
                ("n_candidates", C.c_int), ("n_active", C.c_int), ("n_swept", C.c_int),
                ("n_friction", C.c_int), ("toi_min", C.c_double), ("last_step", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        vp, dp, ip, i, d, l = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_int, C.c_double, C.c_long
        sig = {
            "orc_create": (vp, [vp]), "orc_destroy": (None, [vp]),
            "orc_set_state": (i, [vp, vp, vp]), "orc_get_state": (None, [vp, vp, vp]),
            "orc_get_qtilde": (None, [vp, vp]),
            "orc_body_moments": (None, [vp, i, vp, vp, vp]), "orc_mass_matrix": (None, [vp, i, vp]),
            "orc_vertices": (None, [vp, vp, vp]), "orc_displacements": (None, [vp, vp, vp]),
            "orc_ortho": (d, [vp, d, d, vp, vp]),
            "orc_d2_pp": (d, [vp, vp]), "orc_d2_pe": (d, [vp, vp, vp]),
            "orc_d2_pt_plane": (d, [vp, vp, vp, vp]), "orc_d2_ee_line": (d, [vp, vp, vp, vp]),
            "orc_pt_dist2": (d, [vp, vp, vp, vp, vp]), "orc_ee_dist2": (d, [vp, vp, vp, vp, vp]),
            "orc_pair_dist2": (d, [i, vp, vp]), "orc_barrier": (d, [d, d]),
            "orc_pair_barrier": (i, [i, vp, d, d, d, i, vp, vp, vp]),
            "orc_ee_cross2": (d, [vp]), "orc_ee_mollifier": (d, [d, d, vp, vp]),
            "orc_adjoint_step": (i, [vp, vp, vp, vp, vp, vp, vp]),
            "orc_sym_eig": (None, [i, vp, vp, vp]), "orc_project_psd": (None, [i, vp]),
            "orc_accd": (i, [i, vp, vp, d, d, i, vp]),
            "orc_friction_pair": (d, [vp, vp, vp, vp, d, d, vp, vp]),
            "orc_closest_weights": (d, [i, vp, vp, vp]),
            "orc_candidates": (l, [vp, vp, vp, i, vp, vp, vp, l]),
            "orc_energy_grad_hess": (i, [vp, vp, vp, vp, i]), "orc_energy": (d, [vp, vp]),
            "orc_hess_nblocks": (l, [vp]), "orc_hess_copy": (None, [vp, vp, vp, vp]),
            "orc_active_pairs": (l, [vp, vp, vp, vp, vp, vp, vp, l]),
            "orc_grad_rows": (i, [vp, vp, i, vp, vp]),
            "orc_pairs_count": (l, [vp, i]), "orc_pairs_copy": (None, [vp, i, vp, vp, vp, vp, vp]),
            "orc_friction_copy": (None, [vp, vp, vp, vp]),
            "orc_solve": (i, [vp, vp, vp, vp]), "orc_ldl_solve": (i, [i, vp, vp, vp]), "orc_ccd_toi": (i, [vp, vp, vp, vp]),
            "orc_step": (i, [vp, i, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _f64(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None:
        assert a.size == n, (a.size, n)
    return a


# ---------------------------------------------------------------------------
# free functions (geometry, barrier, orthogonality, ACCD)
# ---------------------------------------------------------------------------

def pt_dist2(x0, x1, x2, x3):
    t = C.c_int()
    v = [_f64(a, 3) for a in (x0, x1, x2, x3)]
    d2 = lib().orc_pt_dist2(*[_p(a) for a in v], C.byref(t))
    return d2, t.value


def ee_dist2(x0, x1, x2, x3):
    t = C.c_int()
    v = [_f64(a, 3) for a in (x0, x1, x2, x3)]
    d2 = lib().orc_ee_dist2(*[_p(a) for a in v], C.byref(t))
    return d2, t.value


def pair_dist2(kind, x12):
    t = C.c_int()
    x = _f64(x12, 12)
    return lib().orc_pair_dist2(kind, _p(x), C.byref(t)), t.value


def barrier(d, dhat):
    return lib().orc_barrier(float(d), float(dhat))


def pair_barrier(kind, x12, dhat, kappa, project=True, eps_x=0.0):
    """kappa B(d) of one pair (times the edge-edge mollifier when eps_x > 0)"""
    x = _f64(x12, 12)
    E = np.zeros(1)
    g = np.zeros(12)
    H = np.zeros(144)
    act = lib().orc_pair_barrier(kind, _p(x), dhat, kappa, float(eps_x), int(project), _p(E), _p(g), _p(H))
    return bool(act), E[0], g, H.reshape(12, 12)


def ee_cross2(x12):
    return lib().orc_ee_cross2(_p(_f64(x12, 12)))


def ee_mollifier(c, eps_x):
    dm = C.c_double()
    d2m = C.c_double()
    m = lib().orc_ee_mollifier(float(c), float(eps_x), C.byref(dm), C.byref(d2m))
    return m, dm.value, d2m.value


def ortho(q12, kappa, vol):
    q = _f64(q12, 12)
    g = np.zeros(12)
    H = np.zeros(144)
    V = lib().orc_ortho(_p(q), kappa, vol, _p(g), _p(H))
    return V, g, H.reshape(12, 12)


def sym_eig(A):
    A = _f64(A)
    n = A.shape[0]
    w = np.zeros(n)
    V = np.zeros(n * n)
    lib().orc_sym_eig(n, _p(A), _p(w), _p(V))
    return w, V.reshape(n, n)


def project_psd(A):
    A = _f64(A).copy()
    lib().orc_project_psd(A.shape[0], _p(A))
    return A


def accd(kind, x12, dx12, s=0.1, tmax=1.0, max_iter=10000):
    x, dx = _f64(x12, 12), _f64(dx12, 12)
    t = np.zeros(1)
    st = lib().orc_accd(kind, _p(x), _p(dx), s, tmax, max_iter, _p(t))
    return t[0], st


def ldl_solve(A, b):
    """x = A^-1 b for a symmetric (possibly indefinite) A by the LDL^T
    factorisation without pivoting used by the adjoint's dense solve;
    returns (status, x), status -1 on a zero pivot"""
    A = _f64(A)
    n = A.shape[0]
    b = _f64(b, n)
    x = np.zeros(n)
    r = lib().orc_ldl_solve(n, _p(A), _p(b), _p(x))
    return r, x


def closest_weights(kind, x12):
    """(d2, type, gamma): the friction closest-point weights of a pair"""
    x = _f64(x12, 12)
    ga = np.zeros(4)
    t = C.c_int()
    d2 = lib().orc_closest_weights(int(kind), _p(x), _p(ga), C.byref(t))
    return d2, t.value, ga


def friction_pair(x12, gamma, n, r, mu_lambda, eps):
    x = _f64(x12, 12)
    ga, nn, rr = _f64(gamma, 4), _f64(n, 3), _f64(r, 3)
    g = np.zeros(12)
    H = np.zeros(144)
    e = lib().orc_friction_pair(_p(x), _p(ga), _p(nn), _p(rr), mu_lambda, eps, _p(g), _p(H))
    return e, g, H.reshape(12, 12)


# ---------------------------------------------------------------------------
# scene context
# ---------------------------------------------------------------------------

class Oracle:
    """One scene in the oracle.  ``scene`` is a ``paper_2201_10022_gb300.scenes.Scene``."""

    def __init__(self, scene, newton_tol=None, newton_rel=1e-9, ls_slack_rel=1e-12, cg_tol=1e-12,
                 ccd_s=0.1, newton_max=100, ls_max=30, ccd_max=10000, cg_max=20000, dense_max_dof=3000):
        L = lib()
        self.scene = scene
        self._keep = [np.ascontiguousarray(scene.xbar, dtype=np.float64),
                      np.ascontiguousarray(scene.tri, dtype=np.int32),
                      np.ascontiguousarray(scene.edge, dtype=np.int32),
                      np.ascontiguousarray(scene.vbody, dtype=np.int32),
                      np.ascontiguousarray(scene.density, dtype=np.float64),
                      np.ascontiguousarray(scene.kappa_body, dtype=np.float64),
                      np.ascontiguousarray(scene.is_static, dtype=np.uint8)]
        prm = scene.params
        s = _Scene()
        s.nb, s.nv, s.nt, s.ne = scene.nb, scene.nv, scene.nt, scene.ne
        s.xbar, s.tri, s.edge, s.vbody, s.density, s.kappa_body, s.is_static = [_p(a) for a in self._keep]
        s.dt, s.dhat, s.kappa = prm["dt"], prm["dhat"], prm["kappa"]
        s.gravity[:] = list(prm["gravity"])
        s.mu, s.eps_v = prm.get("mu", 0.0), prm.get("eps_v", 1e-3)
        s.newton_tol = 0.0
        s.ls_slack_rel, s.cg_tol, s.ccd_s = ls_slack_rel, cg_tol, ccd_s
        s.newton_max, s.ls_max, s.ccd_max, s.cg_max, s.dense_max_dof = newton_max, ls_max, ccd_max, cg_max, dense_max_dof
        self._s = s
        self.ctx = L.orc_create(C.byref(s))
        if not self.ctx:
            raise ValueError("oracle: vertices/triangles/edges must be grouped by body in body order")
        self.nb = scene.nb
        self.set_state(scene.q0, scene.qdot0)
        if newton_tol is None:
            x = self.vertices(scene.q0)
            dyn = scene.is_static[scene.vbody] == 0
            ext = x[dyn].max(axis=0) - x[dyn].min(axis=0)
            self.l_bbox = float(np.sqrt((ext * ext).sum()))
            newton_tol = newton_rel * self.l_bbox
        self.newton_tol = newton_tol
        self._s.newton_tol = newton_tol
        L.orc_destroy(self.ctx)
        self.ctx = L.orc_create(C.byref(self._s))
        self.set_state(scene.q0, scene.qdot0)

    def __del__(self):
        if getattr(self, "ctx", None) and _lib is not None:
            _lib.orc_destroy(self.ctx)
            self.ctx = None

    # state ---------------------------------------------------------------
    def set_state(self, q, qdot):
        q = _f64(q, 12 * self.nb)
        qd = _f64(qdot, 12 * self.nb)
        lib().orc_set_state(self.ctx, _p(q), _p(qd))

    def get_state(self):
        q = np.zeros(12 * self.nb)
        qd = np.zeros(12 * self.nb)
        lib().orc_get_state(self.ctx, _p(q), _p(qd))
        return q.reshape(-1, 12), qd.reshape(-1, 12)

    def qtilde(self):
        q = np.zeros(12 * self.nb)
        lib().orc_get_qtilde(self.ctx, _p(q))
        return q.reshape(-1, 12)

    # Sec. 3 ----------------------------------------------------------------
    def moments(self, b):
        vol = np.zeros(1)
        m1 = np.zeros(3)
        S = np.zeros(9)
        lib().orc_body_moments(self.ctx, b, _p(vol), _p(m1), _p(S))
        return vol[0], m1, S.reshape(3, 3)

    def mass_matrix(self, b):
        M = np.zeros(144)
        lib().orc_mass_matrix(self.ctx, b, _p(M))
        return M.reshape(12, 12)

    def vertices(self, q):
        q = _f64(q, 12 * self.nb)
        x = np.zeros(3 * self.scene.nv)
        lib().orc_vertices(self.ctx, _p(q), _p(x))
        return x.reshape(-1, 3)

    def displacements(self, dq):
        return self.vertices(dq)

    # candidate sets ---------------------------------------------------------
    def candidates(self, x0, x1=None, brute=False):
        x0 = _f64(x0)
        x1a = None if x1 is None else _f64(x1)
        L = lib()
        n = L.orc_candidates(self.ctx, _p(x0), None if x1a is None else _p(x1a), int(brute), None, None, None, 0)
        kind = np.zeros(max(n, 1), np.int32)
        pi = np.zeros(max(n, 1), np.int32)
        pj = np.zeros(max(n, 1), np.int32)
        L.orc_candidates(self.ctx, _p(x0), None if x1a is None else _p(x1a), int(brute), _p(kind), _p(pi), _p(pj), n)
        return np.stack([kind[:n], pi[:n], pj[:n]], axis=1)

    # IP ----------------------------------------------------------------------
    def energy_grad_hess(self, q, project=True):
        q = _f64(q, 12 * self.nb)
        E = np.zeros(5)
        g = np.zeros(12 * self.nb)
        st = lib().orc_energy_grad_hess(self.ctx, _p(q), _p(E), _p(g), int(project))
        return st, E, g.reshape(-1, 12)

    def energy(self, q):
        q = _f64(q, 12 * self.nb)
        return lib().orc_energy(self.ctx, _p(q))

    def active_pairs(self, q):
        """active pairs at q by canonical distance (no derivatives)"""
        q = _f64(q, 12 * self.nb)
        L = lib()
        n = L.orc_active_pairs(self.ctx, _p(q), None, None, None, None, None, 0)
        m = max(n, 1)
        kind, pi, pj, ty = (np.zeros(m, np.int32) for _ in range(4))
        d2 = np.zeros(m)
        L.orc_active_pairs(self.ctx, _p(q), _p(kind), _p(pi), _p(pj), _p(ty), _p(d2), n)
        return dict(kind=kind[:n], i=pi[:n], j=pj[:n], type=ty[:n], val=d2[:n])

    def grad_rows(self, q, bodies):
        """gradient rows of the selected bodies (body terms + every contact
        term touching them)"""
        q = _f64(q, 12 * self.nb)
        sel = np.ascontiguousarray(bodies, dtype=np.int32)
        out = np.zeros((len(sel), 12))
        st = lib().orc_grad_rows(self.ctx, _p(q), len(sel), _p(sel), _p(out))
        return st, out

    def hessian(self):
        L = lib()
        n = L.orc_hess_nblocks(self.ctx)
        diag = np.zeros((self.nb, 12, 12))
        bp = np.zeros((max(n, 1), 2), np.int32)
        blocks = np.zeros((max(n, 1), 12, 12))
        L.orc_hess_copy(self.ctx, _p(diag), _p(bp), _p(blocks))
        return diag, bp[:n], blocks[:n]

    def pairs(self, which=1):
        """which: 0 candidates, 1 active (with type and d^2), 2 friction (type, mu*lambda)"""
        L = lib()
        n = L.orc_pairs_count(self.ctx, which)
        m = max(n, 1)
        kind, pi, pj, ty = (np.zeros(m, np.int32) for _ in range(4))
        d2 = np.zeros(m)
        L.orc_pairs_copy(self.ctx, which, _p(kind), _p(pi), _p(pj), _p(ty), _p(d2))
        return dict(kind=kind[:n], i=pi[:n], j=pj[:n], type=ty[:n], val=d2[:n])

    def friction_records(self):
        """lagged friction records (order of pairs(2)): gamma (n x 4), unit
        normal (n x 3), lagged offset r (n x 3)"""
        L = lib()
        n = L.orc_pairs_count(self.ctx, 2)
        m = max(n, 1)
        ga, nn, rr = np.zeros((m, 4)), np.zeros((m, 3)), np.zeros((m, 3))
        L.orc_friction_copy(self.ctx, _p(ga), _p(nn), _p(rr))
        return ga[:n], nn[:n], rr[:n]

    def dense_hessian(self):
        diag, bp, blocks = self.hessian()
        n = 12 * self.nb
        H = np.zeros((n, n))
        for b in range(self.nb):
            H[12 * b:12 * b + 12, 12 * b:12 * b + 12] = diag[b]
        for (a, b), B in zip(bp, blocks):
            H[12 * a:12 * a + 12, 12 * b:12 * b + 12] = B
            H[12 * b:12 * b + 12, 12 * a:12 * a + 12] = B.T
        return H

    def solve(self, rhs):
        rhs = _f64(rhs, 12 * self.nb)
        dq = np.zeros(12 * self.nb)
        it = C.c_int()
        st = lib().orc_solve(self.ctx, _p(rhs), _p(dq), C.byref(it))
        return st, dq.reshape(-1, 12), it.value

    def ccd_toi(self, q, dq):
        q, dq = _f64(q, 12 * self.nb), _f64(dq, 12 * self.nb)
        t = np.zeros(1)
        st = lib().orc_ccd_toi(self.ctx, _p(q), _p(dq), _p(t))
        return st, t[0]

    def adjoint_step(self, q_t, qdot_t, q_next, rhs):
        """one step backwards (implicit function theorem): returns (status,
        M lam, dL/dkappa) with H(q_next) lam = rhs, H the unprojected Hessian
        of the step that started at (q_t, qdot_t); leaves the state there"""
        n = 12 * self.nb
        args = [_f64(a, n) for a in (q_t, qdot_t, q_next, rhs)]
        Mlam = np.zeros(n)
        gk = np.zeros(self.nb)
        st = lib().orc_adjoint_step(self.ctx, *[_p(a) for a in args], _p(Mlam), _p(gk))
        return st, Mlam.reshape(-1, 12), gk

    def step(self, n=1):
        st = Stats()
        r = lib().orc_step(self.ctx, n, C.byref(st))
        return r, st.as_dict()
