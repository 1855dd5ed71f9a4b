"""Seeded synthetic scenes for the affine-body time step.

This module only builds inputs: closed triangle meshes in each body's rest
frame, body layouts, initial affine coordinates ``q = (p, a1, a2, a3)`` with
the rows of ``A`` stored in row order (Sec. 3, Eq. kinematic) and initial
velocities.  It holds none of the method's arithmetic (no mass integrals, no
energies, no distances): both the CUDA library and the CPU oracle derive every
physical quantity from these arrays on their own.

Scene recipes (the paper's meshes are not available, so these stand in for its
workloads; every random draw comes from ``numpy.random.default_rng(seed)``):

* ``cube_stack``   2x2x2 stack of unit cubes, rotations of at most 5 degrees,
                   0.01 m gaps between the rotated cubes' world boxes, on a
                   static 10x10x1 m ground box whose top face is z = 0.
* ``ico_bowl``     icospheres (subdivision 2, radius U(0.05, 0.15) m) at
                   non-overlapping positions in the cube [-1, 1]^3, uniform
                   random orientation, velocity N(0, 0.5) m/s per component,
                   above/inside a static open bowl: the lower half (z <= 0) of
                   a radius-2 subdivision-3 icosphere.
* ``lattice_pile`` jittered nx*ny*nz lattice (pitch 1.2 m, jitter +-0.05 m) of
                   cubes (0.2 m), subdivision-1 icospheres (radius 0.1 m) and
                   1x0.2x0.2 m boxes, types uniform, uniform random
                   orientation, at rest above a static 40x40x1 m ground box.
* ``throw_stack``  cubes (0.2 m) thrown at seeded velocities into a vertical
                   stack of cubes resting on the ground.
* ``random_pair``  two or three small bodies placed close to each other with
                   random orientation; used for brute-force checks.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# meshes (rest frame, centred on the origin, outward-oriented triangles)
# ---------------------------------------------------------------------------


def _orient_outward(verts: np.ndarray, tris: np.ndarray) -> np.ndarray:
    """Flip triangles of a star-shaped closed mesh so their normals point away
    from the origin."""
    out = tris.copy()
    a, b, c = verts[out[:, 0]], verts[out[:, 1]], verts[out[:, 2]]
    n = np.cross(b - a, c - a)
    flip = np.einsum("ij,ij->i", n, (a + b + c) / 3.0) < 0
    out[flip] = out[flip][:, [0, 2, 1]]
    return out


def box_mesh(ax: float, ay: float, az: float):
    """Axis-aligned box with edge lengths (ax, ay, az): 8 vertices, 12 triangles."""
    hx, hy, hz = 0.5 * ax, 0.5 * ay, 0.5 * az
    v = np.array([[sx * hx, sy * hy, sz * hz]
                  for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)], dtype=np.float64)
    # vertex index = 4*ix + 2*iy + iz
    quads = [(0, 1, 3, 2), (4, 6, 7, 5),  # x = -, x = +
             (0, 4, 5, 1), (2, 3, 7, 6),  # y = -, y = +
             (0, 2, 6, 4), (1, 5, 7, 3)]  # z = -, z = +
    t = []
    for q0, q1, q2, q3 in quads:
        t.append((q0, q1, q2))
        t.append((q0, q2, q3))
    return v, _orient_outward(v, np.array(t, dtype=np.int32))


def cube_mesh(edge: float = 1.0):
    return box_mesh(edge, edge, edge)


def icosphere_mesh(subdiv: int, radius: float = 1.0):
    """Icosphere: V = 10*4^s + 2, F = 20*4^s."""
    g = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(-1, g, 0), (1, g, 0), (-1, -g, 0), (1, -g, 0),
         (0, -1, g), (0, 1, g), (0, -1, -g), (0, 1, -g),
         (g, 0, -1), (g, 0, 1), (-g, 0, -1), (-g, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
         (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
         (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
         (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    faces = list(f)
    for _ in range(subdiv):
        cache: dict[tuple[int, int], int] = {}

        def mid(i: int, j: int) -> int:
            key = (min(i, j), max(i, j))
            if key not in cache:
                m = verts[i] + verts[j]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    vv = np.array(verts, dtype=np.float64) * radius
    return vv, _orient_outward(vv, np.array(faces, dtype=np.int32))


def bowl_mesh(radius: float = 2.0, subdiv: int = 3):
    """Open hemispherical shell: the faces of an icosphere whose centroid has
    z < 0, with unused vertices dropped."""
    v, t = icosphere_mesh(subdiv, radius)
    cz = v[t].mean(axis=1)[:, 2]
    t = t[cz < 0.0]
    used = np.unique(t)
    remap = -np.ones(len(v), dtype=np.int64)
    remap[used] = np.arange(len(used))
    return v[used].copy(), remap[t].astype(np.int32)


def mesh_edges(tris: np.ndarray) -> np.ndarray:
    """Unique undirected edges (i < j) of a triangle list, sorted."""
    e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]])
    e = np.sort(e, axis=1)
    return np.unique(e, axis=0).astype(np.int32)


# ---------------------------------------------------------------------------
# rotations
# ---------------------------------------------------------------------------


def quat_to_mat(w, x, y, z) -> np.ndarray:
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ], dtype=np.float64)


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform on SO(3) (normalised Gaussian quaternion)."""
    qv = rng.normal(size=4)
    qv /= np.linalg.norm(qv)
    return quat_to_mat(*qv)


def small_rotation(rng: np.random.Generator, max_deg: float) -> np.ndarray:
    """Rotation about a uniform random axis by an angle uniform in
    [-max_deg, max_deg] degrees."""
    axis = rng.normal(size=3)
    axis /= np.linalg.norm(axis)
    ang = math.radians(rng.uniform(-max_deg, max_deg))
    s = math.sin(0.5 * ang)
    return quat_to_mat(math.cos(0.5 * ang), *(s * axis))


# ---------------------------------------------------------------------------
# scene container
# ---------------------------------------------------------------------------

DEFAULT_PARAMS = dict(dt=0.01, dhat=1e-3, kappa=1e8, gravity=(0.0, 0.0, -9.8),
                      mu=0.0, eps_v=1e-3)


@dataclass
class Scene:
    """SoA scene arrays.  Vertices, triangles and edges are grouped by body in
    body order; ``tri``/``edge`` hold global vertex indices."""
    name: str
    xbar: np.ndarray        # (nv, 3) float64, rest-frame positions
    tri: np.ndarray         # (nt, 3) int32
    edge: np.ndarray        # (ne, 2) int32
    vbody: np.ndarray       # (nv,) int32
    q0: np.ndarray          # (nb, 12) float64: p, then rows of A
    qdot0: np.ndarray       # (nb, 12) float64
    density: np.ndarray     # (nb,) float64
    kappa_body: np.ndarray  # (nb,) float64, orthogonality stiffness per body
    is_static: np.ndarray   # (nb,) uint8
    params: dict = field(default_factory=lambda: dict(DEFAULT_PARAMS))
    seed: int = 0

    @property
    def nb(self) -> int:
        return len(self.q0)

    @property
    def nv(self) -> int:
        return len(self.xbar)

    @property
    def nt(self) -> int:
        return len(self.tri)

    @property
    def ne(self) -> int:
        return len(self.edge)


class _Builder:
    def __init__(self, name: str, seed: int):
        self.name, self.seed = name, seed
        self.xbar, self.tri, self.edge, self.vbody = [], [], [], []
        self.q0, self.qdot0, self.density, self.kappa, self.static = [], [], [], [], []
        self.nv = 0

    def add(self, verts, tris, R=None, p=(0, 0, 0), v=(0, 0, 0), density=1000.0,
            kappa=1e8, static=False, edges=None):
        b = len(self.q0)
        R = np.eye(3) if R is None else np.asarray(R, dtype=np.float64)
        self.xbar.append(np.asarray(verts, dtype=np.float64))
        self.tri.append(np.asarray(tris, dtype=np.int32) + self.nv)
        self.edge.append((mesh_edges(np.asarray(tris)) if edges is None else edges) + self.nv)
        self.vbody.append(np.full(len(verts), b, dtype=np.int32))
        q = np.zeros(12)
        q[:3] = p
        q[3:] = R.reshape(-1)  # rows of A in row order
        qd = np.zeros(12)
        qd[:3] = v
        self.q0.append(q)
        self.qdot0.append(qd)
        self.density.append(density)
        self.kappa.append(kappa)
        self.static.append(1 if static else 0)
        self.nv += len(verts)
        return b

    def build(self, params=None) -> Scene:
        prm = dict(DEFAULT_PARAMS)
        if params:
            prm.update(params)
        return Scene(self.name,
                     np.ascontiguousarray(np.concatenate(self.xbar)),
                     np.ascontiguousarray(np.concatenate(self.tri).astype(np.int32)),
                     np.ascontiguousarray(np.concatenate(self.edge).astype(np.int32)),
                     np.ascontiguousarray(np.concatenate(self.vbody)),
                     np.ascontiguousarray(np.array(self.q0)),
                     np.ascontiguousarray(np.array(self.qdot0)),
                     np.array(self.density, dtype=np.float64),
                     np.array(self.kappa, dtype=np.float64),
                     np.array(self.static, dtype=np.uint8), prm, self.seed)


def _rotated_half_extent(verts: np.ndarray, R: np.ndarray) -> np.ndarray:
    return np.abs(verts @ R.T).max(axis=0)


# ---------------------------------------------------------------------------
# scene recipes
# ---------------------------------------------------------------------------


def cube_stack(seed: int = 1, n: int = 2, gap: float = 0.01, max_deg: float = 5.0,
               **params) -> Scene:
    rng = np.random.default_rng(seed)
    B = _Builder("cube_stack", seed)
    gv, gt = box_mesh(10.0, 10.0, 1.0)
    B.add(gv, gt, p=(0.0, 0.0, -0.5), static=True)
    cv, ct = cube_mesh(1.0)
    rots = [small_rotation(rng, max_deg) for _ in range(n ** 3)]
    h = np.max([_rotated_half_extent(cv, R) for R in rots], axis=0)
    pitch = 2.0 * h + gap
    k = 0
    for iz in range(n):
        for iy in range(n):
            for ix in range(n):
                p = ((ix - 0.5 * (n - 1)) * pitch[0], (iy - 0.5 * (n - 1)) * pitch[1],
                     gap + h[2] + iz * pitch[2])
                B.add(cv, ct, R=rots[k], p=p)
                k += 1
    return B.build(params)


def ico_bowl(seed: int = 2, n: int = 512, subdiv: int = 2, rmin: float = 0.05,
             rmax: float = 0.15, half: float = 1.0, bowl_radius: float = 2.0,
             vel_std: float = 0.5, gap: float = 0.01, **params) -> Scene:
    rng = np.random.default_rng(seed)
    B = _Builder("ico_bowl", seed)
    bv, bt = bowl_mesh(bowl_radius, 3)
    B.add(bv, bt, static=True)
    unit_v, unit_t = icosphere_mesh(subdiv, 1.0)
    centres, radii = [], []
    tries = 0
    while len(centres) < n:
        tries += 1
        if tries > 2_000_000:
            raise RuntimeError("ico_bowl: could not place spheres")
        r = rng.uniform(rmin, rmax)
        c = rng.uniform(-half + r, half - r, size=3)
        if np.linalg.norm(c) + r > bowl_radius - 0.05:
            continue
        if centres:
            d = np.linalg.norm(np.array(centres) - c, axis=1) - np.array(radii) - r
            if d.min() < gap:
                continue
        centres.append(c)
        radii.append(r)
    for c, r in zip(centres, radii):
        R = random_rotation(rng)
        v = rng.normal(0.0, vel_std, size=3)
        B.add(unit_v * r, unit_t, R=R, p=c, v=v)
    return B.build(params)


def lattice_pile(seed: int = 3, nx: int = 25, ny: int = 20, nz: int = 20, pitch: float = 1.2,
                 jitter: float = 0.05, z0: float = 0.6, ground: float = 40.0,
                 types=("cube", "ico1", "box"), **params) -> Scene:
    rng = np.random.default_rng(seed)
    B = _Builder("lattice_pile", seed)
    gv, gt = box_mesh(ground, ground, 1.0)
    B.add(gv, gt, p=(0.0, 0.0, -0.5), static=True)
    meshes = {"cube": cube_mesh(0.2), "ico1": icosphere_mesh(1, 0.1),
              "box": box_mesh(1.0, 0.2, 0.2), "ico2": icosphere_mesh(2, 0.1)}
    for iz in range(nz):
        for iy in range(ny):
            for ix in range(nx):
                kind = types[int(rng.integers(len(types)))]
                R = random_rotation(rng)
                p = np.array([(ix - 0.5 * (nx - 1)) * pitch, (iy - 0.5 * (ny - 1)) * pitch,
                              z0 + iz * pitch]) + rng.uniform(-jitter, jitter, size=3)
                v, t = meshes[kind]
                B.add(v, t, R=R, p=p)
    prm = dict(mu=0.3, eps_v=1e-3)
    prm.update(params)
    return B.build(prm)


def throw_stack(seed: int = 4, n_throw: int = 64, n_stack: int = 10, edge: float = 0.2,
                **params) -> Scene:
    rng = np.random.default_rng(seed)
    B = _Builder("throw_stack", seed)
    gv, gt = box_mesh(20.0, 20.0, 1.0)
    B.add(gv, gt, p=(0.0, 0.0, -0.5), static=True)
    cv, ct = cube_mesh(edge)
    for k in range(n_stack):
        B.add(cv, ct, p=(0.0, 0.0, 0.5 * edge + 0.005 + k * (edge + 0.005)))
    side = int(round(n_throw ** (1.0 / 3.0)))
    assert side ** 3 == n_throw
    pitch = 1.6 * edge
    base = np.array([-3.0, -0.5 * (side - 1) * pitch, 0.5])
    for iz in range(side):
        for iy in range(side):
            for ix in range(side):
                p = base + np.array([ix * pitch, iy * pitch, iz * pitch])
                R = small_rotation(rng, 30.0)
                v = np.array([rng.uniform(4.0, 6.0), rng.normal(0.0, 0.3), rng.uniform(1.0, 2.5)])
                B.add(cv, ct, R=R, p=p, v=v)
    return B.build(params)


def packed_cubes(seed: int = 6, nx: int = 22, ny: int = 22, nz: int = 21, edge: float = 0.2,
                 gap: float = 0.9999e-3, max_deg: float = 1e-4, **params) -> Scene:
    """Contact-dense block of cubes: neighbouring faces `gap` apart (just
    below d-hat = 1e-3, where the barrier force is of the order of the
    weight, so the block starts close to rest), tiny seeded rotations, on a
    static ground box.  Every face-to-face neighbour pair carries active
    point-triangle and edge-edge terms from the first iteration."""
    rng = np.random.default_rng(seed)
    B = _Builder("packed_cubes", seed)
    pitch = edge + gap
    ground = max(nx, ny) * pitch + 2.0
    gv, gt = box_mesh(ground, ground, 1.0)
    B.add(gv, gt, p=(0.0, 0.0, -0.5), static=True)
    cv, ct = cube_mesh(edge)
    for iz in range(nz):
        for iy in range(ny):
            for ix in range(nx):
                p = ((ix - 0.5 * (nx - 1)) * pitch, (iy - 0.5 * (ny - 1)) * pitch, gap + 0.5 * edge + iz * pitch)
                B.add(cv, ct, R=small_rotation(rng, max_deg), p=p)
    prm = dict(mu=0.3, eps_v=1e-3)
    prm.update(params)
    return B.build(prm)


def random_pair(seed: int, kinds=("cube", "ico1"), sep: float = 0.0005, **params) -> Scene:
    """Two bodies, the second placed so that its closest approach to the first
    is a few d-hat; random orientations."""
    rng = np.random.default_rng(seed)
    B = _Builder("random_pair", seed)
    meshes = {"cube": cube_mesh(0.2), "ico1": icosphere_mesh(1, 0.1), "ico2": icosphere_mesh(2, 0.1),
              "box": box_mesh(1.0, 0.2, 0.2), "tet": icosphere_mesh(0, 0.1)}
    v0, t0 = meshes[kinds[0]]
    v1, t1 = meshes[kinds[1 % len(kinds)]]
    R0, R1 = random_rotation(rng), random_rotation(rng)
    B.add(v0, t0, R=R0, p=(0.0, 0.0, 0.0))
    # support points along a random direction n: the bodies are convex, so
    # putting body 1's lowest point along n at `sep` beyond body 0's highest
    # point makes `sep` their distance
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    w0 = v0 @ R0.T
    w1 = v1 @ R1.T
    s0 = w0[np.argmax(w0 @ n)]
    s1 = w1[np.argmin(w1 @ n)]
    p1 = s0 + sep * n - s1
    B.add(v1, t1, R=R1, p=p1)
    return B.build(params)


def scene_batch(seed: int = 5, n_scenes: int = 256, nmin: int = 16, nmax: int = 2048, pitch: float = 0.5,
                jitter: float = 0.05, z0: float = 0.3, vel_sigma: float = 0.5, ground: float = 40.0,
                types=("cube", "ico2"), **params) -> list:
    """Independent scenes of uneven size: per scene a body count N drawn
    log-uniformly from [nmin, nmax], then the lattice-pile layout (jittered
    lattice, uniform rotations, bottom layers filled first) of N bodies of the
    given types (0.2 m cubes, radius-0.1 m icospheres) over a static ground,
    with translational velocities N(0, vel_sigma) per component.  Scene k
    draws from the generator seeded (seed, k).  The pitch clears the largest
    rotated extent (cube half-diagonal 0.173 m) plus the jitter on both
    sides, so no pair starts closer than d-hat."""
    meshes = {"cube": cube_mesh(0.2), "ico1": icosphere_mesh(1, 0.1), "ico2": icosphere_mesh(2, 0.1)}
    edges = {k: mesh_edges(np.asarray(t)) for k, (_, t) in meshes.items()}
    gv, gt = box_mesh(ground, ground, 1.0)
    out = []
    for k in range(n_scenes):
        rng = np.random.default_rng([seed, k])
        n = int(round(np.exp(rng.uniform(np.log(nmin), np.log(nmax)))))
        nz = max(1, int(np.ceil(n ** (1.0 / 3.0))))
        nx = int(np.ceil(np.sqrt(n / nz)))
        ny = int(np.ceil(n / (nx * nz)))
        B = _Builder(f"scene_batch_{k}", seed)
        B.add(gv, gt, p=(0.0, 0.0, -0.5), static=True)
        placed = 0
        for iz in range(nz):
            for iy in range(ny):
                for ix in range(nx):
                    if placed == n:
                        break
                    kind = types[int(rng.integers(len(types)))]
                    R = random_rotation(rng)
                    p = np.array([(ix - 0.5 * (nx - 1)) * pitch, (iy - 0.5 * (ny - 1)) * pitch,
                                  z0 + iz * pitch]) + rng.uniform(-jitter, jitter, size=3)
                    v = rng.normal(0.0, vel_sigma, size=3)
                    verts, tris = meshes[kind]
                    B.add(verts, tris, R=R, p=p, v=v, edges=edges[kind])
                    placed += 1
        prm = dict(mu=0.0)
        prm.update(params)
        out.append(B.build(prm))
    return out


RECIPES = {
    "packed_cubes": packed_cubes,
    "cube_stack": cube_stack,
    "ico_bowl": ico_bowl,
    "lattice_pile": lattice_pile,
    "throw_stack": throw_stack,
}


def make_scene(name: str, **kw) -> Scene:
    """Scene of the named recipe (packed_cubes, cube_stack, ico_bowl,
    lattice_pile, throw_stack); keyword arguments shrink it."""
    return RECIPES[name](**kw)
