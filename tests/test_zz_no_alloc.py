"""The allocation-free CCD entry point (for callers that cannot allocate
device memory when they need a step bound) against the scene-level
abd_ccd_toi: same swept pairs, same start positions and displacements, so
the same time of impact bit for bit, on two calls in a row (the second call
reuses the shared scratch array the first one left behind)."""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_2201_10022_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("which", ["pair", "stack"])
def test_noalloc_ccd_matches_scene_ccd(which):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_10022_gb300 import abd as A
    if which == "pair":
        s = scenes.random_pair(1, kinds=("cube", "ico1"), sep=0.0003)
    else:
        s = scenes.cube_stack(seed=1, gap=0.0004)
    rng = np.random.default_rng(5)
    dyn = s.is_static == 0
    dq = np.zeros_like(s.q0)
    dq[dyn, :3] = rng.normal(size=(dyn.sum(), 3)) * 0.02
    dq[dyn, 3:] = rng.normal(size=(dyn.sum(), 9)) * 0.001
    gpu = A.AbdScene(s)
    toi_ref = gpu.ccd_toi(torch.tensor(s.q0), torch.tensor(dq))
    # the swept pairs and the vertex trajectories, from the oracle
    orc = O.Oracle(s)
    x = orc.vertices(s.q0.reshape(-1))
    dx = orc.displacements(dq.reshape(-1))
    cand = orc.candidates(x, x + dx)
    verts = np.array([[i, *s.tri[j]] if k == 0 else [*s.edge[i], *s.edge[j]] for k, i, j in cand], dtype=np.int32)
    kinds = cand[:, 0].astype(np.uint8)
    dev = torch.device("cuda:0")
    xd = torch.tensor(x, dtype=torch.float64, device=dev).contiguous()
    dxd = torch.tensor(dx, dtype=torch.float64, device=dev).contiguous()
    vd = torch.tensor(verts, device=dev).contiguous()
    kd = torch.tensor(kinds, device=dev).contiguous()
    stream = torch.cuda.current_stream(dev).cuda_stream
    p = gpu.params
    for call in range(2):
        t = ctypes.c_double(-1.0)
        r = A.abd_ccd_toi_pairs_noalloc(xd.data_ptr(), dxd.data_ptr(), s.nv, vd.data_ptr(), kd.data_ptr(), len(cand),
                                        p.ccd_s, p.ccd_max, stream, ctypes.byref(t))
        assert r == 0, A.STATUS[r]
        assert t.value == toi_ref, (call, t.value, toi_ref)
    assert toi_ref < 1.0 or which == "pair"
    # sizes beyond the scratch array are rejected without touching the GPU
    t = ctypes.c_double()
    r = A.abd_ccd_toi_pairs_noalloc(xd.data_ptr(), dxd.data_ptr(), s.nv, vd.data_ptr(), kd.data_ptr(), 1 << 19,
                                    p.ccd_s, p.ccd_max, stream, ctypes.byref(t))
    assert A.STATUS[r] == "ABD_ERR_CAPACITY"


def test_noalloc_guards_and_status_reset():
    """The kernel's own guards: a vertex index of nv and a kind of 2 are
    reported as ABD_ERR_INVALID_ARG (each index is checked before any load
    through it); a valid call straight after returns ABD_OK, so the status
    word of the shared array was cleared; an iteration cap of 1 on a pair
    that needs more advances returns ABD_ERR_CCD_MAXITER with a time of
    impact no larger than the uncapped one."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_10022_gb300 import abd as A
    A.load()
    dev = torch.device("cuda:0")
    # one point above a triangle, moving onto it: the additive CCD needs
    # several advances to get within s of the start distance
    x = np.array([[0.2, 0.2, 0.01], [0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    dx = np.array([[0.0, 0.0, -0.02], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    xd = torch.tensor(x, dtype=torch.float64, device=dev).contiguous()
    dxd = torch.tensor(dx, dtype=torch.float64, device=dev).contiguous()
    stream = torch.cuda.current_stream(dev).cuda_stream

    def call(verts, kinds, ccd_max=10000):
        vd = torch.tensor(np.asarray(verts, np.int32).reshape(-1, 4), device=dev).contiguous()
        kd = torch.tensor(np.asarray(kinds, np.uint8), device=dev).contiguous()
        t = ctypes.c_double(-1.0)
        r = A.abd_ccd_toi_pairs_noalloc(xd.data_ptr(), dxd.data_ptr(), 4, vd.data_ptr(), kd.data_ptr(), len(kinds),
                                        0.1, ccd_max, stream, ctypes.byref(t))
        return A.STATUS[r], t.value

    st_ok, toi_ok = call([[0, 1, 2, 3]], [0])
    assert st_ok == "ABD_OK" and 0.0 < toi_ok < 1.0
    assert call([[0, 1, 2, 4]], [0])[0] == "ABD_ERR_INVALID_ARG"   # vertex index nv
    assert call([[0, 1, 2, 3]], [2])[0] == "ABD_ERR_INVALID_ARG"   # unknown kind
    assert call([[0, 1, 2, 3], [0, 1, 2, 3]], [0, 0]) == (st_ok, toi_ok)  # status cleared
    st_cap, toi_cap = call([[0, 1, 2, 3]], [0], ccd_max=1)
    assert st_cap == "ABD_ERR_CCD_MAXITER" and 0.0 <= toi_cap <= toi_ok
    assert call([[0, 1, 2, 3]], [0]) == (st_ok, toi_ok)
