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
