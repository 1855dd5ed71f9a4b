"""i-AABB culling counters (Sec. 4.2) of the candidate enumeration: the
primitive pairs of the body pairs equal a host count over the body pairs
whose d-hat-dilated boxes overlap, the candidates equal the oracle's, and the
restriction to the other body's box lies between them."""
import numpy as np
import pytest

import oracle as O
from paper_2201_10022_gb300 import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def abd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_10022_gb300 import abd as A
    A.load()
    return A


def _prim_counts(s):
    nv = np.bincount(s.vbody, minlength=s.nb)
    nt = np.bincount(s.vbody[s.tri[:, 0]], minlength=s.nb)
    ne = np.bincount(s.vbody[s.edge[:, 0]], minlength=s.nb)
    return nv, nt, ne


def _body_pair_prims(s, x, dhat):
    lo = np.full((s.nb, 3), np.inf)
    hi = np.full((s.nb, 3), -np.inf)
    np.minimum.at(lo, s.vbody, x)
    np.maximum.at(hi, s.vbody, x)
    nv, nt, ne = _prim_counts(s)
    tot = 0
    for a in range(s.nb):
        for b in range(a + 1, s.nb):
            if s.is_static[a] and s.is_static[b]:
                continue
            if ((lo[a] - hi[b]) <= dhat).all() and ((lo[b] - hi[a]) <= dhat).all():
                tot += int(nv[a] * nt[b] + nv[b] * nt[a] + ne[a] * ne[b])
    return tot


@pytest.mark.parametrize("name", ["stack", "packed", "pair"])
def test_culling_counters(abd, name):
    if name == "stack":
        s = scenes.cube_stack(seed=1, gap=0.0004)
    elif name == "packed":
        s = scenes.packed_cubes(nx=3, ny=3, nz=2)
    else:
        s = scenes.random_pair(1, kinds=("ico1", "box"), sep=0.0003)
    orc = O.Oracle(s)
    g = abd.AbdScene(s)
    q = torch.tensor(s.q0)
    g.energy_grad_hess(q)  # buffers grown
    c0 = g.counters()
    _, _, cnt = g.energy_grad_hess(q)
    c1 = g.counters()
    body = c1["prim_pairs_body"] - c0["prim_pairs_body"]
    iaabb = c1["prim_pairs_iaabb"] - c0["prim_pairs_iaabb"]
    cand = c1["prim_pairs_cand"] - c0["prim_pairs_cand"]
    st, _, _ = orc.energy_grad_hess(s.q0.reshape(-1))
    assert st == 0
    x = orc.vertices(s.q0.reshape(-1)).reshape(-1, 3)
    assert body == _body_pair_prims(s, x, s.params["dhat"])
    assert cand == cnt["n_candidates"] == orc.pairs(0)["kind"].size
    assert cand <= iaabb < body
