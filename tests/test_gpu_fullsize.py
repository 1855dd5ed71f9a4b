"""Full-size parity (10,165 bodies, about 2.7 million active pairs): the
contact-dense packed block of cubes, through the C ABI.  Candidate and
active sets (with distance types and squared distances) bit-exact against
the oracle, total energy within 1e-10, gradient rows of sampled bodies
within 1e-10 of the largest row entry."""
import numpy as np
import pytest

import oracle as O
from paper_2201_10022_gb300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_packed_block_full_size():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_10022_gb300 import abd as A
    s = scenes.packed_cubes()
    assert s.nb > 10000
    gpu = A.AbdScene(s)
    orc = O.Oracle(s)
    q = s.q0
    E, g, cnt = gpu.energy_grad_hess(torch.tensor(q))
    assert cnt["n_active"] > 2_000_000
    # active set, types and d^2: bit-exact
    ag = gpu.pairs(1)
    ao = orc.active_pairs(q.reshape(-1))
    kg = np.stack([ag["kind"], ag["i"], ag["j"], ag["type"]], 1)
    ko = np.stack([ao["kind"], ao["i"], ao["j"], ao["type"]], 1)
    og, oo = np.lexsort(kg.T[::-1]), np.lexsort(ko.T[::-1])
    np.testing.assert_array_equal(kg[og], ko[oo])
    np.testing.assert_array_equal(ag["val"][og], ao["val"][oo])
    # candidate set: bit-exact
    cg = gpu.pairs(0)
    co = orc.candidates(orc.vertices(q.reshape(-1)))
    kc = np.stack([cg["kind"], cg["i"], cg["j"]], 1)
    assert kc.shape == co.shape
    np.testing.assert_array_equal(kc[np.lexsort(kc.T[::-1])], co[np.lexsort(co.T[::-1])])
    # total energy and sampled gradient rows
    Eo = orc.energy(q.reshape(-1))
    assert E[0] == pytest.approx(Eo, rel=1e-10)
    rng = np.random.default_rng(0)
    sel = np.sort(rng.choice(np.nonzero(s.is_static == 0)[0], 24, replace=False))
    st, rows = orc.grad_rows(q.reshape(-1), sel)
    assert st == 0
    gg = g.cpu().numpy()[sel]
    assert np.abs(gg - rows).max() <= 1e-10 * np.abs(rows).max()
