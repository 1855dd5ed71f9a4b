"""Host-side parts of the many-scene form: the batch recipe (size law,
determinism, clearances) and the argument checks of abd_step_batch, which
return before any CUDA call."""
import ctypes as C

import numpy as np
import pytest

from paper_2201_10022_gb300 import abd, scenes

INVALID = {v: k for k, v in abd.STATUS.items()}["ABD_ERR_INVALID_ARG"]


def _world_boxes(s):
    q = s.q0
    A = q[:, 3:].reshape(-1, 3, 3)
    x = np.einsum("vij,vj->vi", A[s.vbody], s.xbar) + q[s.vbody, :3]
    lo = np.full((s.nb, 3), np.inf)
    hi = np.full((s.nb, 3), -np.inf)
    np.minimum.at(lo, s.vbody, x)
    np.maximum.at(hi, s.vbody, x)
    return lo, hi


def test_batch_sizes_follow_the_log_uniform_law():
    S = scenes.scene_batch(n_scenes=64, nmin=16, nmax=2048)
    n = np.array([s.nb - 1 for s in S])  # minus the ground
    assert n.min() >= 16 and n.max() <= 2048
    # log N is uniform on [ln 16, ln 2048]: its mean is their midpoint, and
    # 64 draws put the sample mean within ~4 standard errors
    u = (np.log(n) - np.log(16)) / (np.log(2048) - np.log(16))
    assert abs(u.mean() - 0.5) < 4 * np.sqrt(1 / 12 / len(u))
    assert all(s.is_static[0] == 1 and s.is_static[1:].sum() == 0 for s in S)


def test_batch_is_deterministic_per_scene_seed():
    a = scenes.scene_batch(n_scenes=3, nmax=64)
    b = scenes.scene_batch(n_scenes=5, nmax=64)
    for x, y in zip(a, b[:3]):
        assert np.array_equal(x.q0, y.q0) and np.array_equal(x.qdot0, y.qdot0) and np.array_equal(x.xbar, y.xbar)
    c = scenes.scene_batch(seed=6, n_scenes=3, nmax=64)
    assert not np.array_equal(a[0].q0, c[0].q0)


def test_batch_bodies_start_separated():
    """world boxes of distinct bodies are apart by more than d-hat on some
    axis, and every dynamic body is above the ground by more than d-hat"""
    for s in scenes.scene_batch(n_scenes=6, nmax=200):
        lo, hi = _world_boxes(s)
        dhat = s.params["dhat"]
        dyn = np.arange(1, s.nb)
        assert (lo[dyn, 2] > hi[0, 2] + dhat).all()
        gap = np.maximum(lo[dyn][:, None, :] - hi[dyn][None, :, :], lo[dyn][None, :, :] - hi[dyn][:, None, :])
        sep = gap.max(axis=2)
        np.fill_diagonal(sep, np.inf)
        assert sep.min() > dhat


def test_step_batch_argument_checks():
    L = abd.load()
    assert abd.abd_step_batch([], 1, 1, None, None) == 0  # empty batch: nothing to do
    fake = C.c_void_p(0x1000)
    assert abd.abd_step_batch([fake, fake], 1, 2, None, None) == INVALID
    assert abd.abd_step_batch([None], 1, 1, None, None) == INVALID
    assert abd.abd_step_batch([fake], 1, 0, None, None) == INVALID
    assert abd.abd_step_batch([fake], -1, 1, None, None) == INVALID
    assert L is not None
