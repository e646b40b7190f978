"""Pins the oracle to brute force (the naive search of Sec. 3) on tiny inputs."""
import itertools

import numpy as np
import pytest

import oracle
from brute import INF32, brute_edt, brute_edt_many, feature_valid


def _all_masks(H, W):
    n = H * W
    idx = np.arange(1 << n, dtype=np.int64)
    bits = (idx[:, None] >> np.arange(n)[None, :]) & 1
    return bits.astype(np.uint8).reshape(-1, H, W)


@pytest.mark.parametrize("H,W", [(4, 4), (3, 5), (2, 7), (1, 9)])
@pytest.mark.parametrize("mode", [oracle.TO_OBJECT, oracle.TO_BACKGROUND])
def test_every_small_mask(H, W, mode):
    masks = _all_masks(H, W)
    ref = brute_edt_many(masks, mode)
    for m, r in zip(masks, ref):
        D, F = oracle.edt(m, mode)
        assert np.array_equal(D, r)
        assert feature_valid(m, mode, D, F)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("mode", [oracle.TO_OBJECT, oracle.TO_BACKGROUND])
def test_random_2d_up_to_16(seed, mode):
    rng = np.random.default_rng(100 + seed)
    for _ in range(40):
        H, W = rng.integers(1, 17, size=2)
        p = rng.choice([0.02, 0.1, 0.3, 0.7, 0.95])
        m = (rng.random((H, W)) < p).astype(np.uint8)
        D, F = oracle.edt(m, mode)
        np.testing.assert_array_equal(D, brute_edt(m, mode))
        assert feature_valid(m, mode, D, F)
        Db, Fb = oracle.edt2d_basic(m, mode)
        np.testing.assert_array_equal(Db, D)
        assert feature_valid(m, mode, Db, Fb)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("mode", [oracle.TO_OBJECT, oracle.TO_BACKGROUND])
def test_random_3d_up_to_8(seed, mode):
    rng = np.random.default_rng(200 + seed)
    for _ in range(20):
        shape = tuple(int(v) for v in rng.integers(1, 9, size=3))
        p = rng.choice([0.01, 0.05, 0.2, 0.6])
        m = (rng.random(shape) < p).astype(np.uint8)
        D, F = oracle.edt(m, mode)
        np.testing.assert_array_equal(D, brute_edt(m, mode))
        assert feature_valid(m, mode, D, F)


def test_3d_slab_equals_2d():
    """A volume with one z-slice is the 2-D transform of that slice."""
    rng = np.random.default_rng(7)
    for _ in range(20):
        H, W = rng.integers(1, 20, size=2)
        m = (rng.random((H, W)) < 0.1).astype(np.uint8)
        D2, _ = oracle.edt(m)
        D3, F3 = oracle.edt(m[None])
        np.testing.assert_array_equal(D3[0], D2)


def test_no_source_gives_inf_and_minus_one():
    for shape in [(5, 7), (1, 1), (3, 4, 2)]:
        D, F = oracle.edt(np.zeros(shape, np.uint8), oracle.TO_OBJECT)
        assert np.all(D == INF32) and np.all(F == -1)
        D, F = oracle.edt(np.ones(shape, np.uint8), oracle.TO_BACKGROUND)
        assert np.all(D == INF32) and np.all(F == -1)


def test_all_sources_gives_zero_and_identity():
    for shape in [(5, 7), (1, 1), (3, 4, 2)]:
        D, F = oracle.edt(np.ones(shape, np.uint8), oracle.TO_OBJECT)
        assert np.all(D == 0)
        np.testing.assert_array_equal(F.reshape(-1), np.arange(np.prod(shape)))
