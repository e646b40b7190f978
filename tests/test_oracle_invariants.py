"""Closed forms and invariants of the exact squared EDT, checked on the oracle."""
import numpy as np
import pytest

import oracle
from brute import INF32, feature_valid, sources


@pytest.mark.parametrize("shape", [(9, 10), (1, 17), (23, 1), (31, 40)])
def test_single_source_closed_form(shape):
    rng = np.random.default_rng(11)
    for _ in range(5):
        q = tuple(int(rng.integers(0, n)) for n in shape)
        m = np.zeros(shape, np.uint8)
        m[q] = 1
        D, F = oracle.edt(m)
        yy, xx = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), indexing="ij")
        np.testing.assert_array_equal(D, (yy - q[0]) ** 2 + (xx - q[1]) ** 2)


def test_single_voxel_closed_form_3d():
    m = np.zeros((6, 7, 8), np.uint8)
    m[2, 5, 1] = 1
    D, F = oracle.edt(m)
    z, y, x = np.meshgrid(np.arange(6), np.arange(7), np.arange(8), indexing="ij")
    np.testing.assert_array_equal(D, (z - 2) ** 2 + (y - 5) ** 2 + (x - 1) ** 2)
    assert np.all(F == 2 * 56 + 5 * 8 + 1)


@pytest.mark.parametrize("n", [1, 2, 5, 64, 301])
def test_one_row_is_1d_definition(n):
    """H = 1: D(j) = min over sources k of (j - k)^2."""
    rng = np.random.default_rng(n)
    m = (rng.random((1, n)) < 0.1).astype(np.uint8)
    if m.sum() == 0:
        m[0, n // 2] = 1
    D, F = oracle.edt(m)
    ks = np.nonzero(m[0])[0]
    j = np.arange(n)
    np.testing.assert_array_equal(D[0], ((j[:, None] - ks[None, :]) ** 2).min(1))
    Dt, _ = oracle.edt(m.T.copy())
    np.testing.assert_array_equal(Dt[:, 0], D[0])


def _random_mask(rng, shape, p):
    return (rng.random(shape) < p).astype(np.uint8)


@pytest.mark.parametrize("mode", [0, 1])
def test_invariants_2d(mode):
    rng = np.random.default_rng(5)
    for _ in range(30):
        H, W = rng.integers(1, 60, size=2)
        m = _random_mask(rng, (H, W), rng.choice([0.005, 0.05, 0.5]))
        D, F = oracle.edt(m, mode)
        src = sources(m, mode)
        if not src.any():
            assert np.all(D == INF32)
            continue
        assert np.all((D == 0) == src)
        assert feature_valid(m, mode, D, F)
        # every value is a sum of two squares within the image
        ys = np.arange(H)[:, None] ** 2
        xs = np.arange(W)[None, :] ** 2
        sums = set((ys + xs).reshape(-1).tolist())
        assert set(np.unique(D).tolist()) <= sums
        # 4-neighbour Lipschitz bound on the distance
        d = np.sqrt(D.astype(np.float64))
        assert np.all(np.abs(np.diff(d, axis=0)) <= 1 + 1e-12)
        assert np.all(np.abs(np.diff(d, axis=1)) <= 1 + 1e-12)
        # equivariance under flips and transposition
        np.testing.assert_array_equal(oracle.edt(m[::-1].copy(), mode)[0], D[::-1])
        np.testing.assert_array_equal(oracle.edt(m[:, ::-1].copy(), mode)[0], D[:, ::-1])
        np.testing.assert_array_equal(oracle.edt(m.T.copy(), mode)[0], D.T)
        # the two modes are complements
        np.testing.assert_array_equal(oracle.edt((m == 0).astype(np.uint8), 1 - mode)[0], D)


@pytest.mark.parametrize("mode", [0, 1])
def test_invariants_3d(mode):
    rng = np.random.default_rng(6)
    for _ in range(12):
        shape = tuple(int(v) for v in rng.integers(1, 14, size=3))
        m = _random_mask(rng, shape, rng.choice([0.01, 0.1, 0.5]))
        D, F = oracle.edt(m, mode)
        src = sources(m, mode)
        if not src.any():
            continue
        assert np.all((D == 0) == src)
        assert feature_valid(m, mode, D, F)
        for axes in [(1, 0, 2), (2, 1, 0), (0, 2, 1)]:
            mt = np.ascontiguousarray(m.transpose(axes))
            np.testing.assert_array_equal(oracle.edt(mt, mode)[0], D.transpose(axes))
        np.testing.assert_array_equal(oracle.edt(np.ascontiguousarray(m[::-1]), mode)[0], D[::-1])
        d = np.sqrt(D.astype(np.float64))
        for ax in range(3):
            assert np.all(np.abs(np.diff(d, axis=ax)) <= 1 + 1e-12)
