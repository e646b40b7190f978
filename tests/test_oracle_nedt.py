"""The oracle's city-block (Sec. 2.1) and chamfer 4-3 (Sec. 2.2) transforms,
pinned to the paper's worked example (Fig. 12, 13, 15; two printed cells are
typos, see the fixture headers) and to the plain definitions by brute force:
city-block = min over sources of |dx| + |dy|; chamfer 4-3 = min over sources
of 3 max(|dx|, |dy|) + min(|dx|, |dy|) (the cost of the cheapest path of
horizontal / vertical steps of 3 and diagonal steps of 4)."""
import itertools

import numpy as np
import pytest

import oracle
from golden_io import grid, six_object_mask

INF = np.iinfo(np.int32).max
TYPO_CITYBLOCK = (5, 8)      # printed 3 in Fig. 12(c) and 13(c); the distance is 2
TYPO_CHAMFER_FWD = (8, 1)    # printed 14 in Fig. 15(a); the forward scan gives 12


def brute(mask, mode, kind):
    src = (mask != 0) if mode == 0 else (mask == 0)
    H, W = mask.shape
    out = np.full((H, W), INF, np.int64)
    ii, jj = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    for a, b in np.argwhere(src):
        dy, dx = np.abs(ii - a), np.abs(jj - b)
        d = dx + dy if kind == "cityblock" else 3 * np.maximum(dx, dy) + np.minimum(dx, dy)
        out = np.minimum(out, d)
    return out


def _expect(name, got, typo=None, typo_value=None):
    want = grid(name, inf=INF)
    if typo is not None:
        assert want[typo] != typo_value and got[typo] == typo_value
        want = want.copy()
        want[typo] = typo_value
    np.testing.assert_array_equal(got, want)


def test_fig12_cityblock_two_scans():
    m = six_object_mask()
    _expect("fig12b_cityblock_forward.txt", oracle.cityblock(m, 0, stop_after_forward=True))
    _expect("fig12c_cityblock_final.txt", oracle.cityblock(m, 0), TYPO_CITYBLOCK, 2)


def test_fig13_cityblock_four_scans():
    m = six_object_mask()
    _expect("fig13b_cityblock_vertical.txt", oracle.cityblock_4scan(m, 0, stop_after_columns=True))
    _expect("fig12c_cityblock_final.txt", oracle.cityblock_4scan(m, 0), TYPO_CITYBLOCK, 2)


def test_fig15_chamfer43():
    m = six_object_mask()
    _expect("fig15a_chamfer_forward.txt", oracle.chamfer43(m, 0, stop_after_forward=True), TYPO_CHAMFER_FWD, 12)
    _expect("fig15b_chamfer_final.txt", oracle.chamfer43(m, 0))


def test_typo_cells_agree_with_the_definitions():
    m = six_object_mask()
    assert brute(m, 0, "cityblock")[TYPO_CITYBLOCK] == 2
    assert brute(m, 0, "chamfer")[TYPO_CHAMFER_FWD] == 12


@pytest.mark.parametrize("shape", [(3, 4), (2, 6), (1, 9), (4, 3)])
def test_every_small_mask_matches_brute_force(shape):
    H, W = shape
    for bits in range(1 << (H * W)):
        m = np.array([(bits >> k) & 1 for k in range(H * W)], np.uint8).reshape(shape)
        for mode in (0, 1):
            cb = brute(m, mode, "cityblock")
            np.testing.assert_array_equal(oracle.cityblock(m, mode), cb)
            np.testing.assert_array_equal(oracle.cityblock_4scan(m, mode), cb)
            np.testing.assert_array_equal(oracle.chamfer43(m, mode), brute(m, mode, "chamfer"))


def test_random_masks_match_brute_force():
    rng = np.random.default_rng(7)
    for _ in range(300):
        H, W = (int(v) for v in rng.integers(1, 24, 2))
        m = (rng.random((H, W)) < rng.choice([0.005, 0.05, 0.3, 0.9])).astype(np.uint8)
        for mode in (0, 1):
            cb = brute(m, mode, "cityblock")
            np.testing.assert_array_equal(oracle.cityblock(m, mode), cb)
            np.testing.assert_array_equal(oracle.cityblock_4scan(m, mode), cb)
            np.testing.assert_array_equal(oracle.chamfer43(m, mode), brute(m, mode, "chamfer"))


def test_first_column_sources():
    """A source in the first column reaches the pixels below it straight down
    the column (the reading that differs from the listing's border loops)."""
    m = np.zeros((9, 10), np.uint8)
    m[0, 0] = 1
    d = oracle.cityblock(m, 0)
    np.testing.assert_array_equal(d[:, 0], np.arange(9))
    np.testing.assert_array_equal(oracle.chamfer43(m, 0)[:, 0], 3 * np.arange(9))


def test_no_source_gives_int32_max():
    m = np.zeros((4, 5), np.uint8)
    for fn in (oracle.cityblock, oracle.cityblock_4scan, oracle.chamfer43):
        assert np.all(fn(m, 0) == INF)
        assert np.all(fn(m, 1) == 0)
