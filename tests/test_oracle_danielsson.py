"""The oracle's Danielsson transform (Sec. 2.3, relative-position
propagation), an approximation of the exact EDT kept as an accuracy foil.

Pinned to the paper's worked example (Fig. 16(b) after the first scan,
Fig. 16(c) final, one printed cell read as a typo; the paper states that the
example's result equals the exact transform of Fig. 18(c)), to a 4 x 4 mask
whose result was derived by hand from the text and depends on the diagonal
looks, to what the propagation guarantees (every value is the squared length of an offset that
dominates the offset to some source componentwise, so it is never below the
exact squared distance; a single source is reached exactly), and measured
against the exact oracle on the synthetic workloads: how often and by how much
it differs."""
import numpy as np
import pytest

import oracle
from golden_io import grid, pair_rows, pairs, sections, six_object_mask
from paper_2106_03503_gb300 import inputs

INF = np.iinfo(np.int32).max
TYPO_FIG16C = (2, 2)       # 0-based; printed 1,1, the scans give 1,2


def test_fig16b_after_the_first_scan():
    D, DY, DX = oracle.danielsson(six_object_mask(), 0, stop_after_forward=True)
    ey, ex = pairs("fig16b_danielsson_forward.txt")
    np.testing.assert_array_equal(DY, ey)
    np.testing.assert_array_equal(DX, ex)
    np.testing.assert_array_equal(D[0], INF)                       # top row not visited yet


def test_fig16c_final():
    m = six_object_mask()
    D, DY, DX = oracle.danielsson(m, 0)
    ey, ex = pairs("fig16c_danielsson_final.txt")
    # the printed cell is impossible: shorter than the exact distance there
    De, _ = oracle.edt(m, 0)
    assert ey[TYPO_FIG16C] ** 2 + ex[TYPO_FIG16C] ** 2 < De[TYPO_FIG16C]
    assert (ey[TYPO_FIG16C], ex[TYPO_FIG16C]) == (1, 1) and (DY[TYPO_FIG16C], DX[TYPO_FIG16C]) == (1, 2)
    ey[TYPO_FIG16C], ex[TYPO_FIG16C] = 1, 2
    np.testing.assert_array_equal(DY, ey)
    np.testing.assert_array_equal(DX, ex)
    np.testing.assert_array_equal(D, DY * DY + DX * DX)


def test_hand_derived_diagonal_example():
    """The text's diagonal looks (upper-left in the left-to-right pass,
    upper-right in the right-to-left pass; mirrored in the second scan) decide
    one cell of this 4 x 4 mask: (2,2), D = 8, instead of (0,3), D = 9.  Both
    look orders give the same grids here."""
    g = sections("danielsson_diagonal_4x4.txt")
    m = np.array([[int(c) for c in r.split()] for r in g["mask"]], np.uint8)
    for text_order in (False, True):
        _, fy, fx = oracle.danielsson(m, 0, stop_after_forward=True, text_order=text_order)
        ey, ex = pair_rows(g["forward"])
        np.testing.assert_array_equal(fy, ey)
        np.testing.assert_array_equal(fx, ex)
        D, DY, DX = oracle.danielsson(m, 0, text_order=text_order)
        ey, ex = pair_rows(g["final"])
        np.testing.assert_array_equal(DY, ey)
        np.testing.assert_array_equal(DX, ex)
        assert D[3, 3] == 8
    De, _ = oracle.edt(m, 0)
    np.testing.assert_array_equal(D, De)       # exact on this example


def test_example_equals_the_exact_transform():
    """Sec. 2.3: for this example the result is the exact EDT (Fig. 18(c))."""
    D, _, _ = oracle.danielsson(six_object_mask(), 0)
    np.testing.assert_array_equal(D, grid("fig18c_final.txt"))


@pytest.mark.parametrize("mode", [0, 1])
def test_never_below_the_exact_distance(mode):
    rng = np.random.default_rng(16)
    for _ in range(150):
        H, W = (int(v) for v in rng.integers(2, 48, 2))
        m = (rng.random((H, W)) < rng.choice([0.005, 0.03, 0.2, 0.6])).astype(np.uint8)
        D, DY, DX = oracle.danielsson(m, mode)
        De, _ = oracle.edt(m, mode)
        src = (m != 0) if mode == 0 else (m == 0)
        if not src.any():
            assert (D == INF).all() and (DY == -1).all()
            continue
        assert (D >= De).all()
        assert (D[src] == 0).all() and (D[~src] > 0).all()
        assert (D < INF).all()                                     # every pixel reached (H >= 2)


def test_single_source_is_exact():
    rng = np.random.default_rng(17)
    for _ in range(200):
        H, W = (int(v) for v in rng.integers(2, 40, 2))
        m = np.zeros((H, W), np.uint8)
        m[rng.integers(0, H), rng.integers(0, W)] = 1
        D, DY, DX = oracle.danielsson(m, 0)
        (a, b), = np.argwhere(m)
        ii, jj = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
        np.testing.assert_array_equal(DY, np.abs(ii - a))
        np.testing.assert_array_equal(DX, np.abs(jj - b))


def test_single_row_is_not_visited():
    """The scans start at the second row (first scan) and the next-to-last
    row (second scan), so a one-row image keeps only its sources."""
    m = np.array([[0, 1, 0, 0, 1]], np.uint8)
    D, _, _ = oracle.danielsson(m, 0)
    np.testing.assert_array_equal(D, [[INF, 0, INF, INF, 0]])


def _accuracy(m, mode, text_order):
    D, _, _ = oracle.danielsson(m, mode, text_order=text_order)
    De, _ = oracle.edt(m, mode)
    diff = D != De
    err = np.sqrt(D[diff].astype(np.float64)) - np.sqrt(De[diff].astype(np.float64))
    return int(diff.sum()), (float(err.max()) if diff.any() else 0.0)


def test_accuracy_on_the_workloads(capsys):
    """How often and by how much the approximation differs from the exact
    transform: the 512^2 Bernoulli points and both transforms of the 8192^2
    discs mask (the 2-D workloads; the paper gives the method for 2-D only),
    under both readings of the look order (the listing's and the text's),
    which the paper's example does not tell apart."""
    rows = []
    discs = inputs.discs_8192()
    for text_order in (False, True):
        reading = "text order" if text_order else "listing order"
        n, e = _accuracy(inputs.points_512(), 0, text_order)
        rows.append((f"512^2 points p=0.01, to object, {reading}", n, 512 * 512, e))
        for mode, name in ((0, "to object"), (1, "to background")):
            n, e = _accuracy(discs, mode, text_order)
            rows.append((f"8192^2 discs, {name}, {reading}", n, discs.size, e))
    with capsys.disabled():
        for name, n, px, e in rows:
            print(f"\nDanielsson vs exact, {name}: {n} of {px} pixels differ "
                  f"({n / px:.2e}), largest distance error {e:.4f} px")
    for name, n, px, e in rows:
        assert n / px < 1e-3 and e < 0.5
    assert sum(n for _, n, _, _ in rows) > 0      # the approximation is not exact here
