"""Pins the oracle to the worked examples printed in the paper."""
import numpy as np

import oracle
from golden_io import grid, keyed, six_object_mask


def _with_inf(a, maxd):
    out = a.astype(np.int64).copy()
    out[a >= maxd] = -1
    return out


def test_fig18b_vertical_distances():
    """Sec. 3.1, Fig. 18(b): both column scans of the six-object example."""
    Dv, _, maxd = oracle.column_pass(six_object_mask(), oracle.TO_OBJECT)
    np.testing.assert_array_equal(_with_inf(Dv, maxd), grid("fig18b_vertical.txt"))


def test_fig19_downward_scan_only():
    """Sec. 3.1, Fig. 19: the column pass after the downward scan."""
    Dv, _, maxd = oracle.column_pass(six_object_mask(), oracle.TO_OBJECT, down_only=True)
    np.testing.assert_array_equal(_with_inf(Dv, maxd), grid("fig19_downward.txt"))


def test_fig18c_final_distances():
    """Sec. 3.1, Fig. 18(c): final squared distances of the six-object example."""
    D, F = oracle.edt(six_object_mask(), oracle.TO_OBJECT)
    np.testing.assert_array_equal(D, grid("fig18c_final.txt"))


def test_fig18c_by_basic_row_pass():
    """Same figure through the O(M L^2) row pass of Sec. 3.1."""
    D, _ = oracle.edt2d_basic(six_object_mask(), oracle.TO_OBJECT)
    np.testing.assert_array_equal(D, grid("fig18c_final.txt"))


def test_fig8b_single_pixel():
    """Sec. 1.3.1, Fig. 8(b): squared distances from one centre pixel."""
    m = np.zeros((9, 10), np.uint8)
    m[4, 4] = 1
    D, F = oracle.edt(m, oracle.TO_OBJECT)
    np.testing.assert_array_equal(D, grid("fig8b_single_pixel.txt"))
    assert np.all(F == 4 * 10 + 4)


def test_fig21_row1_minimum_and_kstar():
    """Sec. 3.3, Fig. 21: row-1 minimum and the contributing column k*, with
    the paper's ties '2/5' and '5/8'.  The oracle's tie rule (an integer
    intersection goes to the right-hand parabola) picks 5 and 8 there."""
    g = keyed("fig21_row1.txt")
    D, F = oracle.edt(six_object_mask(), oracle.TO_OBJECT)
    np.testing.assert_array_equal(D[0], np.array([int(v) for v in g["min"]]))
    kcol = F[0] % 10 + 1  # 1-based contributing column
    for j, allowed in enumerate(g["kstar"]):
        opts = [int(a) for a in allowed.split("/")]
        assert kcol[j] in opts, (j, kcol[j], opts)
        assert kcol[j] == max(opts)
    # the row's vertical components, as printed
    Dv, _, maxd = oracle.column_pass(six_object_mask(), oracle.TO_OBJECT)
    dv = [-1 if v == "inf" else int(v) for v in g["dv"]]
    np.testing.assert_array_equal(_with_inf(Dv[0], maxd), np.array(dv))


def test_fig21_candidate_rows_match_oracle_minimum():
    """Every printed candidate row D_k is >= the oracle's row, and the oracle
    row equals the element-wise minimum of the printed candidates."""
    g = keyed("fig21_row1.txt")
    rows = np.array([[int(v) for v in g[k]] for k in ("D2", "D5", "D6", "D8")])
    D, _ = oracle.edt(six_object_mask(), oracle.TO_OBJECT)
    np.testing.assert_array_equal(rows.min(0), D[0])


def test_sec331_envelope_state():
    """Sec. 3.3.1 walk-through on row 1: the paper's state js = (1,1,7,11),
    ks = (1,5,8) starts with its dummy first parabola at column 1, whose
    interval [1, 1) is empty; the oracle lists no dummy, so its state must be
    the rest: columns 5 and 8 from positions 1 and 7, the line ending at 11."""
    g = keyed("sec331_envelope_state.txt")
    ks_paper = [int(v) for v in g["ks"]]
    js_paper = [int(v) for v in g["js"]]
    assert js_paper[0] == js_paper[1]          # the dummy owns no position
    Dv, _, maxd = oracle.column_pass(six_object_mask(), oracle.TO_OBJECT)
    site, start = oracle.envelope_state(Dv[0], maxd)
    np.testing.assert_array_equal(site + 1, ks_paper[1:])
    np.testing.assert_array_equal(start + 1, js_paper[1:])
