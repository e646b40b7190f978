"""The float32 square root of Sec. 3.1 (taken once the squared distances are known),
checked for correct rounding with exact midpoint arithmetic."""
import numpy as np

import oracle


def _check_correctly_rounded(D, f):
    """For each D, f must be the float32 nearest to sqrt(D).  With the float
    neighbours f- < f < f+, the midpoints (f- + f)/2 and (f + f+)/2 have at
    most 25 significant bits, so their squares are exact in float64, and D is
    exact too; sqrt(D) is never a midpoint (it is an integer or irrational)."""
    D = D.astype(np.float64)
    f64 = f.astype(np.float64)
    up = np.nextafter(f, np.float32(np.inf)).astype(np.float64)
    dn = np.nextafter(f, np.float32(0)).astype(np.float64)
    hi_mid = (f64 + up) / 2
    lo_mid = (f64 + dn) / 2
    pos = D > 0
    assert np.all(D[pos] < hi_mid[pos] ** 2)
    assert np.all(D[pos] > lo_mid[pos] ** 2)
    assert np.all(f[~pos] == 0)


def test_sqrt_exhaustive_low_range():
    D = np.arange(0, 1 << 22, dtype=np.int32)
    _check_correctly_rounded(D, oracle.sqrt_f32(D))


def test_sqrt_random_and_edges():
    rng = np.random.default_rng(3)
    D = rng.integers(0, 2**31 - 1, size=2_000_000, dtype=np.int64)
    sq = np.arange(1, 46341, dtype=np.int64) ** 2
    edges = np.concatenate([sq - 1, sq, sq + 1, 2 ** np.arange(0, 31, dtype=np.int64),
                            2 ** np.arange(1, 31, dtype=np.int64) - 1, [2**31 - 2]])
    D = np.concatenate([D, edges[(edges >= 0) & (edges < 2**31 - 1)]]).astype(np.int32)
    _check_correctly_rounded(D, oracle.sqrt_f32(D))


def test_sqrt_of_no_source_is_inf():
    assert np.isinf(oracle.sqrt_f32(np.array([np.iinfo(np.int32).max], np.int32))[0])
