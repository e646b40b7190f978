"""The pins must catch plausible mistakes: each case plants one mistake in a
copy of the oracle's C source (on the CPU, in a temporary directory), builds
it, and checks that the golden examples or brute force reject it."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from brute import brute_edt, feature_valid
from golden_io import grid, six_object_mask

SRC = os.path.join(os.path.dirname(oracle.__file__), "edt_oracle.c")

MUTANTS = {
    # column distances (Sec. 3.1)
    "no_upward_sweep": ("long dn = down_only ? -1 : next;", "long dn = -1;"),
    "no_downward_sweep": ("if (dn < 0 || (up >= 0 &&", "if (0 && (up >= 0 &&"),
    "distance_not_squared": ("(int64_t)(i - g) * (int64_t)(i - g);", "(int64_t)(i - g) * (int64_t)(i > g ? 1 : -1);"),
    "stale_nearest_below": ("        if (d[i * stride] == 0)\n            next = i;",
                            "        if (d[i * stride] == 0 && next < 0)\n            next = i;"),
    # envelope (Sec. 3.3.1, Eq. (5) and (6))
    "intersection_sign": ("f[m] - f[k] + m * m - k * k", "f[m] - f[k] - m * m + k * k"),
    "intersection_denominator": ("2 * (m - k));", "(m - k));"),
    "floor_not_ceil": ("if (num > 0 && num % den != 0)", "if (num < 0 && num % den != 0)"),
    "strict_pop": ("if (s > start[cnt - 1])", "if (s >= start[cnt - 1])"),
    "no_pop": ("while (cnt > 0) {", "while (0 && cnt > 0) {"),
    "first_site_not_at_zero": ("            cnt -= 1;\n            s = 0;", "            cnt -= 1;\n            s = m;"),
    "fill_wrong_offset": ("out[j] = f[k] + (j - k) * (j - k);", "out[j] = f[k] + (j - k + 1) * (j - k);"),
    "feature_from_target": ("feat_out[j] = feat_in[k];", "feat_out[j] = feat_in[j];"),
    "wrong_axis_3d": ("envelope_pass(d + z * plane + x, feat + z * plane + x, H, W,",
                      "envelope_pass(d + z * plane + x, feat + z * plane + x, H, 1,"),
    "mode_ignored": ("(mode == ORACLE_TO_OBJECT) ? (mask[p] != 0) : (mask[p] == 0)",
                     "(mask[p] != 0)"),
    "sentinel_too_small": ("int64_t s = 1;", "int64_t s = -40;"),
}


def _build(tmp_path, name, old, new):
    src = open(SRC).read()
    assert old in src, f"mutation anchor for {name} not found"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new, 1))
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-w", "-shared", "-fPIC", str(path), "-o", str(so), "-lm"])
    lib = ctypes.CDLL(str(so))
    i32p = ctypes.POINTER(ctypes.c_int32)
    u8p = ctypes.POINTER(ctypes.c_uint8)
    lib.oracle_edt2d.argtypes = [u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, i32p, i32p]
    lib.oracle_edt3d.argtypes = [u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, i32p, i32p]
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.oracle_column_pass2d.argtypes = [u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, i64p, i32p]
    lib.oracle_envelope_state.restype = ctypes.c_long
    lib.oracle_envelope_state.argtypes = [i64p, ctypes.c_long, ctypes.c_int64, i64p, i64p]
    return lib


def _envelope_state_row1(lib):
    """Listed columns and their first positions (1-based, with the line end)
    of the Sec. 3.3.1 walk-through row, from the variant."""
    m = six_object_mask()
    Dv = np.empty(m.shape, np.int64)
    G = np.empty(m.shape, np.int32)
    lib.oracle_column_pass2d(m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), 9, 10, 0, 0,
                             Dv.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                             G.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    f = np.ascontiguousarray(Dv[0])
    site = np.zeros(12, np.int64)
    start = np.zeros(12, np.int64)
    cnt = lib.oracle_envelope_state(f.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), 10,
                                    oracle.max_dist((9, 10)),
                                    site.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                    start.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    return (site[:cnt] + 1).tolist(), (start[:cnt + 1] + 1).tolist()


def _run(lib, m, mode):
    m = np.ascontiguousarray(m, dtype=np.uint8)
    D = np.empty(m.shape, np.int32)
    F = np.empty(m.shape, np.int32)
    u8 = m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    dp = D.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    fp = F.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
    if m.ndim == 2:
        lib.oracle_edt2d(u8, m.shape[0], m.shape[1], mode, dp, fp)
    else:
        lib.oracle_edt3d(u8, *m.shape, mode, dp, fp)
    return D, F


def _pins_pass(lib):
    D, F = _run(lib, six_object_mask(), 0)
    if not np.array_equal(D, grid("fig18c_final.txt")):
        return False
    # Fig. 21 ties '2/5' and '5/8' resolved to the right-hand parabola
    if not np.array_equal(F[0] % 10 + 1, [5, 5, 5, 5, 5, 5, 8, 8, 8, 8]):
        return False
    # Sec. 3.3.1 walk-through: ks = (1, 5, 8), js = (1, 1, 7, 11) without the
    # paper's dummy first parabola (its interval [1, 1) is empty)
    if _envelope_state_row1(lib) != ([5, 8], [1, 7, 11]):
        return False
    rng = np.random.default_rng(0)
    for t in range(60):
        mode = t % 2
        if t % 3 == 2:
            shape = tuple(int(v) for v in rng.integers(2, 7, size=3))
        else:
            shape = tuple(int(v) for v in rng.integers(2, 14, size=2))
        m = (rng.random(shape) < rng.choice([0.05, 0.2, 0.5])).astype(np.uint8)
        D, F = _run(lib, m, mode)
        if not np.array_equal(D, brute_edt(m, mode)) or not feature_valid(m, mode, D, F):
            return False
    return True


def _pins_pass_in_child(tmp_path, name, old, new):
    """Build and check the variant in a child process: a planted mistake may
    also crash the C code (an index out of bounds), which counts as caught."""
    import sys
    code = (
        "import sys, pathlib; sys.path[:0] = %r\n"
        "import test_oracle_mutants as t\n"
        "lib = t._build(pathlib.Path(%r), %r, %r, %r)\n"
        "sys.exit(0 if t._pins_pass(lib) else 1)\n"
    ) % ([os.path.dirname(os.path.abspath(__file__)), os.path.dirname(os.path.dirname(os.path.abspath(__file__)))],
         str(tmp_path), name, old, new)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, timeout=300)
    return r.returncode == 0, r


def test_unmutated_copy_passes(tmp_path):
    ok, r = _pins_pass_in_child(tmp_path, "identity", "int64_t s = 1;", "int64_t s = 1;")
    assert ok, r.stderr.decode()[-2000:]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    ok, r = _pins_pass_in_child(tmp_path, name, old, new)
    assert not ok, f"planted mistake '{name}' went unnoticed"
