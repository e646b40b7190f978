"""The C ABI without a GPU: libedt builds, loads, exports every function that
include/edt.h declares, and rejects bad arguments before touching a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2106_03503_gb300 import build_lib
    path = build_lib.build()
    return ctypes.CDLL(path)


def declared():
    with open(os.path.join(ROOT, "include", "edt.h")) as fh:
        src = fh.read()
    return sorted(set(re.findall(r"^(?:edt_status|const char \*)\s*(edt_\w+)\s*\(", src, re.M)))


def test_header_declares_the_interface():
    names = declared()
    for must in ("edt_sq2d", "edt_sq3d", "edt_feature", "edt_feature_pair", "edt_feature_host",
                 "edt_feature_pair_host", "edt_batch", "edt_serve_submit",
                 "edt_serve_poll", "edt_feature2d_noalloc", "edt_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def _msg(lib):
    lib.edt_last_error.restype = ctypes.c_char_p
    return lib.edt_last_error().decode()


def test_invalid_arguments_fail_before_any_device_work(lib):
    vp = ctypes.c_void_p
    lib.edt_feature.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                vp, vp, vp, vp]
    shape = (ctypes.c_int * 3)(10, 10, 10)
    dummy = vp(16)
    assert lib.edt_feature(dummy, 2, shape, 7, dummy, dummy, None, None) == 1
    assert "mode" in _msg(lib)
    assert lib.edt_feature(dummy, 4, shape, 0, dummy, dummy, None, None) == 1
    assert lib.edt_feature(dummy, 2, shape, 0, dummy, None, None, None) == 1   # F missing
    big = (ctypes.c_int * 2)(10, 16385)
    assert lib.edt_feature(dummy, 2, big, 0, dummy, dummy, None, None) == 2
    huge = (ctypes.c_int * 2)(40000, 10)
    assert lib.edt_feature(dummy, 2, huge, 0, dummy, dummy, None, None) == 2
    neg = (ctypes.c_int * 2)(0, 10)
    assert lib.edt_feature(dummy, 2, neg, 0, dummy, dummy, None, None) == 1
    v3 = (ctypes.c_int * 3)(10, 3000, 10)
    assert lib.edt_feature(dummy, 3, v3, 0, dummy, dummy, None, None) == 2
    lib.edt_sq2d.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp]
    assert lib.edt_sq2d(None, 4, 4, 0, dummy, None) == 1
    lib.edt_batch.argtypes = [vp, vp, ctypes.c_int, vp]
    assert lib.edt_batch(None, None, 1, None) == 1
    lib.edt_serve_submit.argtypes = [vp, vp, vp]
    assert lib.edt_serve_submit(None, None, None) == 1
    lib.edt_feature2d_noalloc.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp]
    assert lib.edt_feature2d_noalloc(dummy, 4, 4, 3, dummy, dummy, None, None) == 1
    for name in ("edt_feature_pair", "edt_feature_pair_host"):
        fn = getattr(lib, name)
        fn.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), vp, vp, vp, vp, vp]
        assert fn(dummy, 2, shape, dummy, dummy, dummy, None, None) == 1        # F_bg missing
        assert fn(dummy, 2, big, dummy, dummy, dummy, dummy, None) == 2
    lib.edt_feature_host.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                     vp, vp, vp, vp]
    assert lib.edt_feature_host(None, 2, shape, 0, dummy, dummy, None, None) == 1
    assert lib.edt_feature_host(dummy, 2, shape, 9, dummy, dummy, None, None) == 1


def test_version_string(lib):
    lib.edt_version.restype = ctypes.c_char_p
    assert b"libedt" in lib.edt_version()


def test_tuning_table_load_get_save(lib, tmp_path):
    """The autotuner's table on the host: a file merges into it, queries map
    a shape to its class (rounded-up log2 of each side), a save writes it back,
    malformed or out-of-range files are refused and leave it unchanged."""
    i3 = ctypes.c_int * 3
    lib.edt_tune_get.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.edt_tune_load.argtypes = [ctypes.c_char_p]
    lib.edt_tune_save.argtypes = [ctypes.c_char_p]
    good = tmp_path / "tune.txt"
    good.write_text("# comment\n2 10 13 0 8 0 0\n3 9 9 9 0 4 16\n")
    assert lib.edt_tune_load(str(good).encode()) == 0
    w = i3()
    assert lib.edt_tune_get(2, (ctypes.c_int * 2)(1000, 8192), w) == 0 and list(w) == [8, 0, 0]
    assert lib.edt_tune_get(2, (ctypes.c_int * 2)(513, 4097), w) == 0 and list(w) == [8, 0, 0]
    assert lib.edt_tune_get(2, (ctypes.c_int * 2)(512, 8192), w) == 0 and list(w) == [0, 0, 0]
    assert lib.edt_tune_get(3, (ctypes.c_int * 3)(512, 300, 257), w) == 0 and list(w) == [0, 4, 16]
    for bad in ("2 10 13\n", "4 1 1 1 0 0 0\n", "2 10 13 0 12 0 0\n", "3 9 9 9 0 64 0\n"):
        f = tmp_path / "bad.txt"
        f.write_text(bad)
        assert lib.edt_tune_load(str(f).encode()) == 1, bad
    assert lib.edt_tune_load(str(tmp_path / "missing.txt").encode()) == 1
    assert lib.edt_tune_get(3, (ctypes.c_int * 3)(512, 300, 257), w) == 0 and list(w) == [0, 4, 16]
    out = tmp_path / "saved.txt"
    assert lib.edt_tune_save(str(out).encode()) == 0
    lines = [ln.split() for ln in out.read_text().splitlines() if ln and not ln.startswith("#")]
    assert ["2", "10", "13", "0", "8", "0", "0"] in lines and ["3", "9", "9", "9", "0", "4", "16"] in lines
    assert lib.edt_tune_get(4, (ctypes.c_int * 3)(1, 1, 1), w) == 1
    reset = tmp_path / "reset.txt"          # the table is process-wide: leave the rules in force
    reset.write_text("2 10 13 0 0 0 0\n3 9 9 9 0 0 0\n")
    assert lib.edt_tune_load(str(reset).encode()) == 0
