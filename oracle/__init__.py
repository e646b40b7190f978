"""CPU oracle for the exact squared Euclidean distance transform (and the
city-block, chamfer 4-3 and Danielsson transforms of Section 2).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use this package; the CUDA library and its Python
binding never import it.  The arithmetic lives in ``edt_oracle.c`` (plain,
single-threaded C following Section 3 of T. Strutz, "The Distance Transform
and its Computation", written from its definitions and equations); this
module only compiles it with gcc and marshals
numpy arrays through ctypes.

Conventions (shared by value, not by code, with the CUDA library):
  mode 0 = TO_OBJECT      sources are the nonzero mask bytes (Fig. 1c)
  mode 1 = TO_BACKGROUND  sources are the zero mask bytes (Fig. 1b)
  D  int32 squared distance, INT32_MAX when the image has no source pixel
  F  int32 0-based row-major index of a nearest source pixel, -1 without one
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

TO_OBJECT = 0
TO_BACKGROUND = 1
INF32 = np.iinfo(np.int32).max

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "edt_oracle.c")
_SRC_NEDT = os.path.join(_HERE, "nedt_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle_edt.so")
_LIB_OMP_PATH = os.path.join(_BUILD, "liboracle_edt_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None


def _compile(path, extra, required):
    os.makedirs(_BUILD, exist_ok=True)
    if (os.path.exists(path)
            and os.path.getmtime(path) >= max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_NEDT))):
        return path
    tmp = path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-Wno-unknown-pragmas", "-shared", "-fPIC"] + extra + [_SRC, _SRC_NEDT, "-o", tmp, "-lm"]
    if required:
        subprocess.check_call(cmd)
    elif subprocess.run(cmd, capture_output=True).returncode != 0:
        return None
    os.replace(tmp, path)
    return path


def build(force: bool = False) -> str:
    """Compile edt_oracle.c into a shared library (plain gcc, no CUDA): the
    single-threaded checker, and (when gcc has OpenMP) the same source with
    -fopenmp for the all-core CPU baseline timing."""
    if force:
        for p in (_LIB_PATH, _LIB_OMP_PATH):
            if os.path.exists(p):
                os.remove(p)
    _compile(_LIB_OMP_PATH, ["-fopenmp"], required=False)
    return _compile(_LIB_PATH, [], required=True)


def edt_all_cores(mask, mode: int = TO_OBJECT):
    """The same 2-D/3-D transform from the OpenMP build of the same source
    (columns and rows spread over all host cores), for CPU baseline timing.
    Returns (D, F, threads), or None when gcc has no OpenMP."""
    path = _compile(_LIB_OMP_PATH, ["-fopenmp"], required=False)
    if path is None:
        return None
    global _lib_omp
    with _lock:
        if _lib_omp is None:
            lib = ctypes.CDLL(path)
            i32p = ctypes.POINTER(ctypes.c_int32)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            lib.oracle_edt2d.restype = ctypes.c_int
            lib.oracle_edt2d.argtypes = [u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, i32p, i32p]
            lib.oracle_edt3d.restype = ctypes.c_int
            lib.oracle_edt3d.argtypes = [u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, i32p, i32p]
            _lib_omp = lib
    m = _mask(mask)
    D = np.empty(m.shape, dtype=np.int32)
    F = np.empty(m.shape, dtype=np.int32)
    if m.ndim == 2:
        rc = _lib_omp.oracle_edt2d(_ptr(m, ctypes.c_uint8), m.shape[0], m.shape[1], int(mode),
                                   _ptr(D, ctypes.c_int32), _ptr(F, ctypes.c_int32))
    else:
        rc = _lib_omp.oracle_edt3d(_ptr(m, ctypes.c_uint8), *m.shape, int(mode), _ptr(D, ctypes.c_int32),
                                   _ptr(F, ctypes.c_int32))
    if rc != 0:
        raise MemoryError("oracle ran out of memory")
    threads = int(os.environ.get("OMP_NUM_THREADS", 0)) or (os.cpu_count() or 1)
    return D, F, threads


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        lib.oracle_max_dist.restype = ctypes.c_int64
        lib.oracle_max_dist.argtypes = [ctypes.c_int, i32p]
        lib.oracle_edt2d.restype = ctypes.c_int
        lib.oracle_edt2d.argtypes = [u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, i32p, i32p]
        lib.oracle_edt3d.restype = ctypes.c_int
        lib.oracle_edt3d.argtypes = [u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, i32p, i32p]
        lib.oracle_edt2d_basic.restype = ctypes.c_int
        lib.oracle_edt2d_basic.argtypes = lib.oracle_edt2d.argtypes
        lib.oracle_column_pass2d.restype = ctypes.c_int
        lib.oracle_column_pass2d.argtypes = [u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int, i64p, i32p]
        lib.oracle_envelope_state.restype = ctypes.c_long
        lib.oracle_envelope_state.argtypes = [i64p, ctypes.c_long, ctypes.c_int64, i64p, i64p]
        lib.oracle_sqrt_f32.restype = None
        lib.oracle_sqrt_f32.argtypes = [i32p, ctypes.c_long, ctypes.POINTER(ctypes.c_float)]
        for name in ("oracle_cityblock2d", "oracle_cityblock2d_4scan", "oracle_chamfer43_2d"):
            fn = getattr(lib, name)
            fn.restype = ctypes.c_int
            fn.argtypes = [u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, i32p]
        lib.oracle_danielsson2d.restype = ctypes.c_int
        lib.oracle_danielsson2d.argtypes = [u8p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, i32p, i32p, i32p]
        _lib = lib
        return lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _mask(mask) -> np.ndarray:
    m = np.ascontiguousarray(mask)
    if m.dtype == np.bool_:
        m = m.astype(np.uint8)
    if m.dtype != np.uint8:
        raise TypeError(f"mask must be uint8 or bool, got {m.dtype}")
    return m


def max_dist(shape) -> int:
    """One more than the largest squared distance inside an image of `shape`."""
    lib = _load()
    s = np.ascontiguousarray(shape, dtype=np.int32)
    return int(lib.oracle_max_dist(len(shape), _ptr(s, ctypes.c_int32)))


def edt(mask, mode: int = TO_OBJECT, features: bool = True):
    """Exact squared EDT of a 2-D or 3-D uint8 mask: returns (D, F) int32."""
    lib = _load()
    m = _mask(mask)
    D = np.empty(m.shape, dtype=np.int32)
    F = np.empty(m.shape, dtype=np.int32)
    if m.ndim == 2:
        rc = lib.oracle_edt2d(_ptr(m, ctypes.c_uint8), m.shape[0], m.shape[1], int(mode),
                              _ptr(D, ctypes.c_int32), _ptr(F, ctypes.c_int32))
    elif m.ndim == 3:
        rc = lib.oracle_edt3d(_ptr(m, ctypes.c_uint8), m.shape[0], m.shape[1], m.shape[2],
                              int(mode), _ptr(D, ctypes.c_int32), _ptr(F, ctypes.c_int32))
    else:
        raise ValueError("oracle handles 2-D and 3-D masks")
    if rc != 0:
        raise MemoryError("oracle ran out of memory")
    return (D, F) if features else D


def edt2d_basic(mask, mode: int = TO_OBJECT):
    """Same result by the O(M L^2) row pass of Sec. 3.1 (cross-check)."""
    lib = _load()
    m = _mask(mask)
    assert m.ndim == 2
    D = np.empty(m.shape, dtype=np.int32)
    F = np.empty(m.shape, dtype=np.int32)
    rc = lib.oracle_edt2d_basic(_ptr(m, ctypes.c_uint8), m.shape[0], m.shape[1], int(mode),
                                _ptr(D, ctypes.c_int32), _ptr(F, ctypes.c_int32))
    if rc != 0:
        raise MemoryError("oracle ran out of memory")
    return D, F


def column_pass(mask, mode: int = TO_OBJECT, down_only: bool = False):
    """Column scans only: (Dv int64 with max_dist as infinity, G int32, max_dist)."""
    lib = _load()
    m = _mask(mask)
    assert m.ndim == 2
    Dv = np.empty(m.shape, dtype=np.int64)
    G = np.empty(m.shape, dtype=np.int32)
    lib.oracle_column_pass2d(_ptr(m, ctypes.c_uint8), m.shape[0], m.shape[1], int(mode),
                             1 if down_only else 0, _ptr(Dv, ctypes.c_int64),
                             _ptr(G, ctypes.c_int32))
    return Dv, G, max_dist(m.shape)


def envelope_state(f, maxd: int):
    """Envelope list of Sec. 3.3.1 on one line: (sites, starts) as 0-based
    int64 arrays; starts has one more entry, the line length."""
    lib = _load()
    fv = np.ascontiguousarray(f, dtype=np.int64)
    n = fv.shape[0]
    site = np.empty(n + 1, dtype=np.int64)
    start = np.empty(n + 1, dtype=np.int64)
    cnt = lib.oracle_envelope_state(_ptr(fv, ctypes.c_int64), n, int(maxd),
                                    _ptr(site, ctypes.c_int64), _ptr(start, ctypes.c_int64))
    return site[:cnt].copy(), start[:cnt + 1].copy()


def sqrt_f32(D) -> np.ndarray:
    """float32 square root of the squared distances (+inf where D = INT32_MAX)."""
    lib = _load()
    d = np.ascontiguousarray(D, dtype=np.int32)
    out = np.empty(d.shape, dtype=np.float32)
    lib.oracle_sqrt_f32(_ptr(d, ctypes.c_int32), d.size, _ptr(out, ctypes.c_float))
    return out


def _nedt(name, mask, mode, stop):
    lib = _load()
    m = _mask(mask)
    assert m.ndim == 2
    D = np.empty(m.shape, dtype=np.int32)
    if getattr(lib, name)(_ptr(m, ctypes.c_uint8), m.shape[0], m.shape[1], int(mode), int(stop),
                          _ptr(D, ctypes.c_int32)) != 0:
        raise MemoryError("oracle ran out of memory")
    return D


def cityblock(mask, mode: int = TO_OBJECT, stop_after_forward: bool = False):
    """City-block distance transform of Sec. 2.1, two raster scans (int32;
    INT32_MAX where no source is reachable)."""
    return _nedt("oracle_cityblock2d", mask, mode, stop_after_forward)


def cityblock_4scan(mask, mode: int = TO_OBJECT, stop_after_columns: bool = False):
    """City-block transform of Sec. 2.1 by the four scans (columns, then rows)."""
    return _nedt("oracle_cityblock2d_4scan", mask, mode, stop_after_columns)


def danielsson(mask, mode: int = TO_OBJECT, stop_after_forward: bool = False, text_order: bool = False):
    """Danielsson's approximate Euclidean transform, Sec. 2.3 (two scans of
    relative-position propagation): (D, DY, DX), D = DY^2 + DX^2 in int32,
    INT32_MAX and DY = DX = -1 where no position arrived.  text_order: in the
    right-to-left pass of the first scan, look at the right neighbour before
    the upper-right one (the order the paper's text names; its listing, the
    default, has them the other way round)."""
    lib = _load()
    m = _mask(mask)
    assert m.ndim == 2
    D = np.empty(m.shape, dtype=np.int32)
    DY = np.empty(m.shape, dtype=np.int32)
    DX = np.empty(m.shape, dtype=np.int32)
    if lib.oracle_danielsson2d(_ptr(m, ctypes.c_uint8), m.shape[0], m.shape[1], int(mode),
                               int(stop_after_forward), int(bool(text_order)), _ptr(D, ctypes.c_int32),
                               _ptr(DY, ctypes.c_int32),
                               _ptr(DX, ctypes.c_int32)) != 0:
        raise MemoryError("oracle ran out of memory")
    return D, DY, DX


def chamfer43(mask, mode: int = TO_OBJECT, stop_after_forward: bool = False):
    """Chamfer 4-3 distance transform of Sec. 2.2, two raster scans."""
    return _nedt("oracle_chamfer43_2d", mask, mode, stop_after_forward)
