"""Thin Python binding of libedt (C ABI in include/edt.h).

Argument marshalling only: every step of the transform runs in the CUDA
library.  PyTorch supplies device memory and streams.  There is no CPU
fallback: if libedt.so has not been built, importing this module fails.

    from paper_2106_03503_gb300 import edt
    D, F = edt.feature(mask_cuda_uint8)              # 2-D or 3-D
    D = edt.sq2d(mask)                               # squared distances only
    D, F, d = edt.feature(mask, want_dist=True)      # + float32 sqrt
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build_lib

TO_OBJECT = 0
TO_BACKGROUND = 1
INF32 = 2**31 - 1

EDT_OK = 0
EDT_ERR_NOT_READY = 7
_STATUS = {0: "EDT_OK", 1: "EDT_ERR_INVALID", 2: "EDT_ERR_TOO_LARGE", 3: "EDT_ERR_NOMEM",
           4: "EDT_ERR_CUDA", 5: "EDT_ERR_TIMEOUT", 6: "EDT_ERR_BUDGET", 7: "EDT_ERR_NOT_READY"}


class EdtError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


if not os.path.exists(build_lib.LIB):
    raise ImportError(f"libedt is not built ({build_lib.LIB} missing); run "
                      "`python -c 'import __graft_entry__ as g; g.build()'` first")

_lib = ctypes.CDLL(build_lib.LIB)
LIB_PATH = build_lib.LIB

_vp = ctypes.c_void_p
_i32p = ctypes.POINTER(ctypes.c_int)


class Job(ctypes.Structure):
    _fields_ = [("mask", _vp), ("ndim", ctypes.c_int), ("shape", ctypes.c_int * 3),
                ("mode", ctypes.c_int), ("D", _vp), ("F", _vp), ("dist", _vp)]


_lib.edt_sq2d.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp]
_lib.edt_sq3d.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp]
_lib.edt_feature.argtypes = [_vp, ctypes.c_int, _i32p, ctypes.c_int, _vp, _vp, _vp, _vp]
_lib.edt_feature_host.argtypes = [_vp, ctypes.c_int, _i32p, ctypes.c_int, _vp, _vp, _vp, _vp]
_lib.edt_feature_pair.argtypes = [_vp, ctypes.c_int, _i32p, _vp, _vp, _vp, _vp, _vp]
_lib.edt_feature_pair_host.argtypes = [_vp, ctypes.c_int, _i32p, _vp, _vp, _vp, _vp, _vp]
_lib.edt_cityblock2d.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp]
_lib.edt_chamfer43_2d.argtypes = [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp]
_lib.edt_trace_enable.argtypes = [ctypes.c_int]
_lib.edt_trace_enable.restype = ctypes.c_int
_lib.edt_trace_read.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_int64)]
_lib.edt_trace_read.restype = ctypes.c_int
_lib.edt_autotune.argtypes = [_vp, ctypes.c_int, _i32p, ctypes.c_int, _vp]
_lib.edt_autotune.restype = ctypes.c_int
_lib.edt_tune_get.argtypes = [ctypes.c_int, _i32p, _i32p]
_lib.edt_tune_get.restype = ctypes.c_int
_lib.edt_tune_save.argtypes = [ctypes.c_char_p]
_lib.edt_tune_save.restype = ctypes.c_int
_lib.edt_tune_load.argtypes = [ctypes.c_char_p]
_lib.edt_tune_load.restype = ctypes.c_int
_lib.edt_last_error.restype = ctypes.c_char_p
_lib.edt_version.restype = ctypes.c_char_p
for _name in ("edt_sq2d", "edt_sq3d", "edt_feature", "edt_feature_host", "edt_feature_pair"):
    getattr(_lib, _name).restype = ctypes.c_int

EXPORTS = ("edt_sq2d", "edt_sq3d", "edt_feature", "edt_feature_pair", "edt_feature_host",
           "edt_feature_pair_host", "edt_cityblock2d", "edt_chamfer43_2d",
           "edt_plan_create",
           "edt_plan_destroy", "edt_batch", "edt_serve_create", "edt_serve_submit",
           "edt_serve_poll", "edt_serve_destroy", "edt_trace_enable", "edt_trace_read",
           "edt_autotune", "edt_tune_get", "edt_tune_save", "edt_tune_load",
           "edt_autotune_batch", "edt_batch_tune_get", "edt_serve_poll_detail",
           "edt_last_error", "edt_version")


def tune_get(shape):
    """Tuned warps per band of a shape's class: {"rows2d": .., "ypass": ..,
    "xpass": ..}; 0 = the built-in rule."""
    w = (ctypes.c_int * 3)()
    _check(_lib.edt_tune_get(len(shape), _shape_arr(shape), w))
    return {"rows2d": w[0], "ypass": w[1], "xpass": w[2]}


def autotune(mask, mode: int = TO_OBJECT, stream=None):
    """Time the band-geometry candidates on this CUDA mask (edt_autotune) and
    keep the fastest for its shape class; returns tune_get(shape)."""
    m = _mask_arg(mask)
    _check(_lib.edt_autotune(_ptr(m), m.dim(), _shape_arr(m.shape), int(mode), _stream_handle(stream)))
    return tune_get(tuple(m.shape))


def tune_save(path: str):
    """Write the tuning table to a text file (edt_tune_save)."""
    _check(_lib.edt_tune_save(os.fsencode(path)))


def tune_load(path: str):
    """Merge a tuning file into the table (edt_tune_load)."""
    _check(_lib.edt_tune_load(os.fsencode(path)))


def trace_enable(on: bool = True):
    """Start (and reset) or stop per-kernel event timing inside libedt."""
    _check(_lib.edt_trace_enable(1 if on else 0))


def trace_read(kernel: str):
    """(total milliseconds, launches) of `kernel` since tracing was enabled."""
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(_lib.edt_trace_read(kernel.encode(), ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


_lib.edt_plan_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int64]
_lib.edt_plan_create.restype = ctypes.c_int
_lib.edt_plan_destroy.argtypes = [ctypes.c_void_p]
_lib.edt_plan_destroy.restype = ctypes.c_int
_lib.edt_batch.argtypes = [ctypes.c_void_p, ctypes.POINTER(Job), ctypes.c_int, _vp]
_lib.edt_batch.restype = ctypes.c_int
_lib.edt_autotune_batch.argtypes = [ctypes.c_void_p, ctypes.POINTER(Job), ctypes.c_int, _vp]
_lib.edt_autotune_batch.restype = ctypes.c_int
_lib.edt_batch_tune_get.argtypes = [ctypes.c_int, _i32p, _i32p]
_lib.edt_batch_tune_get.restype = ctypes.c_int


def batch_tune_get(shape):
    """Batch geometry of a shape's class: {"rows2d_lgmin": .., "y_pos": ..,
    "x_pos": ..}; 0 = the built-in rule."""
    v = (ctypes.c_int * 3)()
    _check(_lib.edt_batch_tune_get(len(shape), _shape_arr(shape), v))
    return {"rows2d_lgmin": v[0], "y_pos": v[1], "x_pos": v[2]}


# The same layout as Job (edt_job), for filling many jobs at once.
_JOB_DTYPE = np.dtype({"names": ["mask", "ndim", "shape", "mode", "D", "F", "dist"],
                       "formats": [np.uint64, np.int32, (np.int32, 3), np.int32, np.uint64, np.uint64, np.uint64],
                       "offsets": [Job.mask.offset, Job.ndim.offset, Job.shape.offset, Job.mode.offset,
                                   Job.D.offset, Job.F.offset, Job.dist.offset],
                       "itemsize": ctypes.sizeof(Job)})


def _job(mask, mode, D, F, dist):
    j = Job()
    j.mask = mask.data_ptr()
    j.ndim = mask.dim()
    for a in range(3):
        j.shape[a] = int(mask.shape[a]) if a < mask.dim() else 0
    j.mode = int(mode)
    j.D = None if D is None else D.data_ptr()
    j.F = F.data_ptr()
    j.dist = None if dist is None else dist.data_ptr()
    return j


class PreparedBatch:
    """A filled job table (the layout of edt_job) plus references to the
    tensors it points to."""

    def __init__(self, jobs):
        n = len(jobs)
        arr = np.zeros(n, dtype=_JOB_DTYPE)
        arr["mask"] = [j[0].data_ptr() for j in jobs]
        arr["ndim"] = [j[0].dim() for j in jobs]
        arr["shape"] = [tuple(j[0].shape) + (0,) * (3 - j[0].dim()) for j in jobs]
        arr["mode"] = [int(j[1]) for j in jobs]
        arr["D"] = [0 if j[2] is None else j[2].data_ptr() for j in jobs]
        arr["F"] = [j[3].data_ptr() for j in jobs]
        arr["dist"] = [0 if j[4] is None else j[4].data_ptr() for j in jobs]
        self.arr = arr
        self.jobs = list(jobs)


class Plan:
    """A batch plan (edt_plan_create): runs up to n_max 2-D and 3-D jobs as one
    CUDA-graph replay; max_pixels sizes its scratch up front (it grows when a
    batch needs more)."""

    def __init__(self, n_max: int, max_pixels: int):
        self._p = ctypes.c_void_p()
        _check(_lib.edt_plan_create(ctypes.byref(self._p), int(n_max), int(max_pixels)))
        self._keep = None

    @staticmethod
    def prepare(jobs):
        """The job table of `jobs` ((mask, mode, D, F, dist) CUDA tensors; D,
        dist may be None), for repeated runs of the same batch layout."""
        return PreparedBatch(jobs)

    def run(self, jobs, stream=None):
        """jobs: sequence of (mask, mode, D, F, dist) CUDA tensors (D, dist may
        be None), or a PreparedBatch.  Enqueues the batch on `stream`."""
        if isinstance(jobs, PreparedBatch):
            self._keep = jobs
            _check(_lib.edt_batch(self._p, jobs.arr.ctypes.data_as(ctypes.POINTER(Job)), len(jobs.arr),
                                  _stream_handle(stream)))
            return
        self.run(PreparedBatch(jobs), stream)

    def autotune(self, jobs, stream=None):
        """Time the batch-geometry candidates per shape class on these jobs
        (edt_autotune_batch); later batches use the fastest.  Synchronous."""
        pb = jobs if isinstance(jobs, PreparedBatch) else PreparedBatch(jobs)
        _check(_lib.edt_autotune_batch(self._p, pb.arr.ctypes.data_as(ctypes.POINTER(Job)), len(pb.arr),
                                       _stream_handle(stream)))

    def close(self):
        if self._p:
            _check(_lib.edt_plan_destroy(self._p))
            self._p = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch(masks, mode: int = TO_OBJECT, want_dist: bool = False, plan: Plan = None, stream=None):
    """Transform a list of 2-D and 3-D CUDA uint8 masks in one batch; returns a
    list of (D, F[, dist]) tuples."""
    masks = [_mask_arg(m) for m in masks]
    outs = []
    for m in masks:
        D = torch.empty(m.shape, dtype=torch.int32, device=m.device)
        F = torch.empty(m.shape, dtype=torch.int32, device=m.device)
        dist = torch.empty(m.shape, dtype=torch.float32, device=m.device) if want_dist else None
        outs.append((D, F, dist))
    own = plan is None
    if own:
        plan = Plan(len(masks), sum(m.numel() for m in masks))
    plan.run([(m, mode, D, F, dist) for m, (D, F, dist) in zip(masks, outs)], stream)
    if own:
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        plan.close()
    return [(D, F, dist) if want_dist else (D, F) for D, F, dist in outs]


_lib.edt_serve_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t, ctypes.c_int]
_lib.edt_serve_create.restype = ctypes.c_int
_lib.edt_serve_submit.argtypes = [ctypes.c_void_p, ctypes.POINTER(Job), ctypes.POINTER(ctypes.c_uint64)]
_lib.edt_serve_submit.restype = ctypes.c_int
_lib.edt_serve_poll.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]
_lib.edt_serve_poll.restype = ctypes.c_int
_lib.edt_serve_poll_detail.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]
_lib.edt_serve_poll_detail.restype = ctypes.c_int
_lib.edt_serve_destroy.argtypes = [ctypes.c_void_p]
_lib.edt_serve_destroy.restype = ctypes.c_int


class Server:
    """Continuous-batching server (edt_serve_*).  Jobs are host (ideally
    pinned) CPU tensors; results land in host tensors owned by the ticket."""

    def __init__(self, budget_bytes: int, n_streams: int = 2):
        self._s = ctypes.c_void_p()
        _check(_lib.edt_serve_create(ctypes.byref(self._s), int(budget_bytes), int(n_streams)))
        self._live = {}

    def submit(self, mask: torch.Tensor, mode: int = TO_OBJECT, want_D: bool = True,
               want_dist: bool = False, out=None) -> int:
        m = mask.contiguous()
        if m.dtype == torch.bool:
            m = m.view(torch.uint8)
        pin = m.is_pinned()
        if out is None:
            D = torch.empty(m.shape, dtype=torch.int32, pin_memory=pin) if want_D else None
            F = torch.empty(m.shape, dtype=torch.int32, pin_memory=pin)
            dist = torch.empty(m.shape, dtype=torch.float32, pin_memory=pin) if want_dist else None
        else:
            D, F, dist = out
        j = _job(m, mode, D, F, dist)
        t = ctypes.c_uint64()
        _check(_lib.edt_serve_submit(self._s, ctypes.byref(j), ctypes.byref(t)))
        self._live[t.value] = (m, D, F, dist)
        return t.value

    def poll(self, ticket: int):
        """None while running; else (latency_s, (D, F, dist))."""
        lat = ctypes.c_double()
        st = _lib.edt_serve_poll(self._s, ctypes.c_uint64(ticket), ctypes.byref(lat))
        if st == EDT_ERR_NOT_READY:
            return None
        bufs = self._live.pop(ticket, None)
        _check(st)
        return lat.value, bufs[1:]

    def poll_detail(self, ticket: int):
        """None while running; else (latency_s, wait_s, (D, F, dist)), wait_s =
        the time from submission to admission to a stream."""
        lat, wait = ctypes.c_double(), ctypes.c_double()
        st = _lib.edt_serve_poll_detail(self._s, ctypes.c_uint64(ticket), ctypes.byref(lat), ctypes.byref(wait))
        if st == EDT_ERR_NOT_READY:
            return None
        bufs = self._live.pop(ticket, None)
        _check(st)
        return lat.value, wait.value, bufs[1:]

    def close(self):
        if self._s:
            _check(_lib.edt_serve_destroy(self._s))
            self._s = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def version() -> str:
    return _lib.edt_version().decode()


def _check(status: int):
    if status != EDT_OK:
        raise EdtError(status, _lib.edt_last_error().decode())


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _mask_arg(mask: torch.Tensor) -> torch.Tensor:
    if not isinstance(mask, torch.Tensor) or not mask.is_cuda:
        raise TypeError("mask must be a CUDA tensor")
    if mask.dtype == torch.bool:
        mask = mask.view(torch.uint8)
    if mask.dtype != torch.uint8:
        raise TypeError(f"mask must be uint8 or bool, got {mask.dtype}")
    if mask.dim() not in (2, 3):
        raise ValueError("mask must be 2-D [H, W] or 3-D [D, H, W]")
    return mask.contiguous()


def _shape_arr(shape):
    return (ctypes.c_int * len(shape))(*[int(s) for s in shape])


def sq2d(mask, mode: int = TO_OBJECT, out=None, stream=None) -> torch.Tensor:
    """Squared 2-D EDT (int32)."""
    m = _mask_arg(mask)
    assert m.dim() == 2
    D = out if out is not None else torch.empty(m.shape, dtype=torch.int32, device=m.device)
    _check(_lib.edt_sq2d(_ptr(m), m.shape[0], m.shape[1], int(mode), _ptr(D), _stream_handle(stream)))
    return D


def sq3d(mask, mode: int = TO_OBJECT, out=None, stream=None) -> torch.Tensor:
    """Squared 3-D EDT (int32)."""
    m = _mask_arg(mask)
    assert m.dim() == 3
    D = out if out is not None else torch.empty(m.shape, dtype=torch.int32, device=m.device)
    _check(_lib.edt_sq3d(_ptr(m), m.shape[0], m.shape[1], m.shape[2], int(mode), _ptr(D),
                         _stream_handle(stream)))
    return D


def feature(mask, mode: int = TO_OBJECT, want_D: bool = True, want_dist: bool = False,
            out=None, stream=None):
    """Squared EDT + feature map (+ optional float32 sqrt).

    Returns (D, F) or (D, F, dist); D is None when want_D is False.  `out`
    may supply preallocated (D, F, dist) tensors (entries may be None)."""
    m = _mask_arg(mask)
    if out is not None:
        D, F, dist = out
    else:
        D = torch.empty(m.shape, dtype=torch.int32, device=m.device) if want_D else None
        F = torch.empty(m.shape, dtype=torch.int32, device=m.device)
        dist = torch.empty(m.shape, dtype=torch.float32, device=m.device) if want_dist else None
    _check(_lib.edt_feature(_ptr(m), m.dim(), _shape_arr(m.shape), int(mode), _ptr(D), _ptr(F),
                            _ptr(dist), _stream_handle(stream)))
    return (D, F, dist) if (want_dist or (out is not None and out[2] is not None)) else (D, F)


def cityblock(mask, mode: int = TO_OBJECT, out=None, stream=None):
    """City-block distance transform of a 2-D uint8 CUDA tensor (Sec. 2.1):
    int32 distances, INT32_MAX without a source."""
    m = _mask_arg(mask)
    if m.dim() != 2:
        raise ValueError("the city-block transform takes 2-D images")
    D = out if out is not None else torch.empty(m.shape, dtype=torch.int32, device=m.device)
    _check(_lib.edt_cityblock2d(_ptr(m), m.shape[0], m.shape[1], int(mode), _ptr(D), _stream_handle(stream)))
    return D


def chamfer43(mask, mode: int = TO_OBJECT, out=None, stream=None):
    """Chamfer 4-3 distance transform of a 2-D uint8 CUDA tensor (Sec. 2.2):
    int32 distances (3 per straight step, 4 per diagonal step), INT32_MAX
    without a source."""
    m = _mask_arg(mask)
    if m.dim() != 2:
        raise ValueError("the chamfer transform takes 2-D images")
    D = out if out is not None else torch.empty(m.shape, dtype=torch.int32, device=m.device)
    _check(_lib.edt_chamfer43_2d(_ptr(m), m.shape[0], m.shape[1], int(mode), _ptr(D), _stream_handle(stream)))
    return D


def feature_pair(mask, want_D: bool = True, out=None, stream=None):
    """Both transforms of one mask from one read of it: returns
    ((D_obj, F_obj), (D_bg, F_bg)) -- to object and to background."""
    m = _mask_arg(mask)
    if out is not None:
        (Do, Fo), (Db, Fb) = out
    else:
        mk = lambda: torch.empty(m.shape, dtype=torch.int32, device=m.device)  # noqa: E731
        Do = mk() if want_D else None
        Fo = mk()
        Db = mk() if want_D else None
        Fb = mk()
    _check(_lib.edt_feature_pair(_ptr(m), m.dim(), _shape_arr(m.shape), _ptr(Do), _ptr(Fo), _ptr(Db),
                                 _ptr(Fb), _stream_handle(stream)))
    return (Do, Fo), (Db, Fb)


def feature_host(mask: np.ndarray, mode: int = TO_OBJECT, D=None, F=None, dist=None,
                 want_dist: bool = False, stream=None):
    """edt_feature_host on host (numpy or pinned torch CPU) buffers; returns
    (D, F[, dist]) filled in place, synchronously."""
    if isinstance(mask, torch.Tensor):
        m = mask.contiguous()
        shape = tuple(m.shape)
        if D is None:
            D = torch.empty(shape, dtype=torch.int32, pin_memory=m.is_pinned())
        if F is None:
            F = torch.empty(shape, dtype=torch.int32, pin_memory=m.is_pinned())
        if want_dist and dist is None:
            dist = torch.empty(shape, dtype=torch.float32, pin_memory=m.is_pinned())
        p = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())  # noqa: E731
    else:
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        shape = m.shape
        if D is None:
            D = np.empty(shape, np.int32)
        if F is None:
            F = np.empty(shape, np.int32)
        if want_dist and dist is None:
            dist = np.empty(shape, np.float32)
        p = lambda a: None if a is None else ctypes.c_void_p(a.ctypes.data)  # noqa: E731
    _check(_lib.edt_feature_host(p(m), len(shape), _shape_arr(shape), int(mode), p(D), p(F),
                                 p(dist), _stream_handle(stream)))
    return (D, F, dist) if want_dist else (D, F)


def feature_pair_host(mask, out=None, want_D: bool = True, stream=None):
    """edt_feature_pair_host on host (numpy or pinned torch CPU) buffers:
    returns ((D_obj, F_obj), (D_bg, F_bg)) filled in place, synchronously."""
    if isinstance(mask, torch.Tensor):
        m = mask.contiguous()
        shape = tuple(m.shape)
        mk = lambda: torch.empty(shape, dtype=torch.int32, pin_memory=m.is_pinned())  # noqa: E731
        p = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())  # noqa: E731
    else:
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        shape = m.shape
        mk = lambda: np.empty(shape, np.int32)  # noqa: E731
        p = lambda a: None if a is None else ctypes.c_void_p(a.ctypes.data)  # noqa: E731
    if out is not None:
        (Do, Fo), (Db, Fb) = out
    else:
        Do, Fo, Db, Fb = (mk() if want_D else None), mk(), (mk() if want_D else None), mk()
    _check(_lib.edt_feature_pair_host(p(m), len(shape), _shape_arr(shape), p(Do), p(Fo), p(Db), p(Fb),
                                      _stream_handle(stream)))
    return (Do, Fo), (Db, Fb)
