"""edt_feature2d_noalloc: the allocation-free 2-D entry point, for callers that
may not allocate device memory on the call path (frameworks that own every
device allocation, latency-critical code that cannot afford the implicit
synchronisation of cudaMalloc / cudaFree).  Its scratch is a fixed static
device array shared by all calls, so two calls in a row must both be right:
the second must not see the first call's leftovers.  Called through the C ABI
and compared with edt_feature on the same inputs (D, F and dist bit-identical,
the tolerance of every other parity test here), with and without the optional
D and dist outputs; around a call, neither the device's default memory pool
nor the device's free memory may grow or shrink.

This file is named to be collected last."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# CUmemPool_attribute values (cuda.h)
_USED_MEM_CURRENT = 7
_USED_MEM_HIGH = 8


def _noalloc(lib, m, mode, D, F, dist, stream):
    fn = lib.edt_feature2d_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    ptr = lambda t: ctypes.c_void_p(t.data_ptr() if t is not None else 0)
    return fn(ctypes.c_void_p(m.data_ptr()), m.shape[0], m.shape[1], mode,
              ptr(D), ptr(F), ptr(dist), ctypes.c_void_p(stream.cuda_stream))


class _DeviceMemory:
    """Driver-level view of device memory: the default memory pool's used
    bytes (with its high-water mark) and the free bytes of the device."""

    def __init__(self, device):
        self.cu = ctypes.CDLL("libcuda.so.1")
        self.pool = ctypes.c_void_p()
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), device) == 0
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def _attr(self, a):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, a, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)   # resets the high-water mark to the current use
        assert self.cu.cuMemPoolSetAttribute(self.pool, _USED_MEM_HIGH, ctypes.byref(zero)) == 0

    def snapshot(self):
        free, total = ctypes.c_size_t(), ctypes.c_size_t()
        assert self.cu.cuMemGetInfo_v2(ctypes.byref(free), ctypes.byref(total)) == 0
        return {"pool_used": self._attr(_USED_MEM_CURRENT), "pool_high": self._attr(_USED_MEM_HIGH),
                "free": free.value}


def test_noalloc_matches_edt_feature_twice_in_a_row():
    import torch
    from paper_2106_03503_gb300 import edt, inputs

    stream = torch.cuda.current_stream()
    mem = _DeviceMemory(torch.cuda.current_device())
    cases = [(inputs.discs_mask(1500, 2304, 40, 5, 60, 77), 0),
             (inputs.bernoulli_mask((777, 4099), 0.003, 78), 1),
             (inputs.discs_8192(), 0)]
    for m_np, mode in cases:
        m = torch.from_numpy(m_np).cuda()
        Dr, Fr, dr = edt.feature(m, mode, want_dist=True)
        torch.cuda.synchronize()
        for rep in range(2):  # two calls in a row on the shared static scratch
            D = torch.full_like(Dr, -7)
            F = torch.full_like(Fr, -7)
            dist = torch.full_like(dr, -7.0)
            torch.cuda.synchronize()
            mem.reset_high()
            before = mem.snapshot()
            st = _noalloc(edt._lib, m, mode, D, F, dist, stream)
            assert st == 0, edt._lib.edt_last_error().decode()
            torch.cuda.synchronize()
            after = mem.snapshot()
            assert torch.equal(D, Dr)
            assert torch.equal(F, Fr)
            assert torch.equal(dist.view(torch.int32), dr.view(torch.int32))
            # no stream-ordered allocation inside the call ...
            assert after["pool_high"] == before["pool_used"] == after["pool_used"], (before, after)
            # ... and no plain allocation either (the first call on a device
            # may map the static array itself, so this is checked from the
            # second call on)
            if rep > 0:
                assert after["free"] == before["free"], (before, after)


def test_noalloc_optional_outputs():
    """D and dist are optional (NULL); F alone, F with D, F with dist give the
    same bits as the full call."""
    import torch
    from paper_2106_03503_gb300 import edt, inputs

    stream = torch.cuda.current_stream()
    m = torch.from_numpy(inputs.discs_mask(900, 1000, 25, 5, 60, 79)).cuda()
    for mode in (0, 1):
        Dr, Fr, dr = edt.feature(m, mode, want_dist=True)
        for want_D, want_dist in ((False, False), (True, False), (False, True)):
            D = torch.full_like(Dr, -7) if want_D else None
            F = torch.full_like(Fr, -7)
            dist = torch.full_like(dr, -7.0) if want_dist else None
            st = _noalloc(edt._lib, m, mode, D, F, dist, stream)
            assert st == 0, edt._lib.edt_last_error().decode()
            torch.cuda.synchronize()
            assert torch.equal(F, Fr)
            if want_D:
                assert torch.equal(D, Dr)
            if want_dist:
                assert torch.equal(dist.view(torch.int32), dr.view(torch.int32))


def test_noalloc_rejects_images_beyond_its_scratch():
    import torch
    from paper_2106_03503_gb300 import edt

    m = torch.zeros((16384, 16384), dtype=torch.uint8, device="cuda")
    D = torch.empty((1,), dtype=torch.int32, device="cuda")
    st = _noalloc(edt._lib, m, 0, D, D, D, torch.cuda.current_stream())
    assert st == 2  # EDT_ERR_TOO_LARGE
    assert "static scratch" in edt._lib.edt_last_error().decode()
