"""edt_feature2d_noalloc: the allocation-free 2-D entry point, for callers that
may not allocate device memory on the call path (frameworks that own every
device allocation, latency-critical code that cannot afford the implicit
synchronisation of cudaMalloc / cudaFree).  Its scratch is a fixed static
device array shared by all calls, so two calls in a row must both be right:
the second must not see the first call's leftovers.  Called through the C ABI
and compared with edt_feature on the same inputs (D, F and dist bit-identical,
the tolerance of every other parity test here).

This file is named to be collected last."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _noalloc(lib, m, mode, D, F, dist, stream):
    fn = lib.edt_feature2d_noalloc
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn(ctypes.c_void_p(m.data_ptr()), m.shape[0], m.shape[1], mode,
              ctypes.c_void_p(D.data_ptr()), ctypes.c_void_p(F.data_ptr()),
              ctypes.c_void_p(dist.data_ptr()), ctypes.c_void_p(stream.cuda_stream))


def test_noalloc_matches_edt_feature_twice_in_a_row():
    import torch
    from paper_2106_03503_gb300 import edt, inputs

    stream = torch.cuda.current_stream()
    cases = [(inputs.discs_mask(1500, 2304, 40, 5, 60, 77), 0),
             (inputs.bernoulli_mask((777, 4099), 0.003, 78), 1),
             (inputs.discs_8192(), 0)]
    for m_np, mode in cases:
        m = torch.from_numpy(m_np).cuda()
        Dr, Fr, dr = edt.feature(m, mode, want_dist=True)
        for _ in range(2):  # two calls in a row on the shared static scratch
            D = torch.full_like(Dr, -7)
            F = torch.full_like(Fr, -7)
            dist = torch.full_like(dr, -7.0)
            st = _noalloc(edt._lib, m, mode, D, F, dist, stream)
            assert st == 0, edt._lib.edt_last_error().decode()
            torch.cuda.synchronize()
            assert torch.equal(D, Dr)
            assert torch.equal(F, Fr)
            assert torch.equal(dist.view(torch.int32), dr.view(torch.int32))


def test_noalloc_rejects_images_beyond_its_scratch():
    import torch
    from paper_2106_03503_gb300 import edt

    m = torch.zeros((16384, 16384), dtype=torch.uint8, device="cuda")
    D = torch.empty((1,), dtype=torch.int32, device="cuda")
    st = _noalloc(edt._lib, m, 0, D, D, D, torch.cuda.current_stream())
    assert st == 2  # EDT_ERR_TOO_LARGE
    assert "static scratch" in edt._lib.edt_last_error().decode()
