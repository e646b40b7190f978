"""Helpers for the GPU parity tests: run the CUDA path through the C ABI
binding and compare with the oracle (D bit-exact, F a nearest source,
dist bit-exact to the correctly rounded float32 square root)."""
import numpy as np
import torch

import oracle
from brute import INF32


def feature_valid_fast(mask, mode, D, F):
    """Vectorised check that F(p) is a source at squared distance D(p)."""
    src = (mask != 0) if mode == 0 else (mask == 0)
    Fr = F.reshape(-1).astype(np.int64)
    Dr = D.reshape(-1).astype(np.int64)
    none = Dr == INF32
    if np.any(Fr[none] != -1):
        return "F != -1 where D is infinite"
    ok = ~none
    if not np.all((Fr[ok] >= 0) & (Fr[ok] < src.size)):
        return "F out of range"
    if not np.all(src.reshape(-1)[Fr[ok]]):
        return "F is not a source pixel"
    shape = mask.shape
    strides = [int(np.prod(shape[a + 1:])) for a in range(len(shape))]
    p = np.nonzero(ok)[0]
    q = Fr[ok]
    d2 = np.zeros(p.shape, np.int64)
    for s, n in zip(strides, shape):
        d2 += ((p // s) % n - (q // s) % n) ** 2
    if not np.array_equal(d2, Dr[ok]):
        return "F does not attain D"
    return None


def assert_same_features(F, Fo):
    if not np.array_equal(F, Fo):
        bad = np.argwhere(F != Fo)
        i = tuple(bad[0])
        raise AssertionError(f"F differs from the oracle's at {len(bad)} pixels, first {i}: "
                             f"gpu {F[i]} oracle {Fo[i]}")


def run_gpu(mask, mode, want_dist=True):
    from paper_2106_03503_gb300 import edt
    t = torch.from_numpy(np.ascontiguousarray(mask)).cuda()
    out = edt.feature(t, mode=mode, want_dist=want_dist)
    torch.cuda.synchronize()
    return tuple(None if o is None else o.cpu().numpy() for o in out)


def check_against_oracle(mask, mode, want_dist=True, ref=None, ref_F=None):
    D, F, *rest = run_gpu(mask, mode, want_dist)
    if ref is None:
        Do, Fo = oracle.edt(mask, mode)
    else:
        Do, Fo = ref, ref_F
    if not np.array_equal(D, Do):
        bad = np.argwhere(D != Do)
        i = tuple(bad[0])
        raise AssertionError(f"D mismatch at {len(bad)} pixels, first {i}: gpu {D[i]} oracle {Do[i]}")
    msg = feature_valid_fast(mask, mode, D, F)
    assert msg is None, msg
    if Fo is not None:
        # the same nearest source as the oracle: both keep the rightmost column
        # at an integer intersection (Eq. (6)) and the upper source in a column
        assert_same_features(F, Fo)
    if want_dist:
        dist = rest[0]
        assert np.array_equal(dist.view(np.uint32), oracle.sqrt_f32(Do).view(np.uint32)), "sqrt mismatch"
    return D, F
