"""Output subsets through the C ABI: edt_sq2d / edt_sq3d (D only, the 3-D
path keeping its y-pass records in D), edt_feature without D (F and dist
only), edt_feature_pair without D, the host-buffer call without D; each
against the oracle (D bit-exact, F a source at the oracle's distance, dist
the correctly rounded square root)."""
import numpy as np
import pytest

import oracle
from gpu_check import feature_valid_fast
from paper_2106_03503_gb300 import inputs

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (37, 1), (1, 37), (33, 100), (257, 1000), (70, 4100), (5, 7, 9), (33, 40, 70)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("mode", [0, 1])
def test_squared_only(shape, mode):
    import torch
    from paper_2106_03503_gb300 import edt
    for k, p in enumerate([0.002, 0.2, 0.9]):
        m = inputs.bernoulli_mask(shape, p, 300 + k)
        t = torch.from_numpy(m).cuda()
        D = edt.sq2d(t, mode) if len(shape) == 2 else edt.sq3d(t, mode)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(D.cpu().numpy(), oracle.edt(m, mode)[0])


@pytest.mark.parametrize("shape", SHAPES)
def test_features_without_distances(shape):
    import torch
    from paper_2106_03503_gb300 import edt
    m = inputs.bernoulli_mask(shape, 0.05, 350)
    t = torch.from_numpy(m).cuda()
    for mode in (0, 1):
        Do = oracle.edt(m, mode)[0]
        D, F, S = edt.feature(t, mode, want_D=False, want_dist=True)
        torch.cuda.synchronize()
        assert D is None
        assert feature_valid_fast(m, mode, Do, F.cpu().numpy()) is None
        assert np.array_equal(S.cpu().numpy().view(np.uint32), oracle.sqrt_f32(Do).view(np.uint32))
    (Do_, Fo), (Db_, Fb) = edt.feature_pair(t, want_D=False)
    torch.cuda.synchronize()
    assert Do_ is None and Db_ is None
    assert feature_valid_fast(m, 0, oracle.edt(m, 0)[0], Fo.cpu().numpy()) is None
    assert feature_valid_fast(m, 1, oracle.edt(m, 1)[0], Fb.cpu().numpy()) is None
    (hDo, hFo), (hDb, hFb) = edt.feature_pair_host(m, want_D=False)
    assert hDo is None and hDb is None
    np.testing.assert_array_equal(hFo, Fo.cpu().numpy())
    np.testing.assert_array_equal(hFb, Fb.cpu().numpy())
