"""Full-size workloads in the launch configuration the benchmark times,
compared with the oracle on every pixel (the oracle finishes them in
seconds to a minute)."""
import numpy as np
import pytest

import oracle
from gpu_check import check_against_oracle
from paper_2106_03503_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_points_512_plain():
    m = inputs.points_512()
    check_against_oracle(m, 0)


@pytest.mark.parametrize("mode", [0, 1])
def test_discs_8192_both_modes(mode):
    m = inputs.discs_8192()
    check_against_oracle(m, mode, want_dist=False)


def test_blobs_512cube():
    m = inputs.blobs_512cube()
    check_against_oracle(m, 0, want_dist=False)


def test_discs_8192_pair_as_benchmarked():
    """The benchmark's step: edt_feature_pair on the 8192^2 discs mask (one
    column pass and one row launch for both transforms); D equal to the
    oracle on every pixel of both transforms, F a nearest source."""
    import torch
    from gpu_check import assert_same_features, feature_valid_fast
    from paper_2106_03503_gb300 import edt
    m_np = inputs.discs_8192()
    (Do, Fo), (Db, Fb) = edt.feature_pair(torch.from_numpy(m_np).cuda())
    torch.cuda.synchronize()
    for mode, (D, F) in ((0, (Do, Fo)), (1, (Db, Fb))):
        D, F = D.cpu().numpy(), F.cpu().numpy()
        D_or, F_or = oracle.edt(m_np, mode)
        np.testing.assert_array_equal(D, D_or)
        assert feature_valid_fast(m_np, mode, D, F) is None
        assert_same_features(F, F_or)


def test_discs_8192_pair_host_as_benchmarked():
    """bench.py's e2e call (host buffers, row pass in four band ranges with
    overlapped copies) on the full 8192^2 workload, against the oracle."""
    import torch
    from paper_2106_03503_gb300 import edt
    m_np = inputs.discs_8192()
    from gpu_check import assert_same_features
    (Do, Fo), (Db, Fb) = edt.feature_pair_host(torch.from_numpy(m_np).pin_memory())
    for mode, (D, F) in ((0, (Do, Fo)), (1, (Db, Fb))):
        D_or, F_or = oracle.edt(m_np, mode)
        np.testing.assert_array_equal(D.numpy(), D_or)
        assert_same_features(F.numpy(), F_or)


def _sparse_sources_check(shape, n_src, seed, mode):
    """Largest accepted shapes: a few random sources (mode 0) or a few random
    background pixels (mode 1); D and F checked on 20000 sampled pixels
    against brute force over the sources (exact squared distances)."""
    import torch
    from paper_2106_03503_gb300 import edt
    rng = np.random.default_rng(seed)
    n = int(np.prod(shape))
    idx = rng.choice(n, size=n_src, replace=False)
    flat = torch.zeros(n, dtype=torch.uint8, device="cuda") if mode == 0 else \
        torch.ones(n, dtype=torch.uint8, device="cuda")
    flat[torch.from_numpy(idx).cuda()] = 1 if mode == 0 else 0
    D, F = edt.feature(flat.view(shape), mode)
    torch.cuda.synchronize()
    src = np.stack(np.unravel_index(idx, shape), -1).astype(np.int64)
    sample = rng.choice(n, size=20000, replace=False)
    p = np.stack(np.unravel_index(sample, shape), -1).astype(np.int64)
    want = ((p[:, None, :] - src[None, :, :]) ** 2).sum(-1).min(1)
    samp = torch.from_numpy(sample).cuda()
    got_D = D.view(-1)[samp].cpu().numpy().astype(np.int64)
    got_F = F.view(-1)[samp].cpu().numpy().astype(np.int64)
    np.testing.assert_array_equal(got_D, want)
    assert np.all(np.isin(got_F, idx))
    q = np.stack(np.unravel_index(got_F, shape), -1)
    np.testing.assert_array_equal(((p - q) ** 2).sum(-1), want)


@pytest.mark.parametrize("mode", [0, 1])
def test_largest_2d_image(mode):
    """32767 x 16384 (537 M pixels, the largest side lengths accepted)."""
    _sparse_sources_check((32767, 16384), 40, 5 + mode, mode)


def test_largest_3d_lines():
    """64 x 2048 x 1024: the largest y and x extents the 3-D passes accept."""
    _sparse_sources_check((64, 2048, 1024), 30, 9, 0)
