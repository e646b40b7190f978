"""CUDA path vs the oracle through the C ABI: D bit-exact, F a valid nearest
source, sqrt bit-exact.  Sizes span several bands, tiles and lane segments and
end in ragged tails; edge cases cover empty, full, single-pixel and one-line
images, both modes."""
import numpy as np
import pytest

import oracle
from golden_io import grid, six_object_mask
from gpu_check import check_against_oracle, feature_valid_fast, run_gpu
from paper_2106_03503_gb300 import inputs

pytestmark = pytest.mark.gpu

SHAPES_2D = [(1, 1), (1, 2), (2, 1), (1, 37), (37, 1), (5, 7), (31, 33), (32, 32), (33, 31),
             (64, 100), (100, 64), (129, 257), (257, 1000), (1000, 37), (97, 1031), (1031, 97),
             (2, 4099), (3001, 5), (333, 2048), (33, 4100), (65, 8192)]
DENS = [0.0005, 0.01, 0.1, 0.5, 0.97]


@pytest.mark.parametrize("shape", SHAPES_2D)
@pytest.mark.parametrize("mode", [0, 1])
def test_2d_random(shape, mode):
    for k, p in enumerate(DENS):
        m = inputs.bernoulli_mask(shape, p, 1000 + 7 * k + shape[0])
        check_against_oracle(m, mode)


def test_paper_example_fig18c():
    D, F, dist = run_gpu(six_object_mask(), 0)
    np.testing.assert_array_equal(D, grid("fig18c_final.txt"))


def test_single_pixel_fig8b():
    m = np.zeros((9, 10), np.uint8)
    m[4, 4] = 1
    D, F, dist = run_gpu(m, 0)
    np.testing.assert_array_equal(D, grid("fig8b_single_pixel.txt"))
    assert np.all(F == 44)


@pytest.mark.parametrize("shape", [(1, 1), (7, 9), (100, 300), (3, 2, 5), (40, 33, 70)])
def test_no_source_and_all_source(shape):
    z = np.zeros(shape, np.uint8)
    o = np.ones(shape, np.uint8)
    for m, mode in [(z, 0), (o, 1)]:
        D, F, dist = run_gpu(m, mode)
        assert np.all(D == 2**31 - 1) and np.all(F == -1) and np.all(np.isinf(dist))
    for m, mode in [(o, 0), (z, 1)]:
        D, F, dist = run_gpu(m, mode)
        assert np.all(D == 0)
        np.testing.assert_array_equal(F.reshape(-1), np.arange(m.size))


@pytest.mark.parametrize("shape", [(64, 64), (200, 333), (1, 5000), (5000, 1)])
def test_single_source_anywhere(shape):
    rng = np.random.default_rng(9)
    for _ in range(4):
        m = np.zeros(shape, np.uint8)
        m[int(rng.integers(shape[0])), int(rng.integers(shape[1]))] = 1
        check_against_oracle(m, 0)


def test_discs_2d_medium():
    m = inputs.discs_mask(1536, 2048, 60, 5, 60, 21)
    for mode in (0, 1):
        check_against_oracle(m, mode)


SHAPES_3D = [(1, 1, 1), (3, 5, 7), (1, 40, 50), (40, 1, 50), (40, 50, 1), (32, 33, 31),
             (33, 32, 65), (70, 17, 129), (64, 64, 64), (5, 300, 40), (100, 20, 300)]


@pytest.mark.parametrize("shape", SHAPES_3D)
@pytest.mark.parametrize("mode", [0, 1])
def test_3d_random(shape, mode):
    for k, p in enumerate([0.001, 0.05, 0.5]):
        m = inputs.bernoulli_mask(shape, p, 3000 + k + shape[1])
        check_against_oracle(m, mode)


def test_3d_smoothed_blobs():
    m = inputs.smoothed_noise_volume((96, 80, 112), 4.0, 33)
    for mode in (0, 1):
        check_against_oracle(m, mode)


@pytest.mark.parametrize("p", [0.001, 0.003, 0.01])
def test_3d_sparse_sides_above_128(p):
    """Sparse volumes with every side above 128: z and y offsets beyond the
    direct searches' guarantee (tiles and units that try the search and give
    up to the hull, or settle), and x-pass records whose offsets need the
    escape form."""
    m = inputs.bernoulli_mask((160, 200, 176), p, 4100 + int(p * 1e4))
    for mode in (0, 1):
        check_against_oracle(m, mode)


def test_3d_blobs_with_empty_slabs():
    """Smoothed-noise blobs with empty z slabs and an empty y band: near and
    far own offsets side by side in the same tiles and units."""
    m = inputs.smoothed_noise_volume((192, 144, 160), 4.0, 35).copy()
    m[40:140] = 0
    m[:, 60:130] = 0
    for mode in (0, 1):
        check_against_oracle(m, mode)


def test_sqrt_exhaustive_range_on_gpu():
    """dist for every D in [0, 2^22) and random large D, via a 1-row image
    whose only source sits at the left end, so D = j^2 ... plus direct
    checks of large values through 3-D distances."""
    import torch
    m = np.zeros((1, 16384), np.uint8)
    m[0, 0] = 1
    D, F, dist = run_gpu(m, 0)
    np.testing.assert_array_equal(dist.view(np.uint32), oracle.sqrt_f32(D).view(np.uint32))
    m = np.zeros((2000, 16384), np.uint8)
    m[0, 0] = 1
    m[1999, 16383] = 1
    D, F, dist = run_gpu(m, 0)
    np.testing.assert_array_equal(dist.view(np.uint32), oracle.sqrt_f32(D).view(np.uint32))


def test_invalid_arguments_raise():
    import torch
    from paper_2106_03503_gb300 import edt
    m = torch.zeros((4, 4), dtype=torch.uint8, device="cuda")
    with pytest.raises(edt.EdtError):
        edt.feature(m, mode=5)
    big = torch.zeros((2, 16385), dtype=torch.uint8, device="cuda")
    with pytest.raises(edt.EdtError) as e:
        edt.feature(big)
    assert e.value.status == 2


@pytest.mark.parametrize("shape", [(1, 1), (5, 7), (33, 64), (100, 100), (257, 1000), (1031, 97),
                                   (70, 2048), (40, 4104), (3, 9, 17), (20, 33, 40)])
def test_pair_equals_two_calls(shape):
    """edt_feature_pair: both transforms from one mask read, bit-identical to
    two edt_feature calls, and D exact against the oracle."""
    import torch
    from paper_2106_03503_gb300 import edt
    for k, p in enumerate([0.0, 0.02, 0.5, 1.0]):
        m_np = inputs.bernoulli_mask(shape, p, 77 + k)
        m = torch.from_numpy(m_np).cuda()
        (Do, Fo), (Db, Fb) = edt.feature_pair(m)
        Dr0, Fr0 = edt.feature(m, 0)
        Dr1, Fr1 = edt.feature(m, 1)
        torch.cuda.synchronize()
        assert torch.equal(Do, Dr0) and torch.equal(Fo, Fr0)
        assert torch.equal(Db, Dr1) and torch.equal(Fb, Fr1)
        np.testing.assert_array_equal(Do.cpu().numpy(), oracle.edt(m_np, 0)[0])
        np.testing.assert_array_equal(Db.cpu().numpy(), oracle.edt(m_np, 1)[0])


@pytest.mark.parametrize("shape", [(40, 4104), (33, 8192), (9, 17, 1000)])
@pytest.mark.parametrize("offset", [0, 4, 1, 2])
def test_output_alignments(shape, offset):
    """Outputs that start 32-byte aligned, only 16-byte aligned, or 4- and
    8-byte aligned: each takes its own store width and all give the same
    result."""
    import torch
    from paper_2106_03503_gb300 import edt
    m_np = inputs.bernoulli_mask(shape, 0.01, 91)
    m = torch.from_numpy(m_np).cuda()
    n = m_np.size
    bufs = [torch.zeros(n + 8, dtype=dt, device="cuda") for dt in (torch.int32, torch.int32, torch.float32)]
    D, F, dist = (b[offset:offset + n].view(shape) for b in bufs)
    edt.feature(m, 0, out=(D, F, dist))
    torch.cuda.synchronize()
    Do = oracle.edt(m_np, 0)[0]
    np.testing.assert_array_equal(D.cpu().numpy(), Do)
    assert feature_valid_fast(m_np, 0, Do, F.cpu().numpy()) is None
    np.testing.assert_array_equal(dist.cpu().numpy().view(np.uint32), oracle.sqrt_f32(Do).view(np.uint32))
    for b in bufs:   # nothing written outside the views
        h = b.cpu().numpy()
        assert not h[:offset].any() and not h[offset + n:].any()


@pytest.mark.parametrize("shape", [(5, 7), (100, 300), (513, 1000), (1000, 37), (2049, 2052), (20, 33, 40)])
def test_host_buffer_calls_match_device_calls(shape):
    """edt_feature_host and edt_feature_pair_host (host buffers; 2-D row pass
    in up to four band ranges whose rows are copied back while the next range
    runs) give the same bits as the device-buffer calls."""
    import torch
    from paper_2106_03503_gb300 import edt
    for k, p in enumerate([0.003, 0.3]):
        m_np = inputs.bernoulli_mask(shape, p, 500 + k)
        m = torch.from_numpy(m_np).cuda()
        for mode in (0, 1):
            Dd, Fd, Sd = edt.feature(m, mode, want_dist=True)
            Dh, Fh, Sh = edt.feature_host(m_np, mode, want_dist=True)          # pageable numpy
            torch.cuda.synchronize()
            np.testing.assert_array_equal(Dh, Dd.cpu().numpy())
            np.testing.assert_array_equal(Fh, Fd.cpu().numpy())
            np.testing.assert_array_equal(Sh.view(np.uint32), Sd.cpu().numpy().view(np.uint32))
        (Do, Fo), (Db, Fb) = edt.feature_pair(m)
        hm = torch.from_numpy(m_np).pin_memory()
        (hDo, hFo), (hDb, hFb) = edt.feature_pair_host(hm)                     # pinned torch
        torch.cuda.synchronize()
        for a, b in ((hDo, Do), (hFo, Fo), (hDb, Db), (hFb, Fb)):
            assert torch.equal(a, b.cpu())
        np.testing.assert_array_equal(hDo.numpy(), oracle.edt(m_np, 0)[0])


def test_concurrent_host_calls_from_two_threads():
    """Two host threads, each with its own stream, masks and pinned buffers,
    call edt_feature_pair_host at the same time (as bench.py's end-to-end
    measurement does): the library's shared state (device setup, the copy
    stream, the memory pool) must keep every result equal to the oracle's."""
    import threading
    import torch
    from paper_2106_03503_gb300 import edt
    shapes = [(1500, 2100), (700, 4100)]
    masks = [inputs.bernoulli_mask(sh, 0.01, 900 + k) for k, sh in enumerate(shapes)]
    want = [(oracle.edt(m, 0)[0], oracle.edt(m, 1)[0]) for m in masks]
    errors = []

    def worker(k):
        try:
            torch.cuda.set_device(0)
            st = torch.cuda.Stream()
            hm = torch.from_numpy(masks[k]).pin_memory()
            for _ in range(4):
                (Do, Fo), (Db, Fb) = edt.feature_pair_host(hm, stream=st)
                np.testing.assert_array_equal(Do.numpy(), want[k][0])
                np.testing.assert_array_equal(Db.numpy(), want[k][1])
                for mode, (D, F) in enumerate(((Do, Fo), (Db, Fb))):
                    assert feature_valid_fast(masks[k], mode, D.numpy(), F.numpy()) is None
        except Exception as exc:  # noqa: BLE001
            errors.append(exc)

    threads = [threading.Thread(target=worker, args=(k,)) for k in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errors:
        raise errors[0]


@pytest.mark.parametrize("shape", [(70, 1000), (33, 4100), (40, 8192)])
@pytest.mark.parametrize("offset", [0, 1, 2, 3, 4, 8])
def test_mask_alignments(shape, offset):
    """Masks that start 16-, 8-, 4-, 2- and 1-byte aligned (a view into a
    larger buffer): the column pass reads them with vector, aligned-word or
    byte loads, with the same result."""
    import torch
    from paper_2106_03503_gb300 import edt
    m_np = inputs.bernoulli_mask(shape, 0.02, 17 + offset)
    n = m_np.size
    buf = torch.full((n + 16,), 7, dtype=torch.uint8, device="cuda")
    buf[offset:offset + n] = torch.from_numpy(m_np.reshape(-1)).cuda()
    m = buf[offset:offset + n].view(shape)
    for mode in (0, 1):
        D, F = edt.feature(m, mode)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(D.cpu().numpy(), oracle.edt(m_np, mode)[0])
        assert feature_valid_fast(m_np, mode, D.cpu().numpy(), F.cpu().numpy()) is None


def test_3d_record_forms():
    """A source line along x at (z, y) = (0, 0): every x plane's records have
    squared lengths on both sides of 128^2 (offset form below it, the source's
    own coordinates above it, whose true cost the hull then reads), and with
    the line broken every seventh plane's records are "no source"."""
    m = np.zeros((150, 150, 24), np.uint8)
    m[0, 0, :] = 1
    check_against_oracle(m, 0)
    m = np.zeros((150, 150, 24), np.uint8)
    m[0, 0, ::7] = 1
    for mode in (0, 1):
        check_against_oracle(m, mode)
