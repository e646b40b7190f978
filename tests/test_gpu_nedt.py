"""edt_cityblock2d and edt_chamfer43_2d on the GPU against the oracle's
city-block (Sec. 2.1) and chamfer 4-3 (Sec. 2.2) transforms: bit-exact int32
distances on the paper's example, random masks of many shapes (several bands
and row chunks, ragged tails, widths past 8192 columns, both source classes,
empty and full images) and the full 8192 x 8192 discs image."""
import numpy as np
import pytest

import oracle
from golden_io import grid, six_object_mask
from paper_2106_03503_gb300 import inputs

pytestmark = pytest.mark.gpu
INF = np.iinfo(np.int32).max


def _gpu(mask, mode, kind="cityblock"):
    import torch
    from paper_2106_03503_gb300 import edt
    fn = edt.cityblock if kind == "cityblock" else edt.chamfer43
    D = fn(torch.from_numpy(np.ascontiguousarray(mask)).cuda(), mode)
    torch.cuda.synchronize()
    return D.cpu().numpy()


def test_paper_example_fig12():
    got = _gpu(six_object_mask(), 0)
    want = grid("fig12c_cityblock_final.txt")
    want[5, 8] = 2          # printed 3 in the paper: a typo (see the fixture)
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("shape", [(1, 1), (1, 37), (37, 1), (31, 33), (100, 64), (257, 1000), (65, 2052),
                                   (40, 8192), (33, 8200), (9, 16384)])
@pytest.mark.parametrize("mode", [0, 1])
def test_random_masks(shape, mode):
    for k, p in enumerate([0.0, 0.001, 0.05, 0.5, 1.0]):
        m = inputs.bernoulli_mask(shape, p, 900 + 13 * k + shape[1])
        np.testing.assert_array_equal(_gpu(m, mode), oracle.cityblock(m, mode))


def test_unaligned_output():
    import torch
    from paper_2106_03503_gb300 import edt
    m_np = inputs.bernoulli_mask((70, 4104), 0.01, 3)
    buf = torch.zeros(70 * 4104 + 8, dtype=torch.int32, device="cuda")
    D = buf[3:3 + 70 * 4104].view(70, 4104)
    edt.cityblock(torch.from_numpy(m_np).cuda(), 0, out=D)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(D.cpu().numpy(), oracle.cityblock(m_np, 0))
    h = buf.cpu().numpy()
    assert not h[:3].any() and not h[3 + 70 * 4104:].any()


@pytest.mark.parametrize("mode", [0, 1])
def test_full_size_discs(mode):
    m = inputs.discs_8192()
    np.testing.assert_array_equal(_gpu(m, mode), oracle.cityblock(m, mode))


def test_chamfer_paper_example_fig15():
    np.testing.assert_array_equal(_gpu(six_object_mask(), 0, "chamfer"), grid("fig15b_chamfer_final.txt"))


@pytest.mark.parametrize("shape", [(1, 1), (1, 37), (37, 1), (31, 33), (100, 64), (257, 1000), (300, 130),
                                   (65, 2052), (40, 8192), (33, 8200), (9, 14336)])
@pytest.mark.parametrize("mode", [0, 1])
def test_chamfer_random_masks(shape, mode):
    for k, p in enumerate([0.0, 0.001, 0.05, 0.5, 1.0]):
        m = inputs.bernoulli_mask(shape, p, 700 + 11 * k + shape[1])
        np.testing.assert_array_equal(_gpu(m, mode, "chamfer"), oracle.chamfer43(m, mode))


@pytest.mark.parametrize("mode", [0, 1])
def test_chamfer_full_size_discs(mode):
    m = inputs.discs_8192()
    np.testing.assert_array_equal(_gpu(m, mode, "chamfer"), oracle.chamfer43(m, mode))


def test_chamfer_width_limit():
    import torch
    from paper_2106_03503_gb300 import edt
    with pytest.raises(edt.EdtError) as e:
        edt.chamfer43(torch.zeros((2, 14337), dtype=torch.uint8, device="cuda"))
    assert e.value.status == 2
