"""Seeded structured masks against the oracle through the C ABI: straight
and diagonal lines, checkerboards, sparse and dense point sets and discs, at
shapes next to the kernels' internal boundaries (bands of 32 rows, groups of
up to 32 bands, 32-column tiles, 8-position store chunks, segment lengths and
the 16-byte load widths), both modes.  Lines and checkerboards make many
parabolas meet in one point, so ties are exercised as well; D must be
bit-exact and F a source at distance D."""
import numpy as np
import pytest

from gpu_check import check_against_oracle
from paper_2106_03503_gb300 import inputs

pytestmark = pytest.mark.gpu

SHAPES = [(31, 255), (32, 256), (33, 257), (63, 129), (95, 513), (1023, 40), (1025, 41),
          (2047, 24), (64, 1031), (17, 2049), (130, 8191), (6, 16383)]


def structured(kind, shape, rng):
    H, W = shape
    ii, jj = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    if kind == "rows":            # every k-th row is a source line
        k = int(rng.integers(2, 40))
        return (ii % k == 0).astype(np.uint8)
    if kind == "cols":
        k = int(rng.integers(2, 40))
        return (jj % k == 0).astype(np.uint8)
    if kind == "diag":
        k = int(rng.integers(3, 50))
        return ((ii + jj) % k == 0).astype(np.uint8)
    if kind == "anti":
        k = int(rng.integers(3, 50))
        return ((ii - jj) % k == 0).astype(np.uint8)
    if kind == "checker":
        k = int(rng.integers(1, 9))
        return (((ii // k) + (jj // k)) % 2).astype(np.uint8)
    if kind == "sparse":
        m = np.zeros(shape, np.uint8)
        n = int(rng.integers(1, 6))
        m[rng.integers(0, H, n), rng.integers(0, W, n)] = 1
        return m
    if kind == "dense":
        return (rng.random(shape) < 0.97).astype(np.uint8)
    if kind == "discs":
        return inputs.discs_mask(H, W, max(1, H * W // 20000), 2, 30, int(rng.integers(1 << 30)))
    raise ValueError(kind)


KINDS = ["rows", "cols", "diag", "anti", "checker", "sparse", "dense", "discs"]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("mode", [0, 1])
def test_structured_masks(shape, mode):
    rng = np.random.default_rng(hash((shape, mode)) & 0xFFFFFFFF)
    for kind in KINDS:
        check_against_oracle(structured(kind, shape, rng), mode, want_dist=False)


@pytest.mark.parametrize("shape", [(33, 34, 35), (64, 65, 31), (7, 1025, 9), (5, 9, 1023)])
@pytest.mark.parametrize("mode", [0, 1])
def test_structured_volumes(shape, mode):
    D, H, W = shape
    zz, yy, xx = np.meshgrid(np.arange(D), np.arange(H), np.arange(W), indexing="ij")
    for m in (((zz + yy + xx) % 7 == 0), ((xx % 5 == 0) & (yy % 3 == 0)), ((zz // 2 + yy // 2 + xx // 2) % 2 == 1)):
        check_against_oracle(m.astype(np.uint8), mode, want_dist=False)


@pytest.mark.parametrize("shape", [(31, 255), (33, 257), (1025, 41), (17, 2049), (130, 8191)])
@pytest.mark.parametrize("kind", ["cityblock", "chamfer"])
def test_structured_masks_nedt(shape, kind):
    import torch
    import oracle
    from paper_2106_03503_gb300 import edt
    rng = np.random.default_rng(hash((shape, kind)) & 0xFFFFFFFF)
    gpu = edt.cityblock if kind == "cityblock" else edt.chamfer43
    ref = oracle.cityblock if kind == "cityblock" else oracle.chamfer43
    for k in KINDS:
        m = structured(k, shape, rng)
        for mode in (0, 1):
            got = gpu(torch.from_numpy(np.ascontiguousarray(m)).cuda(), mode)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(got.cpu().numpy(), ref(m, mode), err_msg=f"{kind} {k} mode {mode}")
