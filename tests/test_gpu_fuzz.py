"""Seeded random cases over every entry point against the oracle: 2-D
masks of random shape (small, medium, up to 16383 columns wide or 9000 rows
tall) and structure (Bernoulli at densities from 1e-4 to 1, or the lines,
checkerboards, point sets and discs of test_gpu_structured), through
edt_feature (with sqrt), edt_feature_pair, edt_feature_pair_host, edt_batch,
the city-block and chamfer transforms, and random 3-D volumes.  D is
compared bit for bit, F checked as a source at distance D, sqrt bit for bit.
The case count is fixed (FUZZ_CASES, default 140); a case's seed reproduces
it."""
import os

import numpy as np
import pytest
import torch

import oracle
from gpu_check import feature_valid_fast
from test_gpu_structured import KINDS, structured

pytestmark = pytest.mark.gpu
SEED0 = 20250


def mask2d(rng):
    r = rng.random()
    if r < 0.3:
        H, W = int(rng.integers(1, 300)), int(rng.integers(1, 300))
    elif r < 0.6:
        H, W = int(rng.integers(1, 2500)), int(rng.integers(1, 2500))
    elif r < 0.8:
        H, W = int(rng.integers(1, 40)), int(rng.integers(1, 16384))
    else:
        H, W = int(rng.integers(1, 9000)), int(rng.integers(1, 60))
    if rng.random() < 0.5:
        return (rng.random((H, W)) < 10 ** rng.uniform(-4, 0)).astype(np.uint8)
    return structured(KINDS[int(rng.integers(len(KINDS)))], (H, W), rng)


def check(name, m, mode, D, F=None, dist=None):
    Do, Fo = oracle.edt(m, mode)
    if not np.array_equal(D, Do):
        raise AssertionError(f"{name}: D mismatch at {int((D != Do).sum())} px")
    if F is not None:
        msg = feature_valid_fast(m, mode, D, F)
        if msg:
            raise AssertionError(f"{name}: {msg}")
        if not np.array_equal(F, Fo):   # the oracle breaks ties the same way
            raise AssertionError(f"{name}: F differs from the oracle's at {int((F != Fo).sum())} px")
    if dist is not None and not np.array_equal(dist.view(np.uint32), oracle.sqrt_f32(Do).view(np.uint32)):
        raise AssertionError(f"{name}: sqrt mismatch")


def run_case(seed):
    from paper_2106_03503_gb300 import edt
    rng = np.random.default_rng(seed)
    kind = ["feature", "pair", "host", "batch", "cityblock", "chamfer", "vol"][seed % 7]
    if kind == "vol":
        sh = tuple(int(rng.integers(1, n)) for n in (70, 300, 300))
        m = (rng.random(sh) < 10 ** rng.uniform(-4, 0)).astype(np.uint8)
        mode = int(rng.integers(2))
        D, F, S = edt.feature(torch.from_numpy(m).cuda(), mode, want_dist=True)
        torch.cuda.synchronize()
        check("vol", m, mode, D.cpu().numpy(), F.cpu().numpy(), S.cpu().numpy())
        return
    if kind == "batch":
        ms = [mask2d(rng)[:, :2048] for _ in range(int(rng.integers(1, 12)))]
        mode = int(rng.integers(2))
        outs = edt.batch([torch.from_numpy(np.ascontiguousarray(m)).cuda() for m in ms], mode)
        for m, (D, F) in zip(ms, outs):
            check("batch", np.ascontiguousarray(m), mode, D.cpu().numpy(), F.cpu().numpy())
        return
    m = mask2d(rng)
    mode = int(rng.integers(2))
    if kind == "chamfer":
        m = np.ascontiguousarray(m[:, :14336])
    t = torch.from_numpy(m).cuda()
    if kind == "feature":
        D, F, S = edt.feature(t, mode, want_dist=True)
        torch.cuda.synchronize()
        check(kind, m, mode, D.cpu().numpy(), F.cpu().numpy(), S.cpu().numpy())
    elif kind == "pair":
        (Do, Fo), (Db, Fb) = edt.feature_pair(t)
        torch.cuda.synchronize()
        check(kind, m, 0, Do.cpu().numpy(), Fo.cpu().numpy())
        check(kind, m, 1, Db.cpu().numpy(), Fb.cpu().numpy())
    elif kind == "host":
        (Do, Fo), (Db, Fb) = edt.feature_pair_host(m)
        check(kind, m, 0, Do, Fo)
        check(kind, m, 1, Db, Fb)
    elif kind == "cityblock":
        D = edt.cityblock(t, mode)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(D.cpu().numpy(), oracle.cityblock(m, mode))
    else:
        D = edt.chamfer43(t, mode)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(D.cpu().numpy(), oracle.chamfer43(m, mode))


@pytest.mark.parametrize("seed", range(SEED0, SEED0 + int(os.environ.get("FUZZ_CASES", "140"))))
def test_random_case(seed):
    run_case(seed)
