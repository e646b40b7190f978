"""edt_autotune on the GPU: it picks warp counts from its candidate sets for
the shape's class, later calls of that class use them, and the results are
the same bits as under the built-in rule (and the oracle's D)."""
import numpy as np
import pytest

import oracle
from paper_2106_03503_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(700, 1500), (96, 200, 300)])
def test_autotune_keeps_results(shape, tmp_path):
    import torch
    from paper_2106_03503_gb300 import edt
    m_np = inputs.bernoulli_mask(shape, 0.02, 77)
    m = torch.from_numpy(m_np).cuda()
    before = [edt.feature(m, mode) for mode in (0, 1)]
    torch.cuda.synchronize()
    before = [(D.cpu().numpy(), F.cpu().numpy()) for D, F in before]
    chosen = edt.autotune(m, 0)
    if len(shape) == 2:
        assert chosen["rows2d"] in (4, 8, 16) and chosen["ypass"] == 0 and chosen["xpass"] == 0
    else:
        assert chosen["rows2d"] == 0 and chosen["ypass"] in (4, 8, 16, 32) and chosen["xpass"] in (8, 16, 32)
    for mode, (Db, Fb) in enumerate(before):
        D, F = edt.feature(m, mode)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(D.cpu().numpy(), Db)
        np.testing.assert_array_equal(F.cpu().numpy(), Fb)
        np.testing.assert_array_equal(Db, oracle.edt(m_np, mode)[0])
    # every candidate gives the same bits, not only the chosen one
    path = tmp_path / "t.txt"
    edt.tune_save(str(path))
    cls = [str(len(shape))] + [str((s - 1).bit_length()) for s in shape] + ["0"] * (3 - len(shape))
    saved = [l.split() for l in path.read_text().splitlines() if not l.startswith("#")]
    assert [l[:4] for l in saved].count(cls) == 1
    cands = (4, 8, 16) if len(shape) == 2 else (4, 16, 32)
    for nw in cands:
        line = cls + ([str(nw), "0", "0"] if len(shape) == 2 else ["0", str(nw), str(nw)])
        path.write_text(" ".join(line) + "\n")
        edt.tune_load(str(path))
        D, F = edt.feature(m, 0)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(D.cpu().numpy(), before[0][0])
        np.testing.assert_array_equal(F.cpu().numpy(), before[0][1])
    path.write_text(" ".join(cls + ["0", "0", "0"]) + "\n")
    edt.tune_load(str(path))                 # back to the built-in rule for later tests
