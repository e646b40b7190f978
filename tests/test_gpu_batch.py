"""Batched transforms (edt_plan_create / edt_batch): every job's D must equal
the oracle's bit for bit, F must name a nearest source and dist must be the
correctly rounded square root; and every job is bit-identical to a plain
edt_feature call on the same mask.  Mixed batches of uneven sizes and modes,
plan reuse, and the full batch workload (4096 masks, sides 64..1024, densities
0.001..0.1)."""
import numpy as np
import pytest

import oracle
from gpu_check import feature_valid_fast
from paper_2106_03503_gb300 import inputs

pytestmark = pytest.mark.gpu


def _plain(edt, m, mode, want_dist):
    return edt.feature(m, mode, want_dist=want_dist)


def _jobs(torch, edt, specs, seed):
    rng = np.random.default_rng(seed)
    jobs, refs = [], []
    for k, (H, W, p, mode, want_D, want_dist) in enumerate(specs):
        m = torch.from_numpy(inputs.bernoulli_mask((H, W), p, seed * 1000 + k)).cuda()
        D = torch.full((H, W), -5, dtype=torch.int32, device="cuda") if want_D else None
        F = torch.full((H, W), -5, dtype=torch.int32, device="cuda")
        dist = torch.full((H, W), -5.0, dtype=torch.float32, device="cuda") if want_dist else None
        jobs.append((m, mode, D, F, dist))
        refs.append(edt.feature(m, mode, want_dist=True))
    return jobs, refs


def _check(jobs, refs, torch):
    torch.cuda.synchronize()
    for k, ((m, mode, D, F, dist), (Dr, Fr, dr)) in enumerate(zip(jobs, refs)):
        # against the oracle
        m_np = m.cpu().numpy()
        Do, _ = oracle.edt(m_np, mode)
        F_np = F.cpu().numpy()
        if D is not None:
            assert np.array_equal(D.cpu().numpy(), Do), k
        msg = feature_valid_fast(m_np, mode, Do, F_np)
        assert msg is None, (k, msg)
        if dist is not None:
            assert np.array_equal(dist.cpu().numpy().view(np.uint32), oracle.sqrt_f32(Do).view(np.uint32)), k
        # and bit-identical to the plain call
        if D is not None:
            assert torch.equal(D, Dr)
        assert torch.equal(F, Fr)
        if dist is not None:
            assert torch.equal(dist.view(torch.int32), dr.view(torch.int32))


def test_mixed_batch_matches_plain_calls():
    import torch
    from paper_2106_03503_gb300 import edt
    rng = np.random.default_rng(1)
    specs = []
    for k in range(60):
        H = int(rng.choice([1, 2, 31, 32, 33, 64, 100, 257, 1000, 1500, 3000]))
        W = int(rng.choice([1, 5, 16, 31, 32, 48, 64, 100, 513, 1024, 1500, 2048]))
        p = float(rng.choice([0.0, 0.001, 0.02, 0.3, 0.9, 1.0]))
        specs.append((H, W, p, int(rng.integers(2)), bool(rng.integers(2)), bool(rng.integers(2))))
    jobs, refs = _jobs(torch, edt, specs, 11)
    plan = edt.Plan(len(jobs), sum(j[0].numel() for j in jobs))
    plan.run(jobs)
    _check(jobs, refs, torch)
    # reuse the plan with another batch, twice (alternating job tables)
    for rep in range(2):
        specs2 = [(int(rng.integers(1, 700)), int(rng.integers(1, 2049)), 0.01, rep, True, False)
                  for _ in range(25)]
        jobs2, refs2 = _jobs(torch, edt, specs2, 20 + rep)
        assert sum(j[0].numel() for j in jobs2) <= sum(j[0].numel() for j in jobs)
        plan.run(jobs2)
        _check(jobs2, refs2, torch)
    plan.close()


def test_batch_errors():
    import torch
    from paper_2106_03503_gb300 import edt
    plan = edt.Plan(2, 10_000)
    m3 = torch.zeros((4, 5, 6), dtype=torch.uint8, device="cuda")
    F3 = torch.empty((4, 5, 6), dtype=torch.int32, device="cuda")
    with pytest.raises(edt.EdtError) as e:
        plan.run([(m3, 0, None, F3, None)])
    assert e.value.status == 1
    wide = torch.zeros((2, 2049), dtype=torch.uint8, device="cuda")
    Fw = torch.empty((2, 2049), dtype=torch.int32, device="cuda")
    with pytest.raises(edt.EdtError) as e:
        plan.run([(wide, 0, None, Fw, None)])
    assert e.value.status == 2
    m = torch.zeros((10, 10), dtype=torch.uint8, device="cuda")
    F = torch.empty((10, 10), dtype=torch.int32, device="cuda")
    with pytest.raises(edt.EdtError):
        plan.run([(m, 0, None, F, None)] * 3)
    plan.close()


def test_full_batch_workload_4096():
    """The batch workload at full size: 4096 masks; all jobs bit-identical to
    plain calls, and a sample checked against the oracle."""
    import torch
    from paper_2106_03503_gb300 import edt
    masks_np = inputs.batch_4096()
    masks = [torch.from_numpy(m).cuda() for m in masks_np]
    outs = edt.batch(masks, 0)
    torch.cuda.synchronize()
    for k in range(0, len(masks), 1):
        Dr, Fr = edt.feature(masks[k], 0)
        D, F = outs[k]
        assert torch.equal(D, Dr) and torch.equal(F, Fr), k
    for k in range(0, len(masks), 128):
        Do, _ = oracle.edt(masks_np[k], 0)
        D, F = outs[k]
        D, F = D.cpu().numpy(), F.cpu().numpy()
        assert np.array_equal(D, Do), k
        assert feature_valid_fast(masks_np[k], 0, D, F) is None
