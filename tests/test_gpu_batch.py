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
        Do, Fo = oracle.edt(m_np, mode)
        F_np = F.cpu().numpy()
        if D is not None:
            assert np.array_equal(D.cpu().numpy(), Do), k
        msg = feature_valid_fast(m_np, mode, Do, F_np)
        assert msg is None, (k, msg)
        assert np.array_equal(F_np, Fo), (k, "F differs from the oracle's")
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
    # a volume whose rows are wider than the batched x pass holds
    m3 = torch.zeros((2, 4, 1000), dtype=torch.uint8, device="cuda")
    F3 = torch.empty((2, 4, 1000), dtype=torch.int32, device="cuda")
    with pytest.raises(edt.EdtError) as e:
        plan.run([(m3, 0, None, F3, None)])
    assert e.value.status == 2
    m = torch.zeros((10, 10), dtype=torch.uint8, device="cuda")
    F = torch.empty((10, 10), dtype=torch.int32, device="cuda")
    with pytest.raises(edt.EdtError):
        plan.run([(m, 0, None, F, None)] * 3)            # more jobs than n_max
    with pytest.raises(edt.EdtError) as e:
        plan.autotune([(m, 0, None, F, None)] * 3)       # the autotuner's batches must fit the plan too
    assert e.value.status == 1
    with pytest.raises(edt.EdtError) as e:
        plan.run([(m, 5, None, F, None)])                # bad mode
    assert e.value.status == 1
    plan.close()


def _mixed_specs(rng, n):
    """2-D jobs up to 2048 wide, wider 2-D jobs and 3-D volumes, mixed."""
    specs = []
    for k in range(n):
        kind = k % 4
        p = float(rng.choice([0.0, 0.0007, 0.01, 0.2, 0.9, 1.0]))
        if kind == 3:
            shape = (int(rng.integers(1, 70)), int(rng.integers(1, 130)), int(rng.integers(1, 300)))
        elif kind == 2:
            shape = (int(rng.integers(1, 200)), int(rng.integers(2049, 9000)))
        else:
            shape = (int(rng.integers(1, 700)), int(rng.integers(1, 2049)))
        specs.append((shape, p, int(rng.integers(2)), bool(rng.integers(2)), bool(rng.integers(2))))
    return specs


def _run_mixed(torch, edt, plan, specs, seed):
    jobs = []
    for k, (shape, p, mode, want_D, want_dist) in enumerate(specs):
        m_np = inputs.bernoulli_mask(shape, p, seed * 1000 + k)
        m = torch.from_numpy(m_np).cuda()
        D = torch.full(shape, -5, dtype=torch.int32, device="cuda") if want_D else None
        F = torch.full(shape, -5, dtype=torch.int32, device="cuda")
        dist = torch.full(shape, -5.0, dtype=torch.float32, device="cuda") if want_dist else None
        jobs.append((m, mode, D, F, dist))
    plan.run(jobs)
    torch.cuda.synchronize()
    return jobs


def test_mixed_2d_3d_wide_batch_matches_oracle():
    """One replay with narrow 2-D, wide 2-D (beyond 2048 columns) and 3-D jobs
    of uneven sizes, both modes, optional outputs: every job against the
    oracle and bit-identical to a plain call."""
    import torch
    from paper_2106_03503_gb300 import edt
    rng = np.random.default_rng(3)
    specs = _mixed_specs(rng, 40)
    plan = edt.Plan(len(specs), 1 << 20)     # small scratch up front: the plan grows
    for rep in range(2):
        jobs = _run_mixed(torch, edt, plan, specs, 40 + rep)
        refs = [edt.feature(m, mode, want_dist=True) for (m, mode, _, _, _) in jobs]
        _check(jobs, refs, torch)
    plan.close()


def test_batch_autotune_candidates_give_the_same_bits(tmp_path):
    """edt_autotune_batch picks a geometry per shape class; every candidate
    (forced through a tuning file) gives the same D, F bits as a plain call."""
    import torch
    from paper_2106_03503_gb300 import edt
    rng = np.random.default_rng(5)
    specs = [((int(rng.integers(100, 600)), int(rng.integers(100, 1500))), 0.01, 0, True, False)
             for _ in range(6)]
    specs += [((int(rng.integers(20, 60)), int(rng.integers(40, 200)), int(rng.integers(40, 260))), 0.0, 0, True,
               False) for _ in range(4)]
    plan = edt.Plan(len(specs), 1 << 22)
    jobs = _run_mixed(torch, edt, plan, specs, 60)
    for k, (m, mode, D, F, dist) in enumerate(jobs):   # smoothed-noise volumes for the 3-D jobs
        if m.dim() == 3:
            jobs[k] = (torch.from_numpy(inputs.smoothed_noise_volume(tuple(m.shape), 3.0, 70 + k)).cuda(), mode, D, F,
                       dist)
    refs = [edt.feature(m, mode) for (m, mode, _, _, _) in jobs]
    plan.autotune(jobs)
    torch.cuda.synchronize()
    for (m, mode, D, F, _), (Dr, Fr) in zip(jobs, refs):
        assert torch.equal(D, Dr) and torch.equal(F, Fr)
    for lgmin, pos in ((6, 32), (7, 128), (8, 64)):
        path = tmp_path / f"t{lgmin}.txt"
        lines = []
        for (m, _, _, _, _) in jobs:
            cls = [int(np.ceil(np.log2(v))) if v > 1 else 0 for v in m.shape] + [0] * (3 - m.dim())
            lines.append(f"b {m.dim()} {cls[0]} {cls[1]} {cls[2]} {lgmin if m.dim() == 2 else 0} "
                         f"{pos if m.dim() == 3 else 0} {pos if m.dim() == 3 else 0}")
        path.write_text("\n".join(lines) + "\n")
        edt.tune_load(str(path))
        for (m, _, _, _, _) in jobs:
            got = edt.batch_tune_get(tuple(m.shape))
            if m.dim() == 2:
                assert got["rows2d_lgmin"] == lgmin
            else:
                assert got["y_pos"] == pos and got["x_pos"] == pos
        for (m, mode, D, F, dist) in jobs:
            D.fill_(-9)
            F.fill_(-9)
        plan.run(jobs)
        torch.cuda.synchronize()
        for (m, mode, D, F, _), (Dr, Fr) in zip(jobs, refs):
            assert torch.equal(D, Dr) and torch.equal(F, Fr), (lgmin, pos, tuple(m.shape))
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
        Do, Fo = oracle.edt(masks_np[k], 0)
        D, F = outs[k]
        D, F = D.cpu().numpy(), F.cpu().numpy()
        assert np.array_equal(D, Do), k
        assert feature_valid_fast(masks_np[k], 0, D, F) is None
        assert np.array_equal(F, Fo), k


def test_batch_patch_search_clamp_and_ragged_patches():
    """The batch's row search on 4 x 8 patches keeps vertical offsets as int8,
    clamped at +-127: a single source in a narrow image puts offsets of 126
    (kept exact: with the source in row 1, the band of rows 96..127 settles),
    127 and 128 and beyond (a best of 127^2 or more: the band falls back to
    the hull) in the same columns; heights that are not a multiple of 4 and widths
    that are not a multiple of 8 leave partial patches; widths 1024 and 1025
    sit on both sides of the direct search's limit."""
    import torch
    from paper_2106_03503_gb300 import edt
    masks = []
    for (H, W, i, j) in [(300, 20, 0, 5), (300, 20, 1, 5), (300, 20, 299, 19), (260, 70, 130, 35), (129, 9, 0, 0)]:
        m = np.zeros((H, W), np.uint8)
        m[i, j] = 1
        masks.append(m)
    rng = np.random.default_rng(31)
    for H in (1, 2, 3, 5, 6, 7, 33, 35):
        for W in (1, 7, 9, 15, 17, 33):
            masks.append(inputs.bernoulli_mask((H, W), float(rng.choice([0.05, 0.3])), 3100 + 37 * H + W))
    for W in (1016, 1023, 1024, 1025):
        masks.append(inputs.bernoulli_mask((70, W), 0.002, 3300 + W))
    jobs, refs = [], []
    for k, m_np in enumerate(masks):
        m = torch.from_numpy(m_np).cuda()
        mode = k % 2 if k >= 5 else 0
        D = torch.full(m.shape, -5, dtype=torch.int32, device="cuda")
        F = torch.full(m.shape, -5, dtype=torch.int32, device="cuda")
        dist = torch.full(m.shape, -5.0, dtype=torch.float32, device="cuda")
        jobs.append((m, mode, D, F, dist))
        refs.append(edt.feature(m, mode, want_dist=True))
    plan = edt.Plan(len(jobs), sum(m.size for m in masks))
    plan.run(jobs)
    _check(jobs, refs, torch)
    plan.close()
