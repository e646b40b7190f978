"""Serving (edt_serve_*): each result equals the oracle's (D bit-exact, F a
nearest source, dist the correctly rounded square root), and is the same
served alone, served in a mix of concurrent 2-D / 3-D requests of mixed sizes
and computed by a plain edt_feature call; budget refusal and bad requests fail
at submission."""
import time

import numpy as np
import pytest

import oracle
from gpu_check import feature_valid_fast
from paper_2106_03503_gb300 import inputs

pytestmark = pytest.mark.gpu


def _wait(srv, t, timeout=120.0):
    t0 = time.time()
    while True:
        r = srv.poll(t)
        if r is not None:
            return r
        if time.time() - t0 > timeout:
            raise TimeoutError(f"ticket {t} not done after {timeout} s")
        time.sleep(0.0005)


def _specs():
    rng = np.random.default_rng(5)
    specs = []
    for k in range(40):
        if k % 5 == 4:
            s = int(rng.integers(16, 90))
            specs.append(("3d", (s, s, s), 4.0, 500 + k))
        else:
            s = int(rng.choice([40, 128, 300, 1000, 2100, 3000]))
            specs.append(("2d", (s, s), float(np.exp(rng.uniform(np.log(0.001), np.log(0.1)))), 500 + k))
    return specs


def _mask(spec):
    kind, shape, par, seed = spec
    if kind == "2d":
        return inputs.bernoulli_mask(shape, par, seed)
    return inputs.smoothed_noise_volume(shape, par, seed)


def test_alone_equals_in_the_mix_equals_plain():
    import torch
    from paper_2106_03503_gb300 import edt
    specs = _specs()
    masks = [torch.from_numpy(_mask(s)).pin_memory() for s in specs]
    plain = []
    for k, m in enumerate(masks):
        D, F, d = edt.feature(m.cuda(), k % 2, want_dist=True)
        plain.append((D.cpu(), F.cpu(), d.cpu()))
    srv = edt.Server(8 << 30, n_streams=3)
    # alone: one request at a time
    alone = []
    for k, m in enumerate(masks):
        t = srv.submit(m, k % 2, want_dist=True)
        lat, out = _wait(srv, t)
        assert lat > 0
        alone.append(out)
    # in the mix: all requests in flight together
    tickets = [srv.submit(m, k % 2, want_dist=True) for k, m in enumerate(masks)]
    mix = [None] * len(tickets)
    pending = set(range(len(tickets)))
    t0 = time.time()
    while pending:
        for k in list(pending):
            r = srv.poll(tickets[k])
            if r is not None:
                mix[k] = r[1]
                pending.discard(k)
        assert time.time() - t0 < 300
        time.sleep(0.0005)
    srv.close()
    for k in range(len(masks)):
        # the oracle decides: every served D bit-exact, F a nearest source,
        # dist the correctly rounded square root
        m_np = masks[k].numpy()
        Do, Fo = oracle.edt(m_np, k % 2)
        for D, F, d in (alone[k], mix[k]):
            D, F, d = D.numpy(), F.numpy(), d.numpy()
            assert np.array_equal(D, Do), k
            msg = feature_valid_fast(m_np, k % 2, D, F)
            assert msg is None, (k, msg)
            assert np.array_equal(F, Fo), (k, "F differs from the oracle's")
            assert np.array_equal(d.view(np.uint32), oracle.sqrt_f32(Do).view(np.uint32)), k
        # and the same bits alone, in the mix and from a plain call
        for a, b, c in zip(plain[k], alone[k], mix[k]):
            assert torch.equal(a.view(torch.int32), b.view(torch.int32)), k
            assert torch.equal(a.view(torch.int32), c.view(torch.int32)), k


def test_budget_and_bad_requests():
    import torch
    from paper_2106_03503_gb300 import edt
    srv = edt.Server(1 << 30, n_streams=1)
    big = torch.zeros((16000, 16000), dtype=torch.uint8)
    with pytest.raises(edt.EdtError) as e:
        srv.submit(big, 0)
    assert e.value.status == 6  # EDT_ERR_BUDGET
    bad = torch.zeros((3, 40000), dtype=torch.uint8)
    with pytest.raises(edt.EdtError) as e:
        srv.submit(bad, 0)
    assert e.value.status == 2
    with pytest.raises(edt.EdtError) as e:
        srv.submit(torch.zeros((4, 4), dtype=torch.uint8), 7)
    assert e.value.status == 1
    ok = srv.submit(torch.ones((64, 64), dtype=torch.uint8), 1)
    lat, (D, F, dist) = _wait(srv, ok)
    assert torch.all(D == 2**31 - 1) and torch.all(F == -1)
    srv.close()
    # a budget beyond the device's free memory is refused before any allocation
    free, _ = torch.cuda.mem_get_info()
    with pytest.raises(edt.EdtError) as e:
        edt.Server(free + (1 << 30), n_streams=1)
    assert e.value.status == 6
