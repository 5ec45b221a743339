"""Serving loop (hm_server_*): requests that run concurrently on the GPU must
each get exactly the result they get alone (tolerance 0: the matching is a
unique integer set), admission must respect the device-memory budget, and
requests must actually overlap when slots and memory allow."""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2602_22976_gb300 as hmlib

pytestmark = pytest.mark.gpu

MiB = 1 << 20


@pytest.fixture(scope="module", autouse=True)
def _built():
    hmlib.build()
    assert torch.cuda.is_available(), "needs a CUDA device"
    hmlib.lib()


def footprint(h):  # admission estimate documented in include/hm.h
    return 36 * h.kappa + 64 * h.m + 72 * h.n + 16 * MiB


def requests(seed, count):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        kappa = int(np.exp(rng.uniform(np.log(1e3), np.log(3e5))))
        h = synth.serve_request(kappa, seed=seed * 1000 + i)
        if i % 4 == 3:
            h.weights = None  # unweighted requests in the mix
        out.append(h)
    return out


def test_mix_equals_alone():
    hs = requests(1, 16)
    alone = [hmlib.solve_host(h) for h in hs]
    with hmlib.Server(slots=4) as srv:
        tickets = [srv.submit(h) for h in hs]
        got = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(hs) and st["queued"] == 0 and st["inflight"] == 0
    for h, a, (r, lat) in zip(hs, alone, got):
        o = oracle.match(h)
        assert np.array_equal(r.edges, a.edges) and np.array_equal(r.edges, o.edges)
        assert r.rounds == a.rounds == o.rounds
        assert r.weight == a.weight == oracle.weight(h, o.in_matching)
        assert lat > 0


def test_admission_respects_memory_budget():
    hs = requests(2, 10)
    budget = max(footprint(h) for h in hs) + footprint(min(hs, key=lambda x: x.kappa)) // 2
    with hmlib.Server(slots=6, hbm_budget_bytes=budget) as srv:
        tickets = [srv.submit(h) for h in hs]
        got = [srv.wait(t)[0] for t in tickets]
        st = srv.stats()
    assert st["budget_bytes"] == budget
    assert 0 < st["peak_reserved_bytes"] <= budget
    for h, r in zip(hs, got):
        o = oracle.match(h)
        assert np.array_equal(r.edges, o.edges) and r.rounds == o.rounds


def test_requests_overlap_when_allowed():
    hs = [synth.serve_request(2_000_000, seed=50 + i) for i in range(8)]
    with hmlib.Server(slots=4) as srv:
        tickets = [srv.submit(h) for h in hs]
        res = [srv.wait(t)[0] for t in tickets]
        st = srv.stats()
    assert st["peak_inflight"] >= 2
    for h, r in zip(hs[:2], res[:2]):
        o = oracle.match(h)
        assert np.array_equal(r.edges, o.edges)


def test_refusals():
    h = synth.serve_request(100_000, seed=7)
    with hmlib.Server(slots=1, hbm_budget_bytes=footprint(h) - 1) as srv:
        with pytest.raises(hmlib.HMError) as ei:
            srv.submit(h)
        assert ei.value.status == hmlib.HM_ENOMEM
        assert hmlib.lib().hm_server_wait(srv.handle, 12345, None, None, None, None, None) == hmlib.HM_EINVAL
    L = hmlib.lib()
    import ctypes
    s = ctypes.c_void_p()
    assert L.hm_server_create(ctypes.byref(s), 0, 0) == hmlib.HM_EINVAL


def test_queued_requests_are_grouped():
    """With one slot and a full queue, compatible requests queued behind the
    head run as one batch; each still gets its solo result, and unweighted
    requests group only with the same seed."""
    rng = np.random.default_rng(9)
    hs = []
    for i in range(24):
        h = synth.serve_request(int(np.exp(rng.uniform(np.log(1e3), np.log(2e5)))), seed=900 + i)
        if i >= 16:
            h.weights = None
            h.seed = 77 if i < 20 else 78  # two seeds: two unweighted groups
        hs.append(h)
    with hmlib.Server(slots=1) as srv:
        tickets = [srv.submit(h) for h in hs]
        got = [srv.wait(t)[0] for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(hs)
    assert st["peak_group"] >= 2 and st["groups"] < len(hs)
    for h, r in zip(hs, got):
        o = oracle.match(h)
        assert np.array_equal(r.edges, o.edges) and r.rounds == o.rounds
        assert r.weight == oracle.weight(h, o.in_matching)


def test_invalid_request_inside_a_group():
    """A request with a pin outside [0, n) fails on the device; its group then
    runs request by request, so only that request reports HM_EINVAL."""
    hs = [synth.serve_request(20_000, seed=300 + i) for i in range(6)]
    bad = hs[3]
    bad.pins = bad.pins.copy()
    bad.pins[5] = bad.n + 7
    with hmlib.Server(slots=1) as srv:
        tickets = [srv.submit(h) for h in hs]
        got = [srv.wait(t, allow=(hmlib.HM_OK, hmlib.HM_EINVAL))[0] for t in tickets]
    for i, (h, r) in enumerate(zip(hs, got)):
        if i == 3:
            assert r.status == hmlib.HM_EINVAL
        else:
            o = oracle.match(h)
            assert r.status == hmlib.HM_OK and np.array_equal(r.edges, o.edges)


def test_full_size_requests_in_a_mix():
    """Requests drawn from the serving workload's distribution (kappa
    log-uniform in [1e3, 1e7], |e| ~ Zipf(2) on [2, 256]) submitted at once
    to the server the bench uses (8 slots): every result equals the CPU
    oracle's."""
    rng = np.random.default_rng(21)
    kap = np.exp(rng.uniform(np.log(1e3), np.log(1e7), size=24)).astype(np.int64)
    kap[0] = 10_000_000  # the largest size of the distribution
    hs = [synth.serve_request(int(k), seed=2100 + i) for i, k in enumerate(kap)]
    with hmlib.Server(slots=8) as srv:
        tickets = [srv.submit(h) for h in hs]
        got = [srv.wait(t)[0] for t in tickets]
    for h, r in zip(hs, got):
        o = oracle.match(h)
        assert np.array_equal(r.edges, o.edges) and r.rounds == o.rounds
        assert r.weight == oracle.weight(h, o.in_matching)
