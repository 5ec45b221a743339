"""GPU path vs the CPU oracle, through the C ABI (libhm.so).

The order on edges is strict, so the matching is unique: the matched edge
set, the round count, the per-round winner counts and the matching weight
(the exact sum rounded once to float64, on both sides) must be identical. The
per-vertex state after a capped run (T[v] of round r, or matched) must
equal the oracle's state after r rounds.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from cursor_work import active_sets as _active_sets, entries_ahead_of_the_match as _entries_ahead_of_the_match
import paper_2602_22976_gb300 as hmlib
from conftest import golden_cases, golden_hypergraph

pytestmark = pytest.mark.gpu

OK, EINVAL, ETIMEOUT = hmlib.HM_OK, hmlib.HM_EINVAL, hmlib.HM_ETIMEOUT
WIN = hmlib.STAT_COLUMNS.index("winners")


@pytest.fixture(scope="session", autouse=True)
def _built():
    hmlib.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    hmlib.lib()


def run_gpu(h, cap=None):
    with hmlib.Matcher.from_hypergraph(h) as mt:
        if cap is not None:
            mt.set_round_cap(cap)
        mt.match()
        res = mt.result(allow=(OK, ETIMEOUT))
        stats = mt.round_stats()
        vs = mt.vertex_state()
    return res, stats, vs


def assert_parity(h, res=None, stats=None, o=None):
    if res is None:
        res, stats, _ = run_gpu(h)
    o = o or oracle.match(h)
    assert res.status == OK
    assert res.rounds == o.rounds
    assert np.array_equal(res.edges, o.edges)
    assert res.count == int(o.in_matching.sum())
    assert stats[:o.rounds, WIN].tolist() == o.round_stats[:, 2].tolist()
    assert res.weight == oracle.weight(h, o.in_matching)
    return o


@pytest.mark.parametrize("case", golden_cases(), ids=lambda c: c["name"])
def test_golden(case):
    h = golden_hypergraph(case)
    res, stats, _ = run_gpu(h)
    assert res.edges.tolist() == case["matching"]
    assert res.rounds == case["rounds"]
    assert_parity(h, res, stats)


def test_small_config():
    """n=10,000, m=20,000, |e| ~ U{2..8}, weights in (0,1], seed 1."""
    assert_parity(synth.small())


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_powerlaw_scaled(seed):
    """Power-law shape (Zipf(2) sizes on [2,1024], gamma=2.2 degrees) at 1/10 scale."""
    assert_parity(synth.large(seed=seed, n=1_000_000, m=2_000_000))


@pytest.mark.parametrize("n,deg", [(30_000, 16.0), (50_000, 4.0), (20_000, 40.0)])
def test_graph_rgg(n, deg):
    """Graphs (d = 2): random geometric graphs of the DIMACS rgg class."""
    assert_parity(synth.rgg(seed=3, n=n, avg_degree=deg))


def test_unweighted_scaled():
    assert_parity(synth.unweighted(seed=1, n=400_000, m=800_000))
    assert_parity(synth.unweighted(seed=7, n=10_000, m=20_000))


def test_ties_everywhere():
    """Only two weight values: the id tie-break decides most argmaxes."""
    h = synth.small(seed=4, n=3000, m=12_000)
    h.weights = np.where(h.weights > 0.5, 1.0, 0.5).astype(np.float32)
    assert_parity(h)


def test_degenerate_inputs():
    assert_parity(synth.from_edges(5, [], []))                      # no edges
    assert_parity(synth.from_edges(1, [[0]], [1.0]))                # one vertex, one edge
    assert_parity(synth.from_edges(100, [[3], [3], [7]], [0.5, 0.5, 0.25]))  # size-1 edges, tie
    assert_parity(synth.from_edges(50, [[0, 49]], [2.0]))           # mostly isolated vertices


def test_big_edges_and_hubs():
    """Edge sizes across 32/256/2048/4096 and a hub whose kill range is
    split into several chunks."""
    rng = np.random.default_rng(0)
    n = 20_000
    edges, w = [], []
    for k in (31, 32, 33, 255, 256, 257, 2047, 2048, 2049, 4095, 4096, 5000):
        edges.append(sorted(rng.choice(n, size=k, replace=False).tolist()))
        w.append(float(rng.integers(1, 1 << 24)) / (1 << 24))
    for i in range(9000):  # hub: vertex 0 in 9000 small edges
        e = [0] + rng.choice(np.arange(1, n), size=int(rng.integers(1, 4)), replace=False).tolist()
        edges.append(sorted(e))
        w.append(float(rng.integers(1, 1 << 24)) / (1 << 24))
    for i in range(20_000):
        edges.append(sorted(rng.choice(n, size=int(rng.integers(2, 6)), replace=False).tolist()))
        w.append(float(rng.integers(1, 1 << 24)) / (1 << 24))
    h = synth.from_edges(n, edges, w)
    assert_parity(h)
    # make the hub's best edge the global best so it is matched in round 1
    w2 = list(w)
    w2[12] = 1.0
    assert_parity(synth.from_edges(n, edges, w2))


def test_long_path_many_rounds():
    m = 3001
    h = synth.from_edges(m + 1, [[i, i + 1] for i in range(m)], [(i + 1) / 4096 for i in range(m)])
    o = assert_parity(h)
    assert o.rounds == math.ceil(m / 2)


@pytest.mark.parametrize("cap", [1, 2, 3])
def test_vertex_state_after_capped_rounds(cap):
    """a1 parity: T[v] after round r equals the oracle's argmax of round r."""
    for h in (synth.small(seed=5, n=5000, m=15_000), synth.large(seed=6, n=100_000, m=200_000)):
        res, stats, vs = run_gpu(h, cap=cap)
        o = oracle.match(h, max_rounds=cap)
        assert res.status == ETIMEOUT
        assert res.rounds == cap
        assert np.array_equal(vs, oracle.vertex_state(o))
        assert np.array_equal(res.edges, o.edges)


def test_round_cap_timeout_on_path():
    h = synth.from_edges(10, [[i, i + 1] for i in range(9)], [(i + 1) / 16 for i in range(9)])
    res, _, _ = run_gpu(h, cap=1)
    assert res.status == ETIMEOUT and res.rounds == 1 and res.edges.tolist() == [8]
    with hmlib.Matcher.from_hypergraph(h) as mt:
        mt.set_round_cap(1)
        mt.match()
        with pytest.raises(hmlib.HMError) as ei:
            mt.result()
        assert ei.value.status == ETIMEOUT


def test_repeat_profile_and_device_result():
    h = synth.large(seed=2, n=200_000, m=400_000)
    o = oracle.match(h)
    with hmlib.Matcher.from_hypergraph(h) as mt:
        for _ in range(3):
            mt.match()
            res = mt.result()
            assert np.array_equal(res.edges, o.edges) and res.rounds == o.rounds
        prof = mt.profile()
        res = mt.result()
        assert np.array_equal(res.edges, o.edges) and res.rounds == o.rounds
        assert prof["argmax"][1] == prof["win"][1] == prof["kill"][1] >= o.rounds
        assert prof["round_end"][1] == 0  # part of the kill kernel
        mask = torch.zeros(h.m, dtype=torch.uint8, device="cuda")
        mt.result_device(mask)
        torch.cuda.synchronize()
        assert np.array_equal(mask.cpu().numpy(), o.in_matching)
        s = torch.cuda.Stream()
        mt.match(stream=s)
        res = mt.result()
        assert np.array_equal(res.edges, o.edges)


def test_solve_host_matches_handle_path():
    h = synth.small(seed=8)
    o = oracle.match(h)
    res = hmlib.solve_host(h)
    assert np.array_equal(res.edges, o.edges) and res.rounds == o.rounds
    assert res.weight == oracle.weight(h, o.in_matching)
    hu = synth.unweighted(seed=3, n=10_000, m=20_000)
    ou = oracle.match(hu)
    ru = hmlib.solve_host(hu)
    assert np.array_equal(ru.edges, ou.edges) and ru.rounds == ou.rounds


def test_solve_host_graph_and_chunks():
    """hm_solve_host on both sides of its 4M-pin split: above it the pins
    cross in chunks beside the edge phase (a graph gathers its pairs once
    every chunk is in), below it they follow the offsets on one stream."""
    big = synth.large(seed=6, n=400_000, m=600_000)
    big_graph = synth.rgg(seed=8, n=600_000)
    assert big.kappa >= 1 << 22 and big_graph.kappa >= 1 << 22
    for h in (big, big_graph, synth.rgg(seed=8, n=60_000), synth.small(seed=9, n=300, m=500),
              synth.from_edges(3, [[0, 1]], [0.5], seed=1)):
        o = oracle.match(h)
        r = hmlib.solve_host(h)
        assert np.array_equal(r.edges, o.edges) and r.rounds == o.rounds
        assert r.weight == oracle.weight(h, o.in_matching)


def _small_cases():
    rng = np.random.default_rng(11)
    hub = [[0, int(v)] for v in rng.permutation(np.arange(1, 3000))[:2000]]  # a hub of degree 2000
    wide = [list(range(1500))] + [[int(a), int(a) + 1] for a in range(1500, 1600)]  # one 1500-pin edge
    return [synth.small(seed=9, n=300, m=500), synth.small(seed=3),
            synth.serve_request(1000, seed=1), synth.serve_request(30_000, seed=2),
            synth.serve_request(120_000, seed=3), synth.unweighted(seed=4, n=5000, m=10_000),
            synth.rgg(seed=5, n=6000), synth.from_edges(3, [[0, 1]], [0.5], seed=1),
            synth.from_edges(3000, hub, list(rng.random(len(hub), dtype=np.float32) + 0.01), seed=2),
            synth.from_edges(1700, wide, None, seed=3)]


@pytest.mark.parametrize("i", range(10))
def test_solve_host_small_inputs(i):
    """hm_solve_host below 2^17 pins runs the whole matching in one thread
    block (edges of at most 256 pins; the 1500-pin edge of the last case
    takes the handle path): the same matching, round count and exact weight
    as the oracle."""
    h = _small_cases()[i]
    assert h.kappa <= 1 << 17
    o = oracle.match(h)
    r = hmlib.solve_host(h)
    assert np.array_equal(r.edges, o.edges) and r.rounds == o.rounds
    assert r.weight == oracle.weight(h, o.in_matching)


def test_solve_host_small_rejects_bad_input():
    """The one-block path rejects what hm_create rejects, with the same
    messages: an empty edge, a pin outside [0, n), a weight that is not
    finite and > 0, and a vertex twice in one edge (short edges, and edges
    longer than 16 pins, which a warp checks); the next call works."""
    h = synth.serve_request(20_000, seed=4)
    sizes = np.diff(h.eoff)
    long_e = int(np.flatnonzero(sizes > 40)[0])
    short_e = int(np.flatnonzero(sizes == 3)[0])

    def bad(mutate, word):
        x = synth.Hypergraph(h.n, h.m, h.eoff.copy(), h.pins.copy(), h.weights.copy(), h.seed)
        mutate(x)
        r = hmlib.solve_host(x, allow=(OK, EINVAL))
        assert r.status == EINVAL and word in hmlib.last_error(), hmlib.last_error()

    bad(lambda x: x.weights.__setitem__(17, -0.0), "weight of edge 17")
    bad(lambda x: x.pins.__setitem__(123, h.n), "pin at position 123")
    bad(lambda x: x.pins.__setitem__(int(h.eoff[short_e]) + 2, x.pins[int(h.eoff[short_e])]),
        f"duplicate pin: a vertex appears twice in one edge (edge {short_e})")
    bad(lambda x: x.pins.__setitem__(int(h.eoff[long_e + 1]) - 1, x.pins[int(h.eoff[long_e]) + 5]),
        f"(edge {long_e})")

    def empty_edge(x):
        x.eoff[5] = x.eoff[4]  # edge 4 empty, edge 5 longer
    bad(empty_edge, "eoff is not strictly increasing at edge 4")
    o = oracle.match(h)
    r = hmlib.solve_host(h)
    assert np.array_equal(r.edges, o.edges) and r.rounds == o.rounds


@pytest.mark.parametrize("n,m", [(50_000, 100_000), (400_000, 600_000)])
def test_solve_host_rejects_bad_input(n, m):
    """A bad weight fails before the pins are used, a bad pin fails when they
    arrive (in its chunk above 4M pins, in the validation pass below); both
    report HM_EINVAL, and the next call works."""
    h = synth.large(seed=6, n=n, m=m)
    bad_w = synth.Hypergraph(h.n, h.m, h.eoff, h.pins, h.weights.copy(), h.seed)
    bad_w.weights[123] = -1.0
    r = hmlib.solve_host(bad_w, allow=(OK, EINVAL))
    assert r.status == EINVAL and "weight" in hmlib.last_error()
    bad_p = synth.Hypergraph(h.n, h.m, h.eoff, h.pins.copy(), h.weights, h.seed)
    bad_p.pins[h.kappa // 2] = h.n
    r = hmlib.solve_host(bad_p, allow=(OK, EINVAL))
    assert r.status == EINVAL and "pin" in hmlib.last_error()
    o = oracle.match(h)
    r = hmlib.solve_host(h)
    assert np.array_equal(r.edges, o.edges) and r.rounds == o.rounds


def test_random_access_probe():
    """The benchmark's probe library (not part of libhm.so) measures positive
    rates and refuses a too-small array."""
    import bench
    r = bench.probe_random_access(1 << 20, 2_000_000)
    assert set(r) == set(bench.PROBES) and all(v > 0 for v in r.values())
    with pytest.raises(RuntimeError, match="array_bytes"):
        bench.probe_random_access(10, 1)


def test_busy_while_a_match_runs_on_another_stream():
    """HM_EBUSY: a handle refuses a match, a profiled match and an autotune
    on a second stream while its last match is still queued or running on
    the first. The first stream is kept busy by ordinary memory fills queued
    ahead of the match (no kernel waits on anything), so the match cannot
    have finished when the second call is made a few microseconds later."""
    h = synth.large(seed=2, n=500_000, m=1_000_000)
    o = oracle.match(h)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    L = hmlib.lib()
    with hmlib.Matcher.from_hypergraph(h) as mt:
        mt.match(s1)  # builds the CUDA graph
        torch.cuda.synchronize()
        buf = torch.empty(1 << 30, dtype=torch.uint8, device="cuda")
        with torch.cuda.stream(s1):
            for _ in range(100):  # about 100 x 0.15 ms of fills ahead of the match
                buf.fill_(1)
        mt.match(s1)
        assert L.hm_match(mt.handle, s2.cuda_stream) == hmlib.HM_EBUSY
        assert "another stream" in hmlib.last_error()
        ms, launches = np.zeros(5), np.zeros(5, dtype=np.int64)
        assert L.hm_profile_match(mt.handle, s2.cuda_stream, ms.ctypes.data, launches.ctypes.data,
                                  None, 0) == hmlib.HM_EBUSY
        cfg, t = np.zeros(4, dtype=np.int32), ctypes.c_double(0)
        assert L.hm_autotune(mt.handle, s2.cuda_stream, cfg.ctypes.data, ctypes.byref(t)) == hmlib.HM_EBUSY
        r = mt.result()  # waits for the match on s1
        assert r.rounds == o.rounds and np.array_equal(r.edges, o.edges)
        mt.match(s2)  # nothing in flight any more: the second stream is accepted
        r = mt.result()
        assert r.rounds == o.rounds and np.array_equal(r.edges, o.edges)
        del buf


# ------------------------------------------------------------------ errors

def _create(n, m, eoff, pins, w, flags=0):
    L = hmlib.lib()
    h = ctypes.c_void_p()
    st = L.hm_create(ctypes.byref(h), n, m, eoff, pins, w, 1, flags, None)
    if st == OK:
        L.hm_destroy(h)
    return st, hmlib.last_error()


def _dev(a, dt):
    return torch.tensor(a, dtype=dt, device="cuda")


def test_invalid_inputs_rejected():
    i64, i32, f32 = torch.int64, torch.int32, torch.float32
    eoff = _dev([0, 2, 4], i64)
    pins = _dev([0, 1, 1, 2], i32)
    w = _dev([0.5, 0.25], f32)
    assert _create(3, 2, eoff.data_ptr(), pins.data_ptr(), w.data_ptr())[0] == OK
    cases = {
        "eoff[0]": (_dev([1, 2, 4], i64), pins, w, 0),
        "empty edge": (_dev([0, 2, 2, 4], i64), _dev([0, 1, 1, 2], i32), _dev([0.5, 0.5, 0.5], f32), 0),
        "decreasing": (_dev([0, 3, 2, 4], i64), _dev([0, 1, 2, 2], i32), _dev([0.5, 0.5, 0.5], f32), 0),
        "pin >= n": (eoff, _dev([0, 1, 1, 3], i32), w, 0),
        "pin < 0": (eoff, _dev([0, -1, 1, 2], i32), w, 0),
        "zero weight": (eoff, pins, _dev([0.0, 0.5], f32), 0),
        "-0.0 weight": (eoff, pins, _dev([-0.0, 0.5], f32), 0),
        "negative weight": (eoff, pins, _dev([0.5, -1.0], f32), 0),
        "inf weight": (eoff, pins, _dev([float("inf"), 0.5], f32), 0),
        "nan weight": (eoff, pins, _dev([float("nan"), 0.5], f32), 0),
        "duplicate pin": (eoff, _dev([0, 0, 1, 2], i32), w, 0),
    }
    for name, (e, p, ww, fl) in cases.items():
        m = e.numel() - 1
        st, msg = _create(3, m, e.data_ptr(), p.data_ptr(), ww.data_ptr(), fl)
        assert st == EINVAL, (name, st, msg)
        assert msg, name
    # unweighted ignores (invalid) weights
    assert _create(3, 2, eoff.data_ptr(), pins.data_ptr(), _dev([0.0, -1.0], f32).data_ptr(),
                   hmlib.HM_UNWEIGHTED)[0] == OK
    # NULL weights without HM_UNWEIGHTED; host memory instead of device memory
    assert _create(3, 2, eoff.data_ptr(), pins.data_ptr(), None)[0] == EINVAL
    host = np.array([0, 2, 4], dtype=np.int64)
    st, msg = _create(3, 2, host.ctypes.data, pins.data_ptr(), w.data_ptr())
    assert st == EINVAL and "device memory" in msg
    torch.cuda.synchronize()


def test_no_match_yet_and_null_handle():
    h = synth.small(seed=1, n=100, m=200)
    with hmlib.Matcher.from_hypergraph(h) as mt:
        with pytest.raises(hmlib.HMError):
            mt.result()
    assert hmlib.lib().hm_match(None, None) == EINVAL


# ------------------------------------------------------------------ full size

@pytest.mark.slow
def test_full_size_powerlaw():
    """n=10M, m=20M, Zipf(2) sizes on [2,1024], gamma=2.2 degrees (kappa ~ 2.02e8)."""
    h = synth.large()
    assert_parity(h)


@pytest.mark.slow
def test_full_size_unweighted():
    """n=4M, m=8M, |e| ~ U{2..8}, seeded hash priority."""
    assert_parity(synth.unweighted())


def test_each_list_entry_touched_once():
    """The paper compacts the hypergraph after every round (Sec. 4.3) so that
    the whole run costs O(kappa) work. The cursor design reaches that bound
    without moving data: every entry of every vertex list is either skipped
    once by its vertex's cursor (the argmax step) or deactivated once by the
    kill step, so over the whole run the two counters add up to kappa
    exactly."""
    adv = hmlib.STAT_COLUMNS.index("advance")
    kills = hmlib.STAT_COLUMNS.index("kills")
    cases = [synth.large(seed=5, n=300_000, m=600_000), synth.small(seed=3),
             synth.unweighted(seed=2, n=100_000, m=200_000)]
    for h in cases:
        res, stats, _ = run_gpu(h)
        assert res.status == OK
        assert int(stats[:, adv].sum() + stats[:, kills].sum()) == h.kappa


def test_graph_cursors_pass_each_entry_once():
    """Graphs run without a kill step (an edge is live while neither endpoint
    is matched): the kill counter stays 0, and the entries the cursors skip
    are exactly those ahead of each vertex's matching edge."""
    adv = hmlib.STAT_COLUMNS.index("advance")
    kills = hmlib.STAT_COLUMNS.index("kills")
    cases = [synth.rgg(seed=5, n=80_000), synth.rgg(seed=6, n=20_000, avg_degree=40),
             synth.from_edges(5, [[0, 1], [1, 2], [2, 3], [3, 4]], None, seed=1),
             synth.from_edges(6, [[0, 1], [0, 2], [0, 3], [4, 5]], [1.0, 3.0, 2.0, 1.0], seed=1)]
    for h in cases:
        res, stats, _ = run_gpu(h)
        o = oracle.match(h)
        assert res.status == OK and np.array_equal(res.edges, o.edges) and res.rounds == o.rounds
        assert not stats[:, kills].any()
        assert int(stats[:, adv].sum()) == _entries_ahead_of_the_match(h, o)


def test_active_vertices_and_their_degrees_per_round():
    """The count of the vertices kept for each round (HM_STAT_NEXT) and the
    replay's count of their degrees (HM_STAT_DEG) equal, round by round, the
    active vertex sets of the oracle's run and their degree sums, in the
    fixed order and in re-randomised rounds; the replay's live edges and
    live pins at the start of every round (HM_STAT_LEDGES, HM_STAT_LPINS)
    equal the oracle's. A plain match leaves these three columns at 0, and in
    re-randomised rounds it counts the kept vertices of round 1 only (later
    rounds are edge-driven and leave the vertex counts to the replay)."""
    nxt = hmlib.STAT_COLUMNS.index("next")
    dg = hmlib.STAT_COLUMNS.index("deg")
    le = hmlib.STAT_COLUMNS.index("ledges")
    lp = hmlib.STAT_COLUMNS.index("lpins")
    cases = [synth.large(seed=5, n=300_000, m=600_000), synth.small(seed=3),
             synth.unweighted(seed=2, n=100_000, m=200_000), synth.rgg(seed=4, n=50_000),
             synth.from_edges(7, [[0, 1], [1, 2], [2, 3], [3, 4]], None, seed=1)]
    for h, noise in [(c, 0.0) for c in cases] + [(cases[0], 1.0), (cases[3], 0.5)]:
        o = oracle.match(h, noise=noise)
        u, sdeg = _active_sets(h, o)
        assert sdeg[0] == h.kappa
        with hmlib.Matcher.from_hypergraph(h) as mt:
            if noise:
                mt.set_noise(noise)
            mt.match()
            res = mt.result()
            plain = mt.round_stats()
            mt.profile()
            stats = mt.round_stats()
        assert res.status == OK and res.rounds == o.rounds
        if noise:
            assert plain[0, nxt] == u[0] and not plain[1:, nxt].any() and not plain[:, dg].any()
        else:
            assert plain[:o.rounds, nxt].tolist() == u and not plain[:, dg].any()
        assert not plain[:, le].any() and not plain[:, lp].any()
        assert stats[:o.rounds, nxt].tolist() == u
        assert stats[:o.rounds, dg].tolist() == sdeg
        assert stats[:o.rounds, le].tolist() == o.round_stats[:, 0].tolist()
        assert stats[:o.rounds, lp].tolist() == o.round_stats[:, 1].tolist()
        assert not stats[o.rounds:, le].any()  # the closing round finds no live edge


@pytest.mark.parametrize("big_weight", [1.0, 1e-3])
def test_edge_wider_than_16_bit_counters(big_weight):
    """One edge of 70,000 pins: the P counters cannot be 16 bits wide, so the
    32-bit counters run. Heavy, the big edge wins in round 1; light, it dies
    to a small neighbour."""
    rng = np.random.default_rng(7)
    n = 100_000
    edges = [np.sort(rng.choice(n, 70_000, replace=False)).tolist()]
    edges += [rng.choice(n, int(rng.integers(2, 6)), replace=False).tolist() for _ in range(30_000)]
    w = rng.uniform(0.01, 0.99, size=len(edges)).astype(np.float32)
    w[0] = big_weight
    h = synth.from_edges(n, edges, w.tolist(), seed=1)
    assert_parity(h)
