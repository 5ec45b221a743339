"""Re-randomised rounds (hm_set_noise > 0) vs the CPU oracle with the same
noise amplitude, through the C ABI.

Priorities are re-drawn before every round from a counter-based generator
of (seed, round, edge), so the result is still unique: matched edges, round
count, per-round winner counts and live pins, and the matching weight must
be identical, and so must the per-vertex state after a capped run. Round 1
is vertex-driven (a flat scan of every list), later rounds edge-driven; the
cases cover hub vertices of very high degree, edges of up to 1024 pins
(tested by a whole warp), graphs, and switching a handle between the fixed
and the re-randomised order.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2602_22976_gb300 as hmlib

pytestmark = pytest.mark.gpu

OK, EINVAL, ETIMEOUT = hmlib.HM_OK, hmlib.HM_EINVAL, hmlib.HM_ETIMEOUT
WIN = hmlib.STAT_COLUMNS.index("winners")
PROPOSALS = hmlib.STAT_COLUMNS.index("proposals")
LIVE = hmlib.STAT_COLUMNS.index("live")
SCANNED = hmlib.STAT_COLUMNS.index("advance")


@pytest.fixture(scope="module", autouse=True)
def _built():
    hmlib.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    hmlib.lib()


def run_gpu(h, noise, cap=None):
    with hmlib.Matcher.from_hypergraph(h) as mt:
        mt.set_noise(noise)
        if cap is not None:
            mt.set_round_cap(cap)
        mt.match()
        res = mt.result(allow=(OK, ETIMEOUT))
        stats = mt.round_stats()
        vs = mt.vertex_state()
    return res, stats, vs


def assert_parity(h, noise, res=None, stats=None):
    if res is None:
        res, stats, _ = run_gpu(h, noise)
    o = oracle.match(h, noise=noise)
    assert res.status == OK
    assert res.rounds == o.rounds
    assert np.array_equal(res.edges, o.edges)
    assert stats[:o.rounds, WIN].tolist() == o.round_stats[:, 2].tolist()
    # every live entry of every vertex list is seen by the scan: the live
    # pins of each round, exactly
    assert stats[:o.rounds, LIVE].tolist() == o.round_stats[:, 1].tolist()
    assert np.all(stats[:o.rounds, SCANNED] >= stats[:o.rounds, LIVE])
    assert res.weight == oracle.weight(h, o.in_matching)
    return o


def hub_graph(seed, n, hubs, hub_deg, rest):
    """Random small edges plus `hubs` vertices that sit in hub_deg edges each."""
    rng = np.random.default_rng(seed)
    edges, w = [], []
    for hv, d in zip(range(hubs), hub_deg):
        for _ in range(d):
            e = {hv} | set(rng.choice(np.arange(hubs, n), size=int(rng.integers(1, 4)), replace=False).tolist())
            edges.append(sorted(e))
            w.append(float(rng.integers(1, 1 << 24)) / (1 << 24))
    for _ in range(rest):
        edges.append(sorted(rng.choice(n, size=int(rng.integers(2, 7)), replace=False).tolist()))
        w.append(float(rng.integers(1, 1 << 24)) / (1 << 24))
    perm = rng.permutation(len(edges))
    return synth.from_edges(n, [edges[i] for i in perm], [w[i] for i in perm], name=f"hubs{seed}")


@pytest.mark.parametrize("noise", [1e-3, 0.5, 100.0])
def test_small_weighted(noise):
    assert_parity(synth.small(seed=11, n=5000, m=15_000), noise)


@pytest.mark.parametrize("seed", [1, 2])
def test_powerlaw_scaled(seed):
    """Zipf sizes up to 256 and power-law degrees: lists of every length."""
    assert_parity(synth.large(seed=seed, n=200_000, m=400_000, kmax=256), 100.0)


def test_unweighted_cardinality_rounds():
    h = synth.generate(50_000, 100_000, kmin=2, kmax=8, weighted=False, seed=4)
    o = assert_parity(h, 1.0)
    assert o.rounds <= 4 * math.ceil(math.log2(h.m))  # O(log m) rounds (Claim 2)


def test_long_lists_in_chunks():
    """Hubs of degree 2049, 4096, 4097 and 10000, matched or not in various
    rounds: round 1's flat scan folds a hub's list from many chunks, and
    the edge rounds offer thousands of keys to one vertex slot."""
    h = hub_graph(3, 30_000, 4, [2049, 4096, 4097, 10_000], 40_000)
    for noise in (0.25, 50.0):
        assert_parity(h, noise)


def test_degenerate_inputs():
    cases = [synth.from_edges(5, [], []),
             synth.from_edges(3, [[0, 1, 2]], [0.5]),
             synth.from_edges(4, [[0], [1], [2, 3], [3]], [1.0, 0.25, 0.5, 0.75]),
             synth.from_edges(6, [[0, 1], [1, 2], [2, 3], [3, 4], [4, 5]], [1.0] * 5)]
    for h in cases:
        for noise in (0.5, 1e6):
            assert_parity(h, noise)


@pytest.mark.parametrize("cap", [1, 2, 3, 5])
def test_vertex_state_after_capped_rounds(cap):
    """a1 parity: T[v] after round r is the oracle's argmax of round r. Cap 1
    stops after the vertex-driven round; caps 2, 3 and 5 after an edge round,
    where the next round only counts the live edges (HM_ETIMEOUT if one is
    left) and the vertex state is read from that round's key slots."""
    for h in (synth.small(seed=5, n=5000, m=15_000), hub_graph(6, 20_000, 2, [3000, 5000], 20_000),
              synth.large(seed=8, n=30_000, m=60_000, kmax=256), synth.rgg(seed=6, n=20_000)):
        res, stats, vs = run_gpu(h, 10.0, cap=cap)
        o = oracle.match(h, max_rounds=cap, noise=10.0)
        assert res.rounds == min(cap, o.rounds)
        assert np.array_equal(vs, oracle.vertex_state(o))
        assert np.array_equal(res.edges, o.edges)


def test_switch_modes_and_repeat():
    h = synth.large(seed=9, n=100_000, m=200_000, kmax=256)
    fixed = oracle.match(h)
    rand = oracle.match(h, noise=3.0)
    with hmlib.Matcher.from_hypergraph(h) as mt:
        for noise, o in ((0.0, fixed), (3.0, rand), (3.0, rand), (0.0, fixed), (3.0, rand)):
            mt.set_noise(noise)
            mt.match()
            r = mt.result()
            assert np.array_equal(r.edges, o.edges) and r.rounds == o.rounds
        prof = mt.profile()
        r = mt.result()
        assert np.array_equal(r.edges, o.edges) and r.rounds == o.rounds
        # round 1 has a kill kernel; from round 2 on the next round's filter
        # finds the dead edges, and every round's win step ends it
        assert prof["kill"][1] == 1 and prof["win"][1] >= rand.rounds
        assert prof["round_end"][1] == 0  # part of the kill / win kernels
        stats = mt.round_stats()
        assert stats[:rand.rounds, WIN].tolist() == rand.round_stats[:, 2].tolist()
        assert np.all(stats[:rand.rounds, PROPOSALS] > 0)


def test_every_live_edge_wins_in_one_round():
    """Pairwise disjoint edges: all of them win in round 1 and nothing is
    left (no edge round runs); then a chain whose last edge round ends with
    every live edge winning."""
    h = synth.from_edges(12, [[0, 1, 2], [3, 4], [5, 6, 7, 8], [9, 10, 11]], [0.5, 0.25, 0.75, 1.0])
    for noise in (0.5, 1e3):
        o = assert_parity(h, noise)
        assert o.rounds == 1
    chain = synth.from_edges(40, [[i, i + 1] for i in range(39)], [(i % 7 + 1) / 8 for i in range(39)])
    for noise in (0.3, 10.0):
        assert_parity(chain, noise)


def test_different_seeds_differ():
    h = synth.small(seed=12, n=3000, m=9000)
    h2 = synth.small(seed=12, n=3000, m=9000)
    h2.seed = h.seed + 1
    a = assert_parity(h, 100.0)
    b = assert_parity(h2, 100.0)
    assert not np.array_equal(a.edges, b.edges)


def test_invalid_amplitude():
    h = synth.from_edges(3, [[0, 1]], [1.0])
    with hmlib.Matcher.from_hypergraph(h) as mt:
        for bad in (-1.0, float("nan"), float("inf")):
            with pytest.raises(hmlib.HMError) as ei:
                mt.set_noise(bad)
            assert ei.value.status == EINVAL


@pytest.mark.slow
def test_full_size_powerlaw_random():
    """n=10M, m=20M power-law hypergraph (kappa ~ 2.02e8), re-randomised rounds."""
    assert_parity(synth.large(), 1.0)


def test_graph_rgg_random():
    """Re-randomised rounds on a graph (every edge has two pins: the proposal
    takes |e| = 2 without reading offsets)."""
    h = synth.rgg(seed=4, n=40_000, avg_degree=12.0)
    assert_parity(h, 1.0)
