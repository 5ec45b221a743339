"""Pins of the CPU oracle against facts fixed by the paper and by mathematics,
not by the oracle itself:

* hand-derived worked cases (tests/golden, each with its derivation);
* Lemma 2's construction (the exact output and OPT = d);
* Lemma 1's bound w(M) >= OPT/d against an exhaustive optimum;
* the definitions of Sec. 2.1: vertex-disjoint, maximal, locally maximal;
* equality with the sequential greedy algorithm under the same order
  (a different algorithm; local maxima under a fixed order reproduce it);
* closed forms (a monotone path needs ceil(m/2) rounds);
* published test vectors of SplitMix64 and of the MurmurHash3 finaliser;
* planted mistakes (compile-time mutants of oracle.c) must each fail a pin.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from conftest import golden_cases, golden_hypergraph


def random_tiny(rng, n, m, kmax, weight_pool=None):
    edges = []
    for _ in range(m):
        k = int(rng.integers(1, kmax + 1))
        edges.append(sorted(rng.choice(n, size=min(k, n), replace=False).tolist()))
    if weight_pool is None:
        w = (rng.integers(1, 1 << 24, size=m) / float(1 << 24)).tolist()
    else:
        w = rng.choice(weight_pool, size=m).tolist()
    return synth.from_edges(n, edges, w)


# ---------------------------------------------------------------- golden cases

@pytest.mark.parametrize("case", golden_cases(), ids=lambda c: c["name"])
def test_golden(case):
    h = golden_hypergraph(case)
    r = oracle.match(h)
    assert r.status == 0
    assert r.edges.tolist() == case["matching"]
    assert r.rounds == case["rounds"]
    assert r.decided_round.tolist() == case["decided_round"]
    if "opt" in case:
        assert oracle.brute_opt(h)[0] == pytest.approx(case["opt"])


# ---------------------------------------------------------------- Lemma 2

@pytest.mark.parametrize("d", range(2, 9))
def test_lemma2_gadget(d):
    """Lemma 2: n = 2d, pair edges {x_i, y_i} of weight 1 and one edge of
    weight 1+eps through every x_i. Local max takes only that edge; OPT = d."""
    eps = 0.125
    edges = [[i, d + i] for i in range(d)] + [list(range(d))]
    h = synth.from_edges(2 * d, edges, [1.0] * d + [1.0 + eps])
    r = oracle.match(h)
    assert r.edges.tolist() == [d]
    assert r.rounds == 1
    opt, _ = oracle.brute_opt(h)
    assert opt == pytest.approx(d)
    w = oracle.weight(h, r.in_matching)
    assert w == pytest.approx(1.0 + eps)
    assert w >= opt / d  # Lemma 1 holds, with ratio -> 1/d as eps -> 0


# ---------------------------------------------------------------- Lemma 1

def test_lemma1_bound_random():
    rng = np.random.default_rng(7)
    checked = 0
    for trial in range(300):
        n = int(rng.integers(2, 13))
        m = int(rng.integers(1, 15))
        kmax = int(rng.integers(1, 5))
        pool = [0.25, 0.5, 0.75, 1.0] if trial % 3 == 0 else None
        h = random_tiny(rng, n, m, kmax, pool)
        r = oracle.match(h)
        d = int(np.max(np.diff(h.eoff)))
        opt, best = oracle.brute_opt(h)
        wm = oracle.weight(h, r.in_matching)
        assert oracle.check_disjoint(h, best) == -1
        assert wm <= opt + 1e-9
        assert wm >= opt / d - 1e-9
        checked += 1
    assert checked == 300


# ---------------------------------------------------------------- definitions

def _assert_definitions(h, r):
    assert r.status == 0
    assert oracle.check_disjoint(h, r.in_matching) == -1
    assert oracle.check_maximal(h, r.in_matching) == -1
    assert oracle.check_local_max(h, r.in_matching, r.decided_round) == -1
    # every edge is decided in some round, no later than the last round
    if h.m:
        assert r.decided_round.min() >= 1
        assert r.decided_round.max() == r.rounds


def _instances():
    yield synth.small()
    yield synth.small(seed=2, n=500, m=3000)
    yield synth.generate(300, 2000, kmin=1, kmax=5, seed=3)
    yield synth.unweighted(seed=4, n=20_000, m=40_000)
    yield synth.large(seed=5, n=20_000, m=40_000, kmax=256)
    yield synth.generate(50, 4000, kmin=2, kmax=4, seed=6)  # dense: many ties in the argmax
    yield synth.rgg(seed=7, n=5_000)  # a graph (every edge has two pins)


@pytest.mark.parametrize("idx", range(7))
def test_definitions_and_greedy(idx):
    h = list(_instances())[idx]
    r = oracle.match(h)
    _assert_definitions(h, r)
    assert np.array_equal(oracle.greedy(h), r.in_matching)


def test_greedy_equality_with_ties():
    rng = np.random.default_rng(11)
    for _ in range(200):
        h = random_tiny(rng, int(rng.integers(3, 30)), int(rng.integers(1, 60)),
                        int(rng.integers(1, 6)), [0.5, 1.0])
        r = oracle.match(h)
        _assert_definitions(h, r)
        assert np.array_equal(oracle.greedy(h), r.in_matching)


# ---------------------------------------------------------------- order on edges

def test_weighted_order_is_weight_then_smaller_id():
    rng = np.random.default_rng(3)
    w = rng.choice(np.array([0.125, 0.5, 0.5, 1.0, 3.0, 1e-30, 7e30], dtype=np.float32), size=400)
    h = synth.from_edges(2, [[0]] * len(w), w.tolist())
    k = oracle.keys(h)
    # descending key order must equal lexicographic (-w, id)
    expect = np.lexsort((np.arange(len(w)), -w.astype(np.float64)))
    got = sorted(range(len(w)), key=lambda e: -int(k[e]))
    assert got == expect.tolist()


def test_splitmix64_published_vector():
    # SplitMix64 (Steele, Lea, Flood 2014) seeded with 0: first output
    assert oracle.splitmix64_first(0) == 0xE220A8397B1DCDAF


def test_fmix32_published_vectors():
    # MurmurHash3_x86_32 of the empty key equals fmix32(seed) (Appleby):
    # seed 0 -> 0, seed 1 -> 0x514E28B7, seed 0xFFFFFFFF -> 0x81F16F39
    assert oracle.fmix32(0) == 0
    assert oracle.fmix32(1) == 0x514E28B7
    assert oracle.fmix32(0xFFFFFFFF) == 0x81F16F39


def _inv_xorshift(y, s):
    x = y
    for _ in range(32 // s + 1):
        x = y ^ (x >> s)
    return x & 0xFFFFFFFF


def test_fmix32_is_a_bijection():
    """fmix32 is xorshifts and multiplications by odd constants, each
    invertible mod 2^32; undoing them step by step recovers every input."""
    c1 = pow(0x85EBCA6B, -1, 1 << 32)
    c2 = pow(0xC2B2AE35, -1, 1 << 32)
    rng = np.random.default_rng(5)
    xs = [0, 1, 2, 0xFFFFFFFF, 0x80000000] + rng.integers(0, 1 << 32, size=2000).tolist()
    for x in xs:
        y = oracle.fmix32(int(x))
        y = _inv_xorshift(y, 16)
        y = (y * c2) & 0xFFFFFFFF
        y = _inv_xorshift(y, 13)
        y = (y * c1) & 0xFFFFFFFF
        y = _inv_xorshift(y, 16)
        assert y == x


def test_unweighted_order_strict_and_seeded():
    h1 = synth.unweighted(seed=1, n=1000, m=5000)
    k1 = oracle.keys(h1)
    assert len(np.unique(k1)) == len(k1)
    h2 = synth.Hypergraph(h1.n, h1.m, h1.eoff, h1.pins, None, seed=2)
    assert not np.array_equal(oracle.keys(h2), k1)
    assert np.all((k1 >> np.uint64(32)) == np.uint64(0x3F800000))  # high word: bits of 1.0f


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("m", [1, 2, 3, 10, 17, 40])
@pytest.mark.parametrize("increasing", [True, False])
def test_path_closed_form(m, increasing):
    """A path whose weights increase (or are all equal) along it: one edge
    wins per round, so ceil(m/2) rounds, and every other edge is matched."""
    w = [(i + 1) / 64 for i in range(m)] if increasing else [0.5] * m
    h = synth.from_edges(m + 1, [[i, i + 1] for i in range(m)], w)
    r = oracle.match(h)
    assert r.rounds == math.ceil(m / 2)
    first = (m - 1) % 2 if increasing else 0
    assert r.edges.tolist() == list(range(first, m, 2))


def test_round_stats_bookkeeping():
    h = synth.large(seed=9, n=50_000, m=100_000, kmax=512)
    r = oracle.match(h)
    st = r.round_stats
    assert st[0, 0] == h.m and st[0, 1] == h.kappa
    assert st[:, 2].sum() == r.in_matching.sum()
    decided = np.bincount(r.decided_round, minlength=r.rounds + 1)
    for k in range(r.rounds - 1):
        assert st[k + 1, 0] == st[k, 0] - decided[k + 1]
    assert st[-1, 0] == decided[r.rounds]


def test_invariant_under_pin_order_and_repeat():
    h = synth.small(seed=3, n=2000, m=6000)
    r1 = oracle.match(h)
    rng = np.random.default_rng(1)
    pins = h.pins.copy()
    for e in range(h.m):
        seg = pins[h.eoff[e]:h.eoff[e + 1]]
        rng.shuffle(seg)
    h2 = synth.Hypergraph(h.n, h.m, h.eoff, pins, h.weights, h.seed)
    r2 = oracle.match(h2)
    r3 = oracle.match(h)
    assert np.array_equal(r1.in_matching, r2.in_matching) and r1.rounds == r2.rounds
    assert np.array_equal(r1.decided_round, r3.decided_round)


def test_round_cap_and_state():
    h = synth.from_edges(8, [[i, i + 1] for i in range(7)], [(i + 1) / 8 for i in range(7)])
    r = oracle.match(h, max_rounds=1)
    assert r.status == 1 and r.rounds == 1 and r.edges.tolist() == [6]
    vs = oracle.vertex_state(r)
    # round 1: vertex v picks edge v (its heavier edge) except v=0 (edge 0) and v=7 (edge 6)
    assert vs.tolist() == [0, 1, 2, 3, 4, 5, -1, -1]


# ---------------------------------------------------------------- planted mistakes

def _pins_pass(mutant):
    try:
        for c in golden_cases():
            h = golden_hypergraph(c)
            r = oracle.match(h, mutant=mutant)
            if r.status != 0 or r.edges.tolist() != c["matching"] or r.rounds != c["rounds"]:
                return False
        rng = np.random.default_rng(2)
        for _ in range(30):
            h = random_tiny(rng, 12, 20, 4, [0.5, 1.0])
            r = oracle.match(h, mutant=mutant)
            if r.status != 0 or oracle.check_disjoint(h, r.in_matching) != -1:
                return False
            if oracle.check_maximal(h, r.in_matching) != -1:
                return False
            if not np.array_equal(oracle.greedy(h), r.in_matching):
                return False
        return True
    except Exception:
        return False


def test_pins_accept_the_oracle():
    assert _pins_pass(0)


@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5])
def test_pins_reject_planted_mistakes(mutant):
    # 1 reversed tie-break, 2 argmin for argmax, 3 one vertex consulted,
    # 4 no deactivation step, 5 dead edges keep competing
    assert not _pins_pass(mutant)


# ---------------------------------------------------------------- re-randomised rounds

def test_splitmix64_stream_published_vectors():
    # SplitMix64 seeded with 0: outputs 1, 2, 3 (Steele, Lea, Flood 2014)
    assert oracle.splitmix64_at(0, 1) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64_at(0, 2) == 0x6E789E6AA1B965F4
    assert oracle.splitmix64_at(0, 3) == 0x06C45D188009454F


@pytest.mark.parametrize("r,e,x,top24,bits", [
    (1, 0, 0x1F69EA35BA1A6227, 2058730, 1059023338),
    (2, 5, 0x18DD9D9FE048EE4E, 1629597, 1058594205),
    (3, 7, 0xA8A8458085A42786, 11053125, 1066685474),
])
def test_round_priority_worked_example(r, e, x, top24, bits):
    """p_r(e) for seed 0, weight 0.5, amplitude 1, worked step by step. The
    priority stream starts at s0 = the first SplitMix64 output of seed 0,
    0xE220A8397B1DCDAF (the published vector above); round r of edge e uses
    output number k = (r << 32) + e + 1 of that stream, x; U = top 24 bits
    of x times 2^-24; p = 0.5 + 1 * U, each operation rounded to float32
    (the sum is the only inexact step here). A counter off by one in r or e
    gives another x and fails this."""
    s0 = 0xE220A8397B1DCDAF
    assert oracle.splitmix64_first(0) == s0
    k = (r << 32) + e + 1
    assert oracle.splitmix64_at(s0, k) == x
    assert x >> 40 == top24
    u = np.float32(top24) * np.float32(2.0 ** -24)  # exact: a 24-bit integer times a power of two
    p = np.float32(np.float32(0.5) + u)
    assert int(p.view(np.uint32)) == bits
    h = synth.from_edges(20, [[i, i + 1] for i in range(9)], [0.5] * 9, seed=0)
    assert np.float32(oracle.round_priority(h, 1.0, r, e)) == p


def test_round_priorities_in_range():
    h = synth.small(seed=2, n=1000, m=3000)
    ps = np.array([[oracle.round_priority(h, 100.0, r, e) - float(h.weights[e]) for e in range(0, 3000, 7)]
                   for r in (1, 2, 9)])
    assert ps.min() >= 0.0 and ps.max() < 100.0 + 1e-3
    assert abs(ps.mean() - 50.0) < 2.5
    assert not np.array_equal(ps[0], ps[1])  # redrawn every round


def test_tiny_noise_keeps_the_fixed_order():
    """Noise far below the gaps between (distinct) weights cannot reorder
    edges: the re-randomised rounds then reproduce the fixed-order run."""
    rng = np.random.default_rng(4)
    h = synth.small(seed=4, n=3000, m=9000)
    h.weights = ((rng.permutation(9000) + 1) / 16384.0).astype(np.float32)  # distinct, gap 2^-14
    a, b = oracle.match(h), oracle.match(h, noise=2.0 ** -24)
    assert a.rounds == b.rounds and np.array_equal(a.in_matching, b.in_matching)


@pytest.mark.parametrize("idx", range(5))
def test_randomised_definitions(idx):
    h = [synth.small(seed=6), synth.unweighted(seed=3, n=20_000, m=40_000),
         synth.large(seed=5, n=20_000, m=40_000, kmax=256), synth.generate(50, 4000, kmin=2, kmax=4, seed=8),
         synth.generate(300, 2000, kmin=1, kmax=5, seed=9)][idx]
    r = oracle.match(h, noise=100.0)
    assert r.status == 0
    assert oracle.check_disjoint(h, r.in_matching) == -1
    assert oracle.check_maximal(h, r.in_matching) == -1
    assert oracle.check_local_max(h, r.in_matching, r.decided_round, noise=100.0) == -1
    r2 = oracle.match(h, noise=100.0)
    assert np.array_equal(r.in_matching, r2.in_matching) and r.rounds == r2.rounds


def test_randomised_cardinality_bound():
    """With fresh priorities every round the rounds solve the cardinality
    problem (Sec. 3.2); the result is maximal, so |M| >= OPT/d (Lemma 1 with
    unit weights). For the original weights no such bound holds: the local
    maxima are taken under the noisy priorities."""
    rng = np.random.default_rng(12)
    for trial in range(150):
        h = random_tiny(rng, int(rng.integers(2, 13)), int(rng.integers(1, 15)), int(rng.integers(1, 5)))
        h.weights = None
        r = oracle.match(h, noise=float(rng.choice([0.5, 100.0])))
        d = int(np.max(np.diff(h.eoff)))
        opt, _ = oracle.brute_opt(h)
        card = float(r.in_matching.sum())
        assert opt / d - 1e-9 <= card <= opt + 1e-9


def test_randomised_rounds_grow_like_log_m():
    """Claim 2: with fresh uniform priorities every round, O(log m) rounds."""
    for m in (1_000, 10_000, 100_000):
        h = synth.unweighted(seed=1, n=m // 2, m=m)
        r = oracle.match(h, noise=1.0)
        assert r.rounds <= 2 * math.log2(m), (m, r.rounds)


def test_randomised_mutant_caught():
    # mutant 6 draws the priorities once instead of before every round
    h = synth.small(seed=6)
    r = oracle.match(h, noise=100.0, mutant=6)
    assert oracle.check_local_max(h, r.in_matching, r.decided_round, noise=100.0) != -1


def test_weight_is_the_exact_sum_rounded_once():
    """w(M) = sum of w(e) over e in M (Sec. 2.1) is an exact real sum; the
    oracle returns it rounded once to the nearest float64. Exact rational
    arithmetic (fractions.Fraction, whose float() rounds correctly) fixes
    that value independently, on weights from the generators' grid, over a
    wide exponent range, and with subnormal and near-maximal float32
    values, where a running float64 sum would drift."""
    import types
    from fractions import Fraction
    rng = np.random.default_rng(5)
    special = np.array([2.0 ** -149, 1e-38, 1.0, 3.0e38, 0.1, 1.0 - 2.0 ** -24], dtype=np.float32)
    for case in range(60):
        m = int(rng.integers(1, 4000))
        kind = case % 3
        if kind == 0:
            w = ((rng.integers(0, 1 << 24, m) + 1) * 2.0 ** -24).astype(np.float32)
        elif kind == 1:
            w = np.exp(rng.uniform(-85.0, 85.0, m)).astype(np.float32)
        else:
            w = rng.choice(special, m).astype(np.float32)
        mask = rng.random(m) < 0.6
        exact = sum((Fraction(float(x)) for x in w[mask]), Fraction(0))
        assert oracle.weight(types.SimpleNamespace(weights=w), mask.astype(np.uint8)) == float(exact)


def _replay_rounds(h):
    """The fixed-order rounds replayed directly on tiny inputs (plain Python,
    independent of the oracle's C code): each vertex keeps a cursor into its
    list sorted by decreasing key; at the start of a round every unmatched
    vertex moves its cursor past dead entries (to the end when none is
    left). Returns the active vertices per round, their degree sums, the
    cursor moves over the run, the matching and the round count."""
    keys = [int(k) for k in oracle.keys(h)]
    edges = [h.pins[h.eoff[e]:h.eoff[e + 1]].tolist() for e in range(h.m)]
    lists = [[] for _ in range(h.n)]
    for e, pins in enumerate(edges):
        for v in pins:
            lists[v].append(e)
    for v in range(h.n):
        lists[v].sort(key=lambda e: -keys[e])
    alive = [True] * h.m
    matched = [False] * h.n
    cur = [0] * h.n
    moves, U, D, M, rounds = 0, [], [], [], 0
    while True:
        for v in range(h.n):
            if not matched[v]:
                c = cur[v]
                while c < len(lists[v]) and not alive[lists[v][c]]:
                    c += 1
                moves += c - cur[v]
                cur[v] = c
        active = [v for v in range(h.n) if not matched[v] and cur[v] < len(lists[v])]
        if not active:
            break
        rounds += 1
        U.append(len(active))
        D.append(sum(len(lists[v]) for v in active))
        T = {v: lists[v][cur[v]] for v in active}
        winners = [e for e in range(h.m) if alive[e] and all(T.get(v) == e for v in edges[e])]
        for e in winners:
            M.append(e)
            for v in edges[e]:
                matched[v] = True
        for e in range(h.m):
            if alive[e] and any(matched[v] for v in edges[e]):
                alive[e] = False
    return U, D, moves, sorted(M), rounds


@pytest.mark.parametrize("seed", range(4))
def test_active_sets_and_cursor_moves_by_replay(seed):
    """The counts the GPU tests derive from the oracle's run - the active
    vertices and their degree sums per round, and the entries the cursors
    pass (those ahead of each vertex's matching edge, or its whole list) -
    equal a direct replay of the rounds, whose matching and round count
    equal the oracle's, on tiny hypergraphs and graphs with tied weights."""
    from cursor_work import active_sets, entries_ahead_of_the_match
    rng = np.random.default_rng(500 + seed)
    for c in range(30):
        n = int(rng.integers(2, 20))
        m = int(rng.integers(1, 30))
        graph = rng.random() < 0.4
        edges = [rng.choice(n, size=2 if graph else int(rng.integers(1, min(n, 5) + 1)),
                            replace=False).tolist() for _ in range(m)]
        w = None if c % 4 == 3 else list(rng.choice([0.25, 0.5, 1.0], size=m))
        h = synth.from_edges(n, edges, w, seed=seed + 1)
        o = oracle.match(h)
        U, D, moves, M, rounds = _replay_rounds(h)
        assert M == o.edges.tolist() and rounds == o.rounds
        assert (U, D) == active_sets(h, o)
        assert moves == entries_ahead_of_the_match(h, o)
