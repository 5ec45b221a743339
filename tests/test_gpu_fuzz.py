"""Seeded random tiny hypergraphs through every entry point, against the
oracle: the handle path (hm_create + hm_match + hm_result, with the pair
path of graphs), hm_solve_host (whose inputs this small take the one-block
path), hm_match_noalloc, and one batch of all instances. Weights come from
three values, so most edges tie on weight and the edge-id tie-break
decides; every third instance is unweighted (seeded hash priorities), and
about a third are graphs (every edge has two pins). Edges of one pin occur
too."""
import numpy as np
import pytest
import torch

import oracle
import synth
import paper_2602_22976_gb300 as hmlib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    hmlib.build()
    oracle.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    hmlib.lib()


def tiny_instances(seed: int, count: int, weighted: bool):
    """count instances with n in [1, 24], m in [1, 40]; the batch seed is
    shared, because unweighted priorities hash it with the local edge id."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(count):
        n = int(rng.integers(1, 25))
        m = int(rng.integers(1, 41))
        graph = n >= 2 and rng.random() < 0.35
        edges = []
        for _ in range(m):
            k = 2 if graph else int(rng.integers(1, min(n, 6) + 1))
            edges.append(rng.choice(n, size=k, replace=False).tolist())
        w = list(rng.choice([0.25, 0.5, 1.0], size=m)) if weighted else None
        out.append(synth.from_edges(n, edges, w, seed=seed, name=f"tiny{seed}.{c}"))
    return out


def check(h, edges, rounds, weight=None):
    o = oracle.match(h)
    assert np.array_equal(edges, o.edges), h.name
    assert rounds == o.rounds, (h.name, rounds, o.rounds)
    if weight is not None:
        assert weight == oracle.weight(h, o.in_matching), h.name


def noalloc(h):
    dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()
    eoff, pins = dev(h.eoff, np.int64), dev(h.pins, np.int32)
    w = None if h.weights is None else dev(h.weights, np.float32)
    mask = torch.zeros(h.m, dtype=torch.uint8, device="cuda")
    result = torch.zeros(2, dtype=torch.int32, device="cuda")
    flags = hmlib.HM_UNWEIGHTED if w is None else 0
    st = hmlib.lib().hm_match_noalloc(h.n, h.m, eoff.data_ptr(), pins.data_ptr(),
                                      None if w is None else w.data_ptr(), h.seed, flags,
                                      mask.data_ptr(), result.data_ptr(), None)
    assert st == hmlib.HM_OK, hmlib.last_error()
    torch.cuda.synchronize()
    rounds, status = result.cpu().tolist()
    assert status == hmlib.HM_OK
    return np.flatnonzero(mask.cpu().numpy()).astype(np.int32), rounds


@pytest.mark.parametrize("seed", range(6))
def test_tiny_instances_every_entry_point(seed):
    weighted = seed % 3 != 2
    hs = tiny_instances(100 + seed, 40, weighted)
    assert any(int(np.diff(h.eoff).max()) == 2 == int(np.diff(h.eoff).min()) for h in hs)
    for h in hs:
        with hmlib.Matcher.from_hypergraph(h) as mt:
            mt.match()
            r = mt.result()
        check(h, r.edges, r.rounds, r.weight)
        s = hmlib.solve_host(h)
        check(h, s.edges, s.rounds, s.weight)
        e, rounds = noalloc(h)
        check(h, e, rounds)
    with hmlib.Batch(hs) as b:
        b.match()
        for h, r in zip(hs, b.result()):
            assert r.status == hmlib.HM_OK
            check(h, r.edges, r.rounds, r.weight)
