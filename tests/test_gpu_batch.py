"""Batched matching (hm_batch_*): every instance of a batch must get exactly
the matching, round count and weight that the CPU oracle gives it alone."""
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
    assert torch.cuda.is_available(), "needs a CUDA device"
    hmlib.lib()


def mixed_instances(seed, weighted=True, count=40):
    rng = np.random.default_rng(seed)
    hs = []
    for i in range(count):
        kind = i % 3
        n = int(np.exp(rng.uniform(np.log(20), np.log(30_000))))
        gs = seed * 1000 + i
        if kind == 0:
            h = synth.generate(n, 2 * n, kmin=2, kmax=16, weighted=weighted, seed=gs)
        elif kind == 1:
            h = synth.generate(max(n, 300), 2 * max(n, 300), size_dist=synth.SIZE_ZIPF, kmin=2, kmax=256,
                               pin_dist=synth.PINS_POWERLAW, weighted=weighted, seed=gs)
        else:
            h = synth.generate(n, n // 2 + 1, kmin=1, kmax=6, weighted=weighted, seed=gs)
        h.seed = seed  # one priority seed for the whole batch
        hs.append(h)
    return hs


def check_against_oracle(hs, results):
    assert len(results) == len(hs)
    for h, r in zip(hs, results):
        o = oracle.match(h)
        assert r.status == hmlib.HM_OK
        assert r.rounds == o.rounds, (h.name, r.rounds, o.rounds)
        assert np.array_equal(r.edges, o.edges), h.name
        assert r.weight == oracle.weight(h, o.in_matching)


@pytest.mark.parametrize("weighted", [True, False])
def test_batch_matches_solo_oracle(weighted):
    hs = mixed_instances(3 if weighted else 4, weighted)
    with hmlib.Batch(hs) as b:
        ncls, cls, cfg = b.info()
        assert ncls >= 2 and cls.shape == (len(hs),)
        b.match()
        check_against_oracle(hs, b.result())
        b.match()  # a second launch recomputes the same result
        check_against_oracle(hs, b.result())


@pytest.mark.parametrize("weighted", [True, False])
def test_batch_one_class(weighted):
    """HM_ONE_CLASS: every instance in one union; each still gets its solo result."""
    hs = mixed_instances(5 if weighted else 6, weighted, count=30)
    with hmlib.Batch(hs, one_class=True) as b:
        ncls, cls, cfg = b.info()
        assert ncls == 1 and np.all(cls == 0)
        b.match()
        check_against_oracle(hs, b.result())


@pytest.mark.parametrize("weighted", [True, False])
def test_batch_one_class_of_small_instances(weighted):
    """HM_ONE_CLASS over instances all below 65,536 pins (the server's groups
    of small requests): the class runs on the one-block workers, and every
    instance still gets its solo result; a second launch repeats it. One
    member has 300,000 isolated vertices: its working memory (9n + m bytes)
    is above a worker's 2 MiB, so that class runs as a union instead."""
    rng = np.random.default_rng(7 if weighted else 8)
    hs = []
    for i in range(60):
        n = int(rng.integers(10, 3000))
        h = synth.generate(n, 2 * n, kmin=1, kmax=12, weighted=weighted, seed=700 + i)
        h.seed = 2
        hs.append(h)
    with hmlib.Batch(hs, one_class=True) as b:
        b.match()
        check_against_oracle(hs, b.result())
        b.match()
        check_against_oracle(hs, b.result())
    big = synth.generate(300_000, 200, kmin=2, kmax=4, weighted=weighted, seed=799)
    big.seed = 2
    with hmlib.Batch(hs[:5] + [big], one_class=True) as b:
        b.match()
        check_against_oracle(hs[:5] + [big], b.result())


def test_batch_degenerate_members():
    hs = [synth.from_edges(5, [], []),
          synth.from_edges(3, [[0, 1, 2]], [0.5]),
          synth.small(seed=2, n=500, m=1000),
          synth.from_edges(8, [[i, i + 1] for i in range(7)], [(i + 1) / 8 for i in range(7)]),
          synth.from_edges(1, [[0]], [1.0])]
    for h in hs:
        h.seed = 1
    with hmlib.Batch(hs) as b:
        b.match()
        check_against_oracle(hs, b.result())


def test_batch_autotuned_same_result():
    hs = mixed_instances(5, True, count=24)
    with hmlib.Batch(hs, autotune=True) as b:
        ncls, _, cfg = b.info()
        assert cfg.shape == (ncls, 4) and np.all(cfg[:, 0] >= 64)
        b.match()
        check_against_oracle(hs, b.result())


def test_single_handle_autotune_and_config():
    h = synth.large(seed=4, n=200_000, m=400_000)
    o = oracle.match(h)
    with hmlib.Matcher.from_hypergraph(h) as mt:
        assert mt.launch_config() == (64, 0, 0, 0)
        for cfg in [(64, 2, 2, 2), (1024, 0, 4, 0), (128, 1, 0, 4)]:
            assert mt.launch_config(cfg) == cfg
            mt.match()
            r = mt.result()
            assert np.array_equal(r.edges, o.edges) and r.rounds == o.rounds
        best, ms = mt.autotune()
        assert ms > 0 and best[0] in (64, 128, 256, 512, 1024)
        mt.match()
        r = mt.result()
        assert np.array_equal(r.edges, o.edges) and r.rounds == o.rounds
        with pytest.raises(hmlib.HMError):
            mt.launch_config((8, 0, 0, 0))


def test_batch_rejects_cross_instance_inputs():
    """Inside the union a pin of one instance would be another instance's
    vertex, so pins are checked against their own instance's n; and every
    instance's offsets must start at 0 (else its first edges would take the
    previous instance's pins)."""
    a = synth.small(seed=3, n=400, m=800)
    b = synth.small(seed=4, n=400, m=800)
    for h in (a, b):
        h.seed = 1
    bad_pin = synth.Hypergraph(b.n, b.m, b.eoff.copy(), b.pins.copy(), b.weights, 1, "bad pin")
    bad_pin.pins[10] = b.n + 3  # inside the union, outside its own instance
    with pytest.raises(hmlib.HMError) as ei:
        hmlib.Batch([a, bad_pin])
    assert ei.value.status == hmlib.HM_EINVAL
    shifted = synth.Hypergraph(b.n, b.m - 1, b.eoff[1:].copy(), b.pins, b.weights[1:].copy(), 1, "offsets from 2")
    with pytest.raises(hmlib.HMError) as ei:
        hmlib.Batch([a, shifted])
    assert ei.value.status == hmlib.HM_EINVAL
    with hmlib.Batch([a, b]) as ok:  # the valid pair still works
        ok.match()
        check_against_oracle([a, b], ok.result())


def test_full_size_batch_in_bench_configuration():
    """The batching workload at full size, launched as the bench launches it
    (4,096 instances, n log-uniform in [100, 200,000], m = 2n, |e| ~ U{2..16},
    Sigma kappa = 2.04e9, autotuned size classes): every one of the 4,096
    instances equals the CPU oracle run on it alone - matched edge set, round
    count and exact weight. The oracle runs in a process pool over the host
    cores while the GPU works; each oracle run is the plain single-threaded
    one."""
    from oracle_pool import collect, start_batch_oracle
    count, seed = 4096, 1
    pool, pending = start_batch_oracle(count, seed, prio_seed=1)
    hs = synth.batch(count, seed=seed)
    for h in hs:
        h.seed = 1
    with hmlib.Batch(hs, autotune=True) as b:
        b.match()
        res = b.result()
    assert len(res) == count
    ref = collect(pool, pending)
    assert [x[0] for x in ref] == list(range(count))
    mismatched = []
    for (i, edges, rounds, weight, status), h, r in zip(ref, hs, res):
        assert status == 0, i
        assert r.status == hmlib.HM_OK, i
        if not (r.rounds == rounds and np.array_equal(r.edges, edges) and r.weight == weight):
            mismatched.append(i)
    assert not mismatched, f"{len(mismatched)} instances differ from the oracle, first {mismatched[:10]}"


def test_batch_of_graphs():
    """A batch whose instances are all graphs: each size class's union is a
    graph and takes the pair paths of the build and the loop."""
    hs = [synth.rgg(seed=40 + i, n=int(n), avg_degree=d) for i, (n, d) in
          enumerate([(500, 6.0), (3000, 16.0), (20000, 10.0), (800, 30.0), (60000, 16.0)])]
    for h in hs:
        h.seed = 1
    with hmlib.Batch(hs) as b:
        b.match()
        check_against_oracle(hs, b.result())
