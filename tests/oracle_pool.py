"""Oracle runs spread over the host cores, for parity checks of many
independent instances (the batching workload).

Each worker process regenerates its instances from their seeds (the batch
generator draws instance i from its own seed, so nothing large crosses the
process boundary) and runs the single-threaded oracle on each. The pool is
started with the "spawn" method: a process forked after the parent has
initialised CUDA can hang, and spawned workers never touch the GPU.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

_SIZES: dict = {}


def _init_worker():
    os.environ["OMP_NUM_THREADS"] = "1"  # the generator's OpenMP: one thread per worker


def _batch_instance(count: int, seed: int, i: int):
    import synth
    key = (count, seed)
    if key not in _SIZES:
        _SIZES[key] = synth.batch_sizes(count, seed=seed)
    n = int(_SIZES[key][i])
    # the same recipe as synth.batch: instance i has its own generator seed
    h = synth.generate(n, 2 * n, kmin=2, kmax=16, seed=seed * 1_000_003 + i, name=f"batch{i}")
    return h


def _oracle_batch_chunk(args):
    count, seed, prio_seed, idx = args
    import oracle
    out = []
    for i in idx:
        h = _batch_instance(count, seed, i)
        h.seed = prio_seed
        o = oracle.match(h)
        out.append((i, o.edges, o.rounds, oracle.weight(h, o.in_matching), o.status))
    return out


def workers() -> int:
    return max(1, min(32, os.cpu_count() or 1))


def start_batch_oracle(count: int, seed: int, prio_seed: int, procs: int | None = None):
    """Starts the oracle on instances 0..count-1 of synth.batch(count, seed)
    with priority seed prio_seed; returns (pool, async result). The result's
    .get() gives [(i, edges, rounds, weight, status)] in instance order."""
    import oracle
    import synth
    synth.build()   # compile once in the parent, not in every worker
    oracle.build()
    procs = procs or workers()
    # interleaved chunks: instance sizes vary by a factor of 2000
    chunks = [(count, seed, prio_seed, list(range(k, count, 4 * procs))) for k in range(4 * procs)]
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(procs, initializer=_init_worker)
    res = pool.map_async(_oracle_batch_chunk, chunks)
    return pool, res


def collect(pool, res, timeout: float = 1800.0):
    try:
        parts = res.get(timeout)
    finally:
        pool.close()
        pool.join()
    flat = sorted((x for p in parts for x in p), key=lambda x: x[0])
    return flat
