"""Seeded input generators: determinism, shapes, and the no-repeat rule."""
import hashlib
import os
import subprocess
import sys

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _digest(h):
    d = hashlib.sha256()
    for a in (h.eoff, h.pins) + (() if h.weights is None else (h.weights,)):
        d.update(np.ascontiguousarray(a).tobytes())
    return d.hexdigest()


def _no_repeats(h):
    edge_of = np.repeat(np.arange(h.m), np.diff(h.eoff))
    order = np.lexsort((h.pins, edge_of))
    p, e = h.pins[order], edge_of[order]
    return not np.any((p[1:] == p[:-1]) & (e[1:] == e[:-1]))


def test_deterministic_and_seeded():
    a, b, c = synth.small(seed=1), synth.small(seed=1), synth.small(seed=2)
    assert _digest(a) == _digest(b)
    assert _digest(a) != _digest(c)


def test_small_shape():
    h = synth.small()
    sizes = np.diff(h.eoff)
    assert h.n == 10_000 and h.m == 20_000
    assert sizes.min() == 2 and sizes.max() == 8
    assert abs(sizes.mean() - 5.0) < 0.05
    assert h.pins.min() >= 0 and h.pins.max() < h.n
    assert _no_repeats(h)
    w = h.weights
    assert w.dtype == np.float32 and w.min() > 0 and w.max() <= 1
    q = w.astype(np.float64) * (1 << 24)
    assert np.array_equal(q, np.round(q))  # on the 2^-24 grid


def test_powerlaw_shape():
    h = synth.large(n=200_000, m=400_000)
    sizes = np.diff(h.eoff)
    k = np.arange(2, 1025, dtype=np.float64)
    pmf = k ** -2.0
    pmf /= pmf.sum()
    assert sizes.min() >= 2 and sizes.max() <= 1024
    assert abs(sizes.mean() - (k * pmf).sum()) < 0.2
    assert abs((sizes == 2).mean() - pmf[0]) < 0.005
    assert _no_repeats(h)
    deg = np.bincount(h.pins, minlength=h.n)
    # heavy tail: the largest degree is far above the mean degree
    assert deg.max() > 100 * deg.mean()


def test_unweighted_has_no_weights():
    h = synth.unweighted(n=1000, m=2000)
    assert h.weights is None and h.unweighted


def test_thread_count_independent():
    code = ("import synth, hashlib, numpy as np;"
            "h = synth.large(n=50000, m=100000);"
            "print(hashlib.sha256(h.pins.tobytes() + h.eoff.tobytes() + h.weights.tobytes()).hexdigest())")
    outs = []
    for t in ("1", "3"):
        env = dict(os.environ, OMP_NUM_THREADS=t, PYTHONPATH=ROOT)
        outs.append(subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT,
                                   capture_output=True, text=True, check=True).stdout.strip())
    assert outs[0] == outs[1]


def test_batch_and_arrivals():
    ns = synth.batch_sizes(4096)
    assert ns.min() >= 100 and ns.max() <= 200_000
    t = synth.arrivals(10_000, 1000.0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0) and abs(gaps.mean() - 1e-3) < 1e-4


def test_from_edges():
    h = synth.from_edges(4, [[0, 1], [2], [1, 2, 3]], [0.5, 0.25, 1.0])
    assert h.eoff.tolist() == [0, 2, 3, 6] and h.pins.tolist() == [0, 1, 2, 1, 2, 3]
