"""Seeded synthetic hypergraph inputs (input producer only).

The generators live in ``synth.c`` (compiled on first use with gcc/OpenMP);
this module marshals numpy arrays. Nothing here computes any part of the
matching method: it only draws edge sizes, pins and weights.

Workload recipes (the paper's real-world instances are not available, so
these stand in for them; their shapes follow the paper's instance-statistics
tables in the appendix: heavy-tailed edge sizes and vertex degrees):

* ``small``      n=10,000, m=20,000, |e| ~ U{2..8}, pins uniform without
                 repeats, float32 weights uniform on the grid (0,1], seed 1.
* ``large``      n=10M, m=20M, |e| ~ Zipf(2) on [2,1024], pins power-law
                 (P(v) ~ (v+1)^-1/(gamma-1), gamma=2.2) with shuffled ids.
* ``unweighted`` the ``small`` generator at n=4M, m=8M; no weights, a
                 seeded hash priority orders the edges.
* ``batch``      independent instances, n log-uniform in [100, 200000],
                 m=2n, |e| ~ U{2..16}, uniform pins, float32 weights.
* ``serve``      kappa log-uniform in [1e3, 1e7], |e| ~ Zipf(2) on [2,256],
                 m = kappa/7.99, n = m/2, power-law pins.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile libsynth.so next to its source (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                        _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, i32, f64, u64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_uint64
        p = ctypes.c_void_p
        lib.synth_sizes.argtypes = [i64, i32, i32, i32, f64, u64, p]
        lib.synth_sizes.restype = i64
        lib.synth_pins.argtypes = [i64, i64, p, i32, f64, i32, u64, p]
        lib.synth_pins.restype = i32
        lib.synth_weights.argtypes = [i64, u64, p]
        lib.synth_weights.restype = None
        lib.synth_loguniform.argtypes = [i64, f64, f64, u64, p]
        lib.synth_loguniform.restype = None
        lib.synth_arrivals.argtypes = [i64, f64, u64, p]
        lib.synth_arrivals.restype = None
        lib.synth_rgg.argtypes = [i64, f64, u64, p, p]
        lib.synth_rgg.restype = i64
        lib.synth_threads.argtypes = []
        lib.synth_threads.restype = i32
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


@dataclass
class Hypergraph:
    """Edge CSR: pins of edge e are pins[eoff[e]:eoff[e+1]]."""
    n: int
    m: int
    eoff: np.ndarray                 # int64[m+1]
    pins: np.ndarray                 # int32[kappa]
    weights: np.ndarray | None       # float32[m], None for unweighted inputs
    seed: int = 1                    # priority seed (used when weights is None)
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def kappa(self) -> int:
        return int(self.eoff[-1]) if self.m else 0

    @property
    def unweighted(self) -> bool:
        return self.weights is None


SIZE_UNIFORM, SIZE_ZIPF = 0, 1
PINS_UNIFORM, PINS_POWERLAW = 0, 1


def generate(n: int, m: int, *, size_dist: int = SIZE_UNIFORM, kmin: int = 2, kmax: int = 8,
             zipf_s: float = 2.0, pin_dist: int = PINS_UNIFORM, gamma: float = 2.2,
             shuffle: bool = True, weighted: bool = True, seed: int = 1,
             name: str = "") -> Hypergraph:
    lib = _load()
    eoff = np.empty(m + 1, dtype=np.int64)
    kappa = lib.synth_sizes(m, size_dist, kmin, kmax, zipf_s, seed, _ptr(eoff))
    if kappa < 0:
        raise ValueError("synth_sizes: bad size parameters")
    pins = np.empty(max(kappa, 1), dtype=np.int32)[:kappa]
    rc = lib.synth_pins(n, m, _ptr(eoff), pin_dist, gamma, int(shuffle), seed, _ptr(pins))
    if rc != 0:
        raise ValueError(f"synth_pins failed ({rc}): n must be >= the largest edge size")
    w = None
    if weighted:
        w = np.empty(m, dtype=np.float32)
        lib.synth_weights(m, seed, _ptr(w))
    return Hypergraph(n, m, eoff, pins, w, seed, name,
                      dict(size_dist=size_dist, kmin=kmin, kmax=kmax, zipf_s=zipf_s,
                           pin_dist=pin_dist, gamma=gamma, shuffle=shuffle))


def small(seed: int = 1, n: int = 10_000, m: int = 20_000) -> Hypergraph:
    return generate(n, m, kmin=2, kmax=8, seed=seed, name=f"small_n{n}_m{m}")


def large(seed: int = 1, n: int = 10_000_000, m: int = 20_000_000, kmax: int = 1024) -> Hypergraph:
    return generate(n, m, size_dist=SIZE_ZIPF, kmin=2, kmax=kmax, zipf_s=2.0,
                    pin_dist=PINS_POWERLAW, gamma=2.2, shuffle=True, seed=seed,
                    name=f"powerlaw_n{n}_m{m}")


def unweighted(seed: int = 1, n: int = 4_000_000, m: int = 8_000_000) -> Hypergraph:
    return generate(n, m, kmin=2, kmax=8, weighted=False, seed=seed, name=f"unweighted_n{n}_m{m}")


def batch_sizes(count: int = 4096, lo: float = 100, hi: float = 200_000, seed: int = 1) -> np.ndarray:
    out = np.empty(count, dtype=np.int64)
    _load().synth_loguniform(count, lo, hi, seed, _ptr(out))
    return out


def batch(count: int = 4096, lo: float = 100, hi: float = 200_000, seed: int = 1) -> list[Hypergraph]:
    """Independent instances: n log-uniform in [lo,hi], m=2n, |e| ~ U{2..16}."""
    ns = batch_sizes(count, lo, hi, seed)
    return [generate(int(n), 2 * int(n), kmin=2, kmax=16, seed=seed * 1_000_003 + i,
                     name=f"batch{i}") for i, n in enumerate(ns)]


def serve_request(kappa: int, seed: int) -> Hypergraph:
    """One serving request: |e| ~ Zipf(2) on [2,256], m = kappa/7.99, n = m/2."""
    m = max(1, int(round(kappa / 7.99)))
    n = max(256, m // 2)
    return generate(n, m, size_dist=SIZE_ZIPF, kmin=2, kmax=256, zipf_s=2.0,
                    pin_dist=PINS_POWERLAW, gamma=2.2, shuffle=True, seed=seed,
                    name=f"req{seed}")


def arrivals(count: int, rate: float, seed: int = 1) -> np.ndarray:
    out = np.empty(count, dtype=np.float64)
    _load().synth_arrivals(count, rate, seed, _ptr(out))
    return out


def from_edges(n: int, edges: list[list[int]], weights: list[float] | None,
               seed: int = 1, name: str = "") -> Hypergraph:
    """Build a Hypergraph from explicit edge lists (hand-made cases)."""
    eoff = np.zeros(len(edges) + 1, dtype=np.int64)
    for i, e in enumerate(edges):
        eoff[i + 1] = eoff[i] + len(e)
    pins = np.array([v for e in edges for v in e], dtype=np.int32)
    w = None if weights is None else np.asarray(weights, dtype=np.float32)
    return Hypergraph(n, len(edges), eoff, pins, w, seed, name)


def rgg(seed: int = 1, n: int = 1 << 23, avg_degree: float = 16.0) -> Hypergraph:
    """Random geometric graph (every edge has two pins): n points uniform in
    the unit square, an edge between points closer than r, with r chosen so
    that the expected degree is avg_degree (n * pi * r^2); float32 weights
    uniform on the 2^-24 grid of (0, 1]. The DIMACS rgg instances have
    average degree about 16."""
    lib = _load()
    r = math.sqrt(avg_degree / (math.pi * max(n, 1)))
    deg = np.empty(max(n, 1), dtype=np.int64)
    m = lib.synth_rgg(n, r, seed, _ptr(deg), None)
    if m < 0:
        raise RuntimeError(f"synth_rgg failed ({m})")
    off = np.zeros(max(n, 1), dtype=np.int64)
    np.cumsum(deg[:-1], out=off[1:])
    pins = np.empty(2 * max(int(m), 1), dtype=np.int32)
    deg[:] = off
    if lib.synth_rgg(n, r, seed, _ptr(deg), _ptr(pins)) != m:
        raise RuntimeError("synth_rgg: second pass disagrees")
    m = int(m)
    eoff = np.arange(0, 2 * m + 1, 2, dtype=np.int64)
    w = np.empty(max(m, 1), dtype=np.float32)
    lib.synth_weights(m, seed, _ptr(w))
    return Hypergraph(n, m, eoff, pins[:2 * m].copy(), w[:m].copy(), seed, f"rgg_n{n}_deg{avg_degree:g}")


def threads() -> int:
    return int(_load().synth_threads())
