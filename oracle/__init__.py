"""CPU oracle for locally-maximal hypergraph matching - TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg and
reference arm of ``bench.py`` may import this package. The CUDA path never does, and this
package never imports the CUDA path: the two share no code.

The arithmetic is in ``oracle.c`` (plain sequential C, compiled with gcc on
first use); this module only marshals numpy arrays. See the header of
``oracle.c`` for the order on edges and for which passage of the paper each
function follows.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_libs: dict[int, ctypes.CDLL] = {}


def lib_path(mutant: int = 0) -> str:
    return os.path.join(_HERE, "liboracle.so" if mutant == 0 else f"liboracle_mutant{mutant}.so")


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile the oracle (or a planted-mistake variant for the tests)."""
    out = lib_path(mutant)
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-shared", "-fPIC", "-std=c11", "-ffp-contract=off",
                        f"-DORACLE_MUTANT={mutant}", _SRC, "-o", tmp], check=True)
        os.replace(tmp, out)
    return out


def _load(mutant: int = 0) -> ctypes.CDLL:
    if mutant not in _libs:
        lib = ctypes.CDLL(build(mutant))
        i64, i32, u64, p = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p
        lib.oracle_splitmix64_first.argtypes = [u64]
        lib.oracle_splitmix64_first.restype = u64
        lib.oracle_fmix32.argtypes = [ctypes.c_uint32]
        lib.oracle_fmix32.restype = ctypes.c_uint32
        lib.oracle_key.argtypes = [p, i32, u64, i64]
        lib.oracle_key.restype = u64
        lib.oracle_splitmix64_at.argtypes = [u64, u64]
        lib.oracle_splitmix64_at.restype = u64
        lib.oracle_round_priority.argtypes = [p, i32, u64, ctypes.c_float, i64, i64]
        lib.oracle_round_priority.restype = ctypes.c_float
        lib.oracle_match.argtypes = [i64, i64, p, p, p, i32, u64, ctypes.c_float, i64, p, p, p, p, p, p]
        lib.oracle_match.restype = i32
        lib.oracle_greedy.argtypes = [i64, i64, p, p, p, i32, u64, p]
        lib.oracle_greedy.restype = i32
        lib.oracle_brute_opt.argtypes = [i64, i64, p, p, p, p]
        lib.oracle_brute_opt.restype = ctypes.c_double
        for name in ("oracle_check_disjoint", "oracle_check_maximal"):
            getattr(lib, name).argtypes = [i64, i64, p, p, p]
            getattr(lib, name).restype = i64
        lib.oracle_check_local_max.argtypes = [i64, i64, p, p, p, i32, u64, ctypes.c_float, p, p]
        lib.oracle_check_local_max.restype = i64
        _libs[mutant] = lib
    return _libs[mutant]


def _p(a: np.ndarray | None) -> int | None:
    return None if a is None else a.ctypes.data


def _inputs(h):
    eoff = np.ascontiguousarray(h.eoff, dtype=np.int64)
    pins = np.ascontiguousarray(h.pins, dtype=np.int32)
    w = None if h.weights is None else np.ascontiguousarray(h.weights, dtype=np.float32)
    return eoff, pins, w


@dataclass
class Result:
    in_matching: np.ndarray      # uint8[m]
    rounds: int
    decided_round: np.ndarray    # int32[m]
    round_stats: np.ndarray      # int64[rounds, 3]: live edges, live pins, winners
    status: int                  # 0 done, 1 round cap reached
    best_edge: np.ndarray        # int32[n]: T[v] of the last round run (-2 = none)
    matched: np.ndarray          # uint8[n]: vertex covered by M after the last round

    @property
    def edges(self) -> np.ndarray:
        return np.flatnonzero(self.in_matching).astype(np.int32)


def match(h, max_rounds: int | None = None, mutant: int = 0, noise: float = 0.0) -> Result:
    """Run the rounds on hypergraph ``h`` (a ``synth.Hypergraph``-like object
    with n, m, eoff, pins, weights (None = unweighted) and seed). noise > 0:
    priorities re-drawn before every round, amplitude `noise`."""
    lib = _load(mutant)
    eoff, pins, w = _inputs(h)
    cap = h.m + 1 if max_rounds is None else int(max_rounds)
    inm = np.zeros(max(h.m, 1), dtype=np.uint8)
    dec = np.zeros(max(h.m, 1), dtype=np.int32)
    stats = np.zeros((max(cap, 1), 3), dtype=np.int64)
    best = np.zeros(max(h.n, 1), dtype=np.int32)
    matched = np.zeros(max(h.n, 1), dtype=np.uint8)
    rounds = ctypes.c_int(0)
    rc = lib.oracle_match(h.n, h.m, _p(eoff), _p(pins), _p(w), int(w is None), h.seed, float(noise), cap,
                          _p(inm), _p(dec), _p(stats), ctypes.addressof(rounds), _p(best),
                          _p(matched))
    if rc < 0:
        raise MemoryError("oracle_match: allocation failed")
    r = rounds.value
    return Result(inm[:h.m].copy(), r, dec[:h.m].copy(), stats[:min(r, cap)].copy(), rc,
                  best[:h.n].copy(), matched[:h.n].copy())


def vertex_state(res: Result) -> np.ndarray:
    """Per-vertex state after the last round run: -1 if matched, else T[v] (-2 = none)."""
    out = res.best_edge.copy()
    out[res.matched.astype(bool)] = -1
    return out


def greedy(h, mutant: int = 0) -> np.ndarray:
    lib = _load(mutant)
    eoff, pins, w = _inputs(h)
    inm = np.zeros(max(h.m, 1), dtype=np.uint8)
    if lib.oracle_greedy(h.n, h.m, _p(eoff), _p(pins), _p(w), int(w is None), h.seed, _p(inm)) < 0:
        raise MemoryError("oracle_greedy: allocation failed")
    return inm[:h.m].copy()


def brute_opt(h) -> tuple[float, np.ndarray]:
    """Maximum matching weight by exhaustive search (n <= 64, m <= 40)."""
    eoff, pins, w = _inputs(h)
    best = np.zeros(max(h.m, 1), dtype=np.uint8)
    val = _load().oracle_brute_opt(h.n, h.m, _p(eoff), _p(pins), _p(w), _p(best))
    if val < 0:
        raise ValueError("brute_opt: input too large")
    return float(val), best[:h.m].copy()


def check_disjoint(h, in_matching) -> int:
    eoff, pins, _ = _inputs(h)
    inm = np.ascontiguousarray(in_matching, dtype=np.uint8)
    return int(_load().oracle_check_disjoint(h.n, h.m, _p(eoff), _p(pins), _p(inm)))


def check_maximal(h, in_matching) -> int:
    eoff, pins, _ = _inputs(h)
    inm = np.ascontiguousarray(in_matching, dtype=np.uint8)
    return int(_load().oracle_check_maximal(h.n, h.m, _p(eoff), _p(pins), _p(inm)))


def check_local_max(h, in_matching, decided_round, noise: float = 0.0) -> int:
    eoff, pins, w = _inputs(h)
    inm = np.ascontiguousarray(in_matching, dtype=np.uint8)
    dec = np.ascontiguousarray(decided_round, dtype=np.int32)
    return int(_load().oracle_check_local_max(h.n, h.m, _p(eoff), _p(pins), _p(w),
                                              int(w is None), h.seed, float(noise), _p(inm), _p(dec)))


def keys(h) -> np.ndarray:
    """key(e) for every edge, as uint64."""
    lib = _load()
    _, _, w = _inputs(h)
    return np.array([lib.oracle_key(_p(w), int(w is None), h.seed, e) for e in range(h.m)],
                    dtype=np.uint64)


def splitmix64_first(seed: int) -> int:
    return int(_load().oracle_splitmix64_first(seed))


def splitmix64_at(s0: int, k: int) -> int:
    return int(_load().oracle_splitmix64_at(s0, k))


def round_priority(h, noise: float, r: int, e: int) -> float:
    _, _, w = _inputs(h)
    return float(_load().oracle_round_priority(_p(w), int(w is None), h.seed, noise, r, e))


def fmix32(x: int) -> int:
    return int(_load().oracle_fmix32(x))


def weight(h, in_matching) -> float:
    """Matching weight w(M) = sum of w(e) over e in M (Sec. 2.1): the exact
    sum of the float32 weights, rounded once to the nearest float64
    (math.fsum is correctly rounded); |M| for unweighted input."""
    if h.weights is None:
        return float(int(np.count_nonzero(in_matching)))
    return math.fsum(float(x) for x in h.weights[np.asarray(in_matching, dtype=bool)])
