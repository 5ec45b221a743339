"""GB300 locally-maximal hypergraph matching: Python binding of libhm.so.

Argument marshalling only. Every step of the matching runs in the CUDA
kernels of ``libhm.so`` (built in-tree from ``csrc/`` for sm_103a); this
module passes pointers, sizes and streams through the C ABI declared in
``include/hm.h``. PyTorch provides device memory and streams. There is no
CPU fallback: if the library is missing or cannot load, every call raises.

Method: "Efficient Parallel Algorithms for Hypergraph Matching" (Sec. 3.1,
Alg. 1, Alg. 3): rounds in which every vertex takes its best live edge,
edges chosen by all their vertices join the matching, and edges touching
matched vertices are deactivated.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

HM_OK, HM_EINVAL, HM_ENOMEM, HM_ECUDA, HM_ETIMEOUT, HM_EBUSY = range(6)
STATUS_NAMES = {0: "HM_OK", 1: "HM_EINVAL", 2: "HM_ENOMEM", 3: "HM_ECUDA", 4: "HM_ETIMEOUT",
                5: "HM_EBUSY"}
HM_UNWEIGHTED, HM_BORROW_INPUT, HM_VALIDATE, HM_AUTOTUNE, HM_ONE_CLASS = 0x1, 0x2, 0x4, 0x8, 0x10
HM_VERTEX_MATCHED, HM_VERTEX_NONE = -1, -2
STAT_COLUMNS = ("active", "advance", "proposals", "winners", "winpins", "kills", "items", "next", "live", "deg",
                "ledges", "lpins")
KERNELS = ("init", "argmax", "win", "kill", "round_end")

# Every entry point of include/hm.h, in declaration order.
ENTRY_POINTS = ("hm_create", "hm_match", "hm_set_round_cap", "hm_set_noise", "hm_launch_config", "hm_autotune",
                "hm_result", "hm_result_device",
                "hm_round_stats", "hm_vertex_state", "hm_profile_match", "hm_create_ms",
                "hm_solve_host", "hm_match_noalloc", "hm_batch_create",
                "hm_batch_match", "hm_batch_result", "hm_batch_info", "hm_batch_destroy",
                "hm_server_create", "hm_server_submit", "hm_server_wait", "hm_server_stats",
                "hm_server_destroy", "hm_last_error", "hm_destroy")

LIB_PATH = _build.LIB
_lib = None


class HMError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.message = message


def build(force: bool = False) -> str:
    """Compile libhm.so (nvcc, sm_103a) if it is missing or stale."""
    return _build.build(force=force)


def lib() -> ctypes.CDLL:
    """Load libhm.so. Raises if it has not been built: no fallback exists."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libhm.so is not built ({LIB_PATH}); call "
                               "paper_2602_22976_gb300.build() first")
        L = ctypes.CDLL(LIB_PATH)
        p, i64, i32, u32, u64 = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32,
                                 ctypes.c_uint64)
        sig = {
            "hm_create": ([p, i64, i64, p, p, p, u64, u32, p], i32),
            "hm_match": ([p, p], i32),
            "hm_set_round_cap": ([p, i64], i32),
            "hm_set_noise": ([p, ctypes.c_float], i32),
            "hm_launch_config": ([p, p, p], i32),
            "hm_autotune": ([p, p, p, p], i32),
            "hm_result": ([p, p, p, p, p], i32),
            "hm_result_device": ([p, p, p], i32),
            "hm_round_stats": ([p, p, i32, p], i32),
            "hm_vertex_state": ([p, p], i32),
            "hm_profile_match": ([p, p, p, p, p, i32], i32),
            "hm_create_ms": ([p, p], i32),
            "hm_solve_host": ([i64, i64, p, p, p, u64, u32, p, p, p, p, p], i32),
            "hm_match_noalloc": ([i64, i64, p, p, p, u64, u32, p, p, p], i32),
            "hm_batch_create": ([p, i32, p, p, p, p, p, u64, u32, p], i32),
            "hm_batch_match": ([p, p], i32),
            "hm_batch_result": ([p, p, p, p, p], i32),
            "hm_batch_info": ([p, p, p, p], i32),
            "hm_batch_destroy": ([p], None),
            "hm_server_create": ([p, i32, u64], i32),
            "hm_server_submit": ([p, i64, i64, p, p, p, u64, u32, p], i32),
            "hm_server_wait": ([p, i64, p, p, p, p, p], i32),
            "hm_server_stats": ([p, p], i32),
            "hm_server_destroy": ([p], None),
            "hm_last_error": ([], ctypes.c_char_p),
            "hm_destroy": ([p], None),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def last_error() -> str:
    return lib().hm_last_error().decode()


def _check(status: int, allow=(HM_OK,)) -> int:
    if status not in allow:
        raise HMError(status, last_error())
    return status


def _stream_handle(stream) -> int | None:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


@dataclass
class Result:
    edges: np.ndarray     # int32, ascending input edge ids of the matching
    count: int
    rounds: int
    weight: float         # exact sum of the weights, rounded once to float64 (|M| if unweighted)
    status: int           # HM_OK, or HM_ETIMEOUT when a round cap stopped the loop

    @property
    def in_matching(self) -> np.ndarray:
        return self.edges


class Matcher:
    """One hypergraph resident on the GPU (an ``hm_handle``).

    eoff: int64[m+1], pins: int32[kappa], weights: float32[m] or None
    (unweighted; a seeded hash orders the edges). Torch CUDA tensors.
    """

    def __init__(self, n: int, m: int, eoff, pins, weights=None, seed: int = 1, flags: int = 0,
                 stream=None):
        self._h = None
        self.n, self.m = int(n), int(m)
        if weights is None:
            flags |= HM_UNWEIGHTED
        self.unweighted = bool(flags & HM_UNWEIGHTED)
        for name, t in (("eoff", eoff), ("pins", pins), ("weights", weights)):
            if t is not None and not t.is_contiguous():
                raise ValueError(f"{name} must be contiguous")
        h = ctypes.c_void_p()
        st = lib().hm_create(ctypes.byref(h), self.n, self.m, eoff.data_ptr(),
                             pins.data_ptr() if pins is not None and pins.numel() else None,
                             None if weights is None else weights.data_ptr(),
                             seed, flags, _stream_handle(stream))
        _check(st)
        self._h = h

    @classmethod
    def from_hypergraph(cls, hg, device: str = "cuda", stream=None) -> "Matcher":
        import torch
        eoff = torch.from_numpy(np.ascontiguousarray(hg.eoff, dtype=np.int64)).to(device)
        pins = torch.from_numpy(np.ascontiguousarray(hg.pins, dtype=np.int32)).to(device)
        w = None if hg.weights is None else torch.from_numpy(
            np.ascontiguousarray(hg.weights, dtype=np.float32)).to(device)
        torch.cuda.current_stream().synchronize()
        return cls(hg.n, hg.m, eoff, pins, w, seed=hg.seed, stream=stream)

    @property
    def handle(self) -> int:
        if self._h is None:
            raise RuntimeError("matcher is closed")
        return self._h.value

    def set_round_cap(self, cap: int) -> None:
        _check(lib().hm_set_round_cap(self.handle, int(cap)))

    def set_noise(self, amplitude: float) -> None:
        """0: fixed priority order; > 0: priorities re-drawn before every
        round with this noise amplitude (the paper's randomised rounds)."""
        _check(lib().hm_set_noise(self.handle, float(amplitude)))

    def launch_config(self, config=None) -> tuple:
        """Set (kill_chunk, argmax_bpsm, win_bpsm, kill_bpsm) if given; return the one in force."""
        get = np.zeros(4, dtype=np.int32)
        st = None if config is None else np.asarray(config, dtype=np.int32)
        _check(lib().hm_launch_config(self.handle, None if st is None else st.ctypes.data, get.ctypes.data))
        return tuple(int(x) for x in get)

    def autotune(self, stream=None) -> tuple[tuple, float]:
        cfg = np.zeros(4, dtype=np.int32)
        ms = ctypes.c_double(0.0)
        _check(lib().hm_autotune(self.handle, _stream_handle(stream), cfg.ctypes.data, ctypes.byref(ms)))
        return tuple(int(x) for x in cfg), ms.value

    def match(self, stream=None) -> None:
        _check(lib().hm_match(self.handle, _stream_handle(stream)))

    def result(self, allow=(HM_OK,)) -> Result:
        edges = np.empty(max(self.m, 1), dtype=np.int32)
        count = ctypes.c_int64(0)
        rounds = ctypes.c_int32(0)
        weight = ctypes.c_double(0.0)
        st = lib().hm_result(self.handle, edges.ctypes.data, ctypes.byref(count),
                             ctypes.byref(rounds), ctypes.byref(weight))
        _check(st, allow)
        return Result(edges[:count.value].copy(), count.value, rounds.value, weight.value, st)

    def result_device(self, out, stream=None) -> None:
        _check(lib().hm_result_device(self.handle, out.data_ptr(), _stream_handle(stream)))

    def round_stats(self) -> np.ndarray:
        buf = np.zeros((4096, len(STAT_COLUMNS)), dtype=np.int64)
        rows = ctypes.c_int32(0)
        _check(lib().hm_round_stats(self.handle, buf.ctypes.data, 4096, ctypes.byref(rows)))
        return buf[:rows.value].copy()

    def vertex_state(self) -> np.ndarray:
        out = np.empty(max(self.n, 1), dtype=np.int32)
        _check(lib().hm_vertex_state(self.handle, out.ctypes.data))
        return out[:self.n].copy()

    def profile(self, stream=None) -> dict:
        ms = np.zeros(len(KERNELS), dtype=np.float64)
        launches = np.zeros(len(KERNELS), dtype=np.int64)
        rounds = np.zeros((4096, 4), dtype=np.float64)
        _check(lib().hm_profile_match(self.handle, _stream_handle(stream), ms.ctypes.data,
                                      launches.ctypes.data, rounds.ctypes.data, 4096))
        out = {k: (float(ms[i]), int(launches[i])) for i, k in enumerate(KERNELS)}
        out["rounds_ms"] = rounds[:min(int(launches[1]), 4096)].copy()
        return out

    def create_ms(self) -> dict:
        ms = np.zeros(5, dtype=np.float64)
        _check(lib().hm_create_ms(self.handle, ms.ctypes.data))
        return dict(zip(("validate", "order", "relabel", "vertex_csr", "total"), ms.tolist()))

    def close(self) -> None:
        if self._h is not None and _lib is not None:
            _lib.hm_destroy(self._h)
        self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent hypergraphs matched by one graph launch (hm_batch_*).

    hgs: sequence of synth.Hypergraph-like objects (all weighted or all
    unweighted, one seed). Inputs are concatenated and copied to the device.
    """

    def __init__(self, hgs, autotune: bool = False, stream=None, device: str = "cuda", one_class: bool = False):
        import torch
        self._b = None
        self.count = len(hgs)
        self.n = np.array([h.n for h in hgs], dtype=np.int64)
        self.m = np.array([h.m for h in hgs], dtype=np.int64)
        weighted = hgs[0].weights is not None
        if any((h.weights is not None) != weighted for h in hgs):
            raise ValueError("a batch is all weighted or all unweighted")
        eoff = torch.from_numpy(np.concatenate([np.asarray(h.eoff, np.int64) for h in hgs])).to(device)
        pins = torch.from_numpy(np.concatenate([np.asarray(h.pins, np.int32) for h in hgs])).to(device)
        w = None
        if weighted:
            w = torch.from_numpy(np.concatenate([np.asarray(h.weights, np.float32) for h in hgs])).to(device)
        torch.cuda.current_stream().synchronize()
        flags = ((0 if weighted else HM_UNWEIGHTED) | (HM_AUTOTUNE if autotune else 0)
                 | (HM_ONE_CLASS if one_class else 0))
        b = ctypes.c_void_p()
        st = lib().hm_batch_create(ctypes.byref(b), self.count, self.n.ctypes.data, self.m.ctypes.data,
                                   eoff.data_ptr(), pins.data_ptr() if pins.numel() else None,
                                   None if w is None else w.data_ptr(), hgs[0].seed, flags,
                                   _stream_handle(stream))
        _check(st)
        self._b = b

    @property
    def handle(self) -> int:
        if self._b is None:
            raise RuntimeError("batch is closed")
        return self._b.value

    def match(self, stream=None) -> None:
        _check(lib().hm_batch_match(self.handle, _stream_handle(stream)))

    def result(self, allow=(HM_OK,)):
        """Per instance: (edges int32 local ids, count, rounds, weight)."""
        edges = np.empty(max(int(self.m.sum()), 1), dtype=np.int32)
        counts = np.zeros(self.count, dtype=np.int64)
        rounds = np.zeros(self.count, dtype=np.int32)
        weights = np.zeros(self.count, dtype=np.float64)
        st = lib().hm_batch_result(self.handle, edges.ctypes.data, counts.ctypes.data,
                                   rounds.ctypes.data, weights.ctypes.data)
        _check(st, allow)
        offs = np.concatenate([[0], np.cumsum(counts)])
        return [Result(edges[offs[i]:offs[i + 1]].copy(), int(counts[i]), int(rounds[i]),
                       float(weights[i]), st) for i in range(self.count)]

    def info(self) -> tuple[int, np.ndarray, np.ndarray]:
        ncls = ctypes.c_int32(0)
        _check(lib().hm_batch_info(self.handle, ctypes.byref(ncls), None, None))
        cls = np.zeros(self.count, dtype=np.int32)
        cfg = np.zeros((ncls.value, 4), dtype=np.int32)
        _check(lib().hm_batch_info(self.handle, None, cls.ctypes.data, cfg.ctypes.data))
        return ncls.value, cls, cfg

    def close(self) -> None:
        if self._b is not None and _lib is not None:
            _lib.hm_batch_destroy(self._b)
        self._b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


SERVER_STATS = ("completed", "queued", "inflight", "peak_inflight", "reserved_bytes",
                "peak_reserved_bytes", "budget_bytes", "groups", "peak_group")


class Server:
    """hm_server: requests from host arrays, continuous batching on the GPU."""

    def __init__(self, slots: int = 4, hbm_budget_bytes: int = 0):
        self._s = None
        self._keep: dict[int, tuple] = {}
        s = ctypes.c_void_p()
        _check(lib().hm_server_create(ctypes.byref(s), int(slots), int(hbm_budget_bytes)))
        self._s = s

    @property
    def handle(self) -> int:
        if self._s is None:
            raise RuntimeError("server is closed")
        return self._s.value

    def submit(self, hg, arrays=None) -> int:
        """Queue hypergraph `hg`; `arrays` = (eoff, pins, weights) host arrays to
        use instead of hg's (e.g. pinned). They are kept alive until wait()."""
        if arrays is None:
            arrays = (np.ascontiguousarray(hg.eoff, np.int64), np.ascontiguousarray(hg.pins, np.int32),
                      None if hg.weights is None else np.ascontiguousarray(hg.weights, np.float32))
        ptr = lambda a: None if a is None else (a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data)
        eoff, pins, w = arrays
        flags = HM_UNWEIGHTED if w is None else 0
        t = ctypes.c_int64(0)
        _check(lib().hm_server_submit(self.handle, hg.n, hg.m, ptr(eoff), ptr(pins), ptr(w), hg.seed,
                                      flags, ctypes.byref(t)))
        self._keep[t.value] = (arrays, hg.m)
        return t.value

    def wait(self, ticket: int, allow=(HM_OK,)) -> tuple[Result, float]:
        arrays, m = self._keep.pop(ticket)
        edges = np.empty(max(m, 1), dtype=np.int32)
        count = ctypes.c_int64(0)
        rounds = ctypes.c_int32(0)
        weight = ctypes.c_double(0.0)
        lat = ctypes.c_double(0.0)
        st = lib().hm_server_wait(self.handle, ticket, edges.ctypes.data, ctypes.byref(count),
                                  ctypes.byref(rounds), ctypes.byref(weight), ctypes.byref(lat))
        _check(st, allow)
        return Result(edges[:count.value].copy(), count.value, rounds.value, weight.value, st), lat.value

    def stats(self) -> dict:
        out = np.zeros(len(SERVER_STATS), dtype=np.int64)
        _check(lib().hm_server_stats(self.handle, out.ctypes.data))
        return dict(zip(SERVER_STATS, out.tolist()))

    def close(self) -> None:
        if self._s is not None and _lib is not None:
            _lib.hm_server_destroy(self._s)
        self._s = None
        self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_host(hg, stream=None, allow=(HM_OK,)) -> Result:
    """hm_solve_host: HOST arrays in, HOST result out (copies inside the call)."""
    eoff = np.ascontiguousarray(hg.eoff, dtype=np.int64)
    pins = np.ascontiguousarray(hg.pins, dtype=np.int32)
    flags = 0
    w = None
    if hg.weights is None:
        flags |= HM_UNWEIGHTED
    else:
        w = np.ascontiguousarray(hg.weights, dtype=np.float32)
    edges = np.empty(max(hg.m, 1), dtype=np.int32)
    count = ctypes.c_int64(0)
    rounds = ctypes.c_int32(0)
    weight = ctypes.c_double(0.0)
    st = lib().hm_solve_host(hg.n, hg.m, eoff.ctypes.data, pins.ctypes.data if pins.size else None,
                             None if w is None else w.ctypes.data, hg.seed, flags,
                             edges.ctypes.data, ctypes.byref(count), ctypes.byref(rounds),
                             ctypes.byref(weight), _stream_handle(stream))
    _check(st, allow)
    return Result(edges[:count.value].copy(), count.value, rounds.value, weight.value, st)


def solve_host_ptrs(n: int, m: int, eoff_ptr: int, pins_ptr: int, w_ptr: int | None, seed: int,
                    flags: int, edges_ptr: int, stream_handle: int | None):
    """hm_solve_host on raw host pointers (pinned buffers for the end-to-end timing)."""
    count = ctypes.c_int64(0)
    rounds = ctypes.c_int32(0)
    weight = ctypes.c_double(0.0)
    st = lib().hm_solve_host(n, m, eoff_ptr, pins_ptr, w_ptr, seed, flags, edges_ptr,
                             ctypes.byref(count), ctypes.byref(rounds), ctypes.byref(weight),
                             stream_handle)
    _check(st)
    return count.value, rounds.value, weight.value
