#!/usr/bin/env python3
"""Benchmark of the GPU matching loop (libhm.so) on the large power-law
hypergraph: n=10M vertices, m=20M edges, |e| ~ Zipf(2) on [2,1024], vertex
degrees power-law (gamma=2.2), float32 weights in (0,1], kappa ~ 2.02e8.

One step = one hm_match (the whole round loop, all three kernels of every
round, as one CUDA graph) on inputs already resident in HBM.

  value        kappa * rounds * steps / device time      (pins/s, whole job)
  ms_per_step  time to maximal matching (CUDA events on the launching stream)
  e2e          same metric through hm_solve_host from pinned HOST buffers:
               H2D copies, hm_create, hm_match, result D2H inside the timing
  roofline     dominant kernel: algorithmic bytes / its CUDA-event time, from
               a replay with one event pair per kernel launch (hm_profile_match)
  cpu_baseline the CPU oracle (single thread) on the same instance

--impl reference runs the CPU oracle (the reference of this project) on a
bounded sample of the same workload and prints the same JSON line.
Multi-GPU: independent replicas, one instance per rank (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "large": dict(desc="powerlaw hypergraph n=10M m=20M |e|~Zipf(2)[2,1024] gamma=2.2 f32 w in (0,1]",
                  make=lambda seed, sc=1: __import__("synth").large(seed=seed, n=10_000_000 // sc,
                                                                    m=20_000_000 // sc),
                  sample=lambda seed: __import__("synth").large(seed=seed, n=50_000, m=100_000)),
    "small": dict(desc="uniform hypergraph n=10k m=20k |e|~U{2..8} f32 w in (0,1]",
                  make=lambda seed, sc=1: __import__("synth").small(seed=seed, n=10_000 // sc,
                                                                    m=20_000 // sc),
                  sample=lambda seed: __import__("synth").small(seed=seed)),
    "unweighted": dict(desc="uniform hypergraph n=4M m=8M |e|~U{2..8} unweighted, hash priority",
                       make=lambda seed, sc=1: __import__("synth").unweighted(seed=seed, n=4_000_000 // sc,
                                                                              m=8_000_000 // sc),
                       sample=lambda seed: __import__("synth").unweighted(seed=seed, n=40_000, m=80_000)),
}
WORKLOADS["graph"] = dict(
    desc="random geometric graph (DIMACS rgg class) n=2^23 avg degree 16, d=2, f32 w in (0,1]",
    make=lambda seed, sc=1: __import__("synth").rgg(seed=seed, n=(1 << 23) // sc),
    sample=lambda seed: __import__("synth").rgg(seed=seed, n=100_000))
WORKLOADS["batch"] = dict(
    desc="4096 independent hypergraphs, n log-uniform in [100, 200000], m=2n, |e|~U{2..16}, f32 w",
    make=None, sample=lambda seed: __import__("synth").batch(64, seed=seed))
WORKLOADS["serve"] = dict(
    desc="Poisson request stream, kappa log-uniform in [1e3,1e7], |e|~Zipf(2)[2,256], f32 w, "
         "admitted by free HBM",
    make=None, sample=lambda seed: [__import__("synth").serve_request(k, seed=seed * 1000 + i)
                                    for i, k in enumerate([3000, 30000, 300000])])
METRIC = "pins/s (kappa*rounds/time)"
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 400 matches; 20 batch launches; 10 oracle runs for --impl reference)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=tuple(WORKLOADS), default="large")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--e2e-steps", type=int, default=10,
                    help="end-to-end calls timed one by one after two untimed ones; the median is reported")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true",
                    help="default workload: leave out the batch sub-object (the batching workload at full size)")
    ap.add_argument("--no-serve", action="store_true",
                    help="default workload: leave out the serve sub-object (short serving runs)")
    ap.add_argument("--no-plain", action="store_true",
                    help="batch workload: skip the one-hm_match-per-instance comparison")
    ap.add_argument("--one-class", action="store_true",
                    help="batch workload: every instance in one union (HM_ONE_CLASS) instead of size classes")
    ap.add_argument("--scale", type=int, default=1,
                    help="divide n and m of the workload (smaller cases for profiler captures)")
    ap.add_argument("--noise", type=float, default=0.0,
                    help="> 0: the paper's re-randomised rounds with this noise amplitude "
                         "(priorities drawn again before every round); 0: fixed order")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 10 if args.impl == "reference" else (20 if args.workload == "batch" else 400)
    return args


# ------------------------------------------------------------------ helpers

def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def replica_seed(seed: int, rank: int) -> int:
    """Instance seed of a rank: every replica matches its own hypergraph."""
    return seed + 1000 * rank


def replica_totals(units: float, t_ms: float, world: int, device: str = "cuda") -> tuple:
    """Whole-job work and time over independent replicas: the units all ranks
    processed and the slowest rank's time (one SUM and one MAX reduction of
    two host numbers; nothing on the matching path is exchanged)."""
    if world <= 1:
        return units, t_ms
    import torch
    import torch.distributed as dist
    u = torch.tensor([units], dtype=torch.float64, device=device)
    t = torch.tensor([t_ms], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()), float(t.item())


class Clocks:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)], stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(", ") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons, power = [], [], set(), []
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                power.append(float(r[3]))
                for name, val in zip(names, r[5:9]):
                    if val.strip().lower() == "active":
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def kernel_bytes(stats: np.ndarray, n: int, m: int, kappa: int = 0, random: bool = False,
                 p16: bool = True, pairs: bool = False) -> dict:
    """Element bytes of this design per kernel kind, summed over rounds, from
    the per-round counters of hm_round_stats. p16: the fixed order's P
    counters are 16 bits wide (every edge has at most 65535 pins). pairs: a
    graph (fixed order: lists of {edge, other endpoint}, liveness from the
    endpoints' matched flags, no kill step; re-randomised rounds: the same
    edge rounds as a hypergraph, with two pins an edge)."""
    ACT, ADV, PROP, WIN, WPIN, KILL, ITEM, NEXT, LIVE = range(9)
    LEDGES = 10
    pc = 2 if p16 else 4  # bytes of one P counter
    if random:  # flag, counter word read + write, mask; matched flag, two key slots
        init = float(m * (1 + 4 + 4 + 1) + n * (1 + 8 + 8))
    elif pairs:  # mask, P copied from its initial copy; matched flags
        init = float(m * (1 + 2 * pc) + n)
    else:       # flag, mask, P copied from its initial copy (read + write)
        init = float(m * (1 + 1 + 2 * pc))
    b = {"init": init, "argmax": 0.0, "win": 0.0, "kill": 0.0, "round_end": 0.0}
    if random:
        for r, row in enumerate(stats):
            row = row.astype(np.float64)
            if r == 0:
                # round 1, vertex-driven: every list entry; per vertex its offsets
                # and largest key written; proposal = key read, record write,
                # counter word read + write; winner = its id
                b["argmax"] += (row[ADV] * 8 + n * (8 + 8) + row[PROP] * (8 + 8 + 4 + 4) + row[WIN] * 4)
                if pairs:  # winner: order, mask; winner pin: pin, matched flag
                    b["win"] += row[WIN] * (4 + 1 + 4) + row[WPIN] * (4 + 1)
                else:      # winner: offset pair, order, mask; winner pin: pin, record
                           # read + write; kill range: item write
                    b["win"] += row[WIN] * (16 + 4 + 1 + 4) + row[WPIN] * (4 + 16 + 8) + row[ITEM] * 8
                b["kill"] += row[ITEM] * 8 + row[KILL] * (8 + 1)  # killed entry: list entry + flag
                continue
            # an edge round: records in (round 2: every edge, hypergraphs read its
            # live flag; later: the previous round's live edges), a tested pin
            # (pin + matched flag), a live edge's record written and its pins'
            # 8-byte offers; the win pass reads each live record, pin and slot,
            # marks winners (mask) and their pins (flag), and clears the other
            # slot buffer (8 n)
            rec_in = m if r == 1 else float(stats[r - 1, LEDGES])
            flag = m if (r == 1 and not pairs) else 0
            tested = 0.0 if (r == 1 and not pairs) else row[ADV]
            b["argmax"] += (rec_in * 16 + flag + tested * (4 + 1) + row[LEDGES] * 16
                            + row[LIVE] * ((4 if tested == 0 else 0) + 8))
            b["win"] += (row[LEDGES] * 16 + row[LIVE] * (4 + 8) + row[WIN] + row[WPIN]
                         + (n * 8 if row[LIVE] > 0 else 0))
        return b
    for r, row in enumerate(stats):
        row = row.astype(np.float64)
        if pairs:  # winner: order, mask; winner pin: pin, matched flag
            winb = row[WIN] * (4 + 1) + row[WPIN] * (4 + 1)
        else:  # winner: offset pair, order, mask; winner pin: pin, record read +
               # write; kill range: item write
            winb = row[WIN] * (16 + 4 + 1) + row[WPIN] * (4 + 16 + 8) + row[ITEM] * 8
        if pairs:
            if r == 0:  # first entry + its other endpoint + offset pair read, record write
                b["argmax"] += row[ACT] * (4 + 4 + 16 + 16) + row[PROP] * 2 * pc + row[NEXT] * 4
            else:       # list + record + matched flag; skipped entry = pair + flag;
                        # proposal = record write + P read+write; kept vertex = list write
                b["argmax"] += (row[ACT] * (4 + 16 + 1) + row[ADV] * (8 + 1)
                                + row[PROP] * (16 + 2 * pc) + row[NEXT] * 4)
            b["argmax"] += row[WIN] * (4 + 4 + 4)  # winner staged, read, listed
        else:
            if r == 0:  # first entry read + record (T, cursor) write; proposal =
                        # P read+write; kept vertex = list write
                b["argmax"] += row[ACT] * (4 + 8) + row[PROP] * 2 * pc + row[NEXT] * 4
            else:       # list + record + live flag; skipped entry = entry + flag;
                        # proposal = record write + P read+write; kept vertex = list write
                b["argmax"] += (row[ACT] * (4 + 16 + 1) + row[ADV] * (4 + 1)
                                + row[PROP] * (8 + 2 * pc) + row[NEXT] * 4)
            b["argmax"] += row[WIN] * (4 + 4 + 4)  # winner staged, read, listed
        b["win"] += winb + row[WIN] * 4  # the winner list
        # kill range read; killed entry: entry + flag
        b["kill"] += row[ITEM] * 8 + row[KILL] * (4 + 1)
    return b


def method_argmax_bytes(stats: np.ndarray) -> float:
    """Bytes of the method's argmax step (a1) summed over rounds, by the
    per-unit figures of the plain formulation, in which every active vertex
    takes the maximum over its whole list each round: an active vertex moves
    24 bytes (list slot 4, offset pair 16, best 4) and every list entry of an
    active vertex 8 (entry 4, gathered priority-or-dead word 4). Units from
    hm_round_stats: the active vertices of round r (HM_STAT_NEXT) and the sum
    of their degrees (HM_STAT_DEG). The fixed order resumes each vertex at its
    cursor, and the re-randomised rounds from the second on touch only the
    pins of live edges, so the kernels move fewer bytes than this count."""
    NEXT, DEG = 7, 9
    s = stats.astype(np.float64)
    return float(s[:, NEXT].sum() * 24 + s[:, DEG].sum() * 8)


def method_match_bytes(stats: np.ndarray) -> dict:
    """Bytes of the method's steps a1-a4 summed over rounds, by the per-unit
    figures of the plain formulation (every active vertex takes the maximum
    over its whole list, every live edge tests all its pins, every live edge
    is checked against the matched flags, both lists are compacted):
      a1  24 B per active vertex U_r + 8 B per list entry of an active vertex
      a2  24 B per live edge A_r (list slot 4, offset pair 16, priority 4)
          + 8 B per live pin pi_r (pin 4, gathered best 4)
          + 1 B per pin of a winner (matched flag) + 1 B per winner (mask)
      a3  5 B per live pin (pin 4, gathered matched flag 1) + 4 B per live
          edge (priority-or-dead write)
      a4  8 B per live edge and per active vertex (list read 4, write 4)
    Units from hm_round_stats: U_r = HM_STAT_NEXT, sum of their degrees =
    HM_STAT_DEG, A_r = HM_STAT_LEDGES, pi_r = HM_STAT_LPINS (the last three
    filled by the per-kernel replay), winners and their pins."""
    WIN, WPIN, NEXT, DEG, LED, LPI = 3, 4, 7, 9, 10, 11
    s = stats.astype(np.float64)
    a1 = s[:, NEXT].sum() * 24 + s[:, DEG].sum() * 8
    a2 = s[:, LED].sum() * 24 + s[:, LPI].sum() * 8 + s[:, WPIN].sum() + s[:, WIN].sum()
    a3 = s[:, LPI].sum() * 5 + s[:, LED].sum() * 4
    a4 = (s[:, LED].sum() + s[:, NEXT].sum()) * 8
    return {"a1": float(a1), "a2": float(a2), "a3": float(a3), "a4": float(a4),
            "total": float(a1 + a2 + a3 + a4)}


def timed_calls(call, k: int):
    """End-to-end calls through the public API: two untimed ones, then k
    timed one by one on the host clock (each ends with its result on the
    host and a device synchronisation). Returns the median seconds, every
    call's milliseconds and the last call's result."""
    import torch
    sync = torch.cuda.synchronize if torch.cuda.is_available() else (lambda: None)
    for _ in range(2):
        call()
    sync()
    ts, out = [], None
    for _ in range(max(k, 1)):
        t0 = time.perf_counter()
        out = call()
        sync()
        ts.append(time.perf_counter() - t0)
    return float(np.median(ts)), [round(t * 1e3, 3) for t in ts], out


def random_access_roofline(stats: np.ndarray, prof: dict, ra: dict, random: bool) -> dict | None:
    """The round kernels are bound by random single-element accesses, not by
    bytes: a lower bound on each kernel's time is its random accesses at this
    GPU's measured rates (probe_random_access: 1-byte loads, 1-byte
    stores, returning 4-byte atomics). frac = that bound / the kernel's time.
    Counted from hm_round_stats, fixed order only: k_argmax does one live-flag
    load per active vertex and per skipped entry from round 2 on and one
    returning atomic per proposal; k_kill stores every target in round 1 and
    loads every target's flag from round 2 on (the stores to the live ones
    are left out, so its bound is low)."""
    if random:
        return None
    ACT, ADV, PROP = 0, 1, 2
    KILL = 5
    s = stats.astype(np.float64)
    loads = float(s[1:, ACT].sum() + s[1:, ADV].sum())
    atoms = float(s[:, PROP].sum())
    k_loads = float(s[1:, KILL].sum())
    k_stores = float(s[:1, KILL].sum())
    out = {}
    for name, t_ms, bound in (
            ("argmax", prof["argmax"][0], loads / (ra["load1B"] * 1e9) + atoms / (ra["atomic4B"] * 1e9)),
            ("kill", prof["kill"][0], k_loads / (ra["load1B"] * 1e9) + k_stores / (ra["store1B"] * 1e9))):
        out[name] = {"bound_ms": bound * 1e3, "ms": t_ms, "frac": bound * 1e3 / t_ms if t_ms > 0 else None}
    out["note"] = ("time of each kernel's random flag loads, stores and atomics at the measured random-access "
                   "rates, over its measured time")
    return out


# kernel step of the bench line -> (kernel name in profiles/traffic.json, its source file)
TRAFFIC_ROWS = {
    ("init", False): ("k_init", "rounds.cu"),
    ("argmax", False): ("k_argmax", "rounds.cu"),
    ("win", False): ("k_win", "rounds.cu"),
    ("kill", False): ("k_kill", "rounds.cu"),
    ("init", True): ("k_rinit", "rrounds.cu"),
    ("argmax", True): ("k_rflat+k_rpropose+k_epush", "rrounds.cu"),
    ("win", True): ("k_win+k_ewin", "rrounds.cu"),
    ("kill", True): ("k_kill", "rounds.cu"),
}
TRAFFIC_FILE = os.path.join("profiles", "traffic.json")


def kernel_source_hash(source: str = "rounds.cu") -> str:
    """Hash of a kernel source file: a stored ncu traffic figure is only
    valid for the kernel version it was measured on."""
    import hashlib
    p = os.path.join(ROOT, "paper_2602_22976_gb300", "csrc", source)
    with open(p, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def traffic_row(step: str, randomised: bool, workload: str = "large") -> dict | None:
    """The committed ncu row (profiles/traffic.json) of a kernel step, when it
    was measured on this source, in this mode (fixed order / re-randomised
    rounds) and on this workload; else None."""
    p = os.path.join(ROOT, TRAFFIC_FILE)
    if (step, randomised) not in TRAFFIC_ROWS or not os.path.exists(p):
        return None
    name, source = TRAFFIC_ROWS[(step, randomised)]
    want = kernel_source_hash(source)
    mode = "re-randomised" if randomised else "fixed"
    with open(p) as f:
        rows = json.load(f)["rows"]
    best = None
    for r in rows:
        if r["kernel"] == name and r["mode"] == mode and r["workload"] == workload and r["source_hash"] == want:
            if best is None or r.get("scale", 1) < best.get("scale", 1):  # a full-size capture first
                best = r
    return best


def measured_traffic(step: str, randomised: bool, workload: str = "large",
                     design_per_launch: float | None = None) -> float | None:
    """DRAM bytes per launch of a kernel step at the bench's size, from the
    committed ncu row. A row captured on a smaller instance (scale s > 1:
    n and m divided by s) is scaled to the bench's size by the units the
    kernel processes: its measured bytes times the ratio of this design's
    element bytes per launch at the bench's size (design_per_launch) to those
    of the captured run (the row's design_bytes_per_launch). Without that
    ratio a scaled row reads as None."""
    r = traffic_row(step, randomised, workload)
    if r is None:
        return None
    b = float(r["bytes_per_launch"])
    if r.get("scale", 1) == 1:
        return b
    if not design_per_launch or not r.get("design_bytes_per_launch"):
        return None
    return b * design_per_launch / float(r["design_bytes_per_launch"])


PROBES = ("store1B", "load1B", "load4B", "red4B", "atomic4B")


def probe_random_access(array_bytes: int, ops: int = 200_000_000, stream_handle: int | None = None) -> dict:
    """Random single-element access rates of this GPU (1e9 per second), from
    the benchmark's own probe library (libhmprobe.so, built beside libhm.so
    but not part of it)."""
    import ctypes
    import importlib
    L = ctypes.CDLL(importlib.import_module("paper_2602_22976_gb300.build").build_probe())
    L.hmprobe_random_access.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]
    L.hmprobe_random_access.restype = ctypes.c_int
    L.hmprobe_last_error.restype = ctypes.c_char_p
    out = np.zeros(len(PROBES), dtype=np.float64)
    rc = L.hmprobe_random_access(int(array_bytes), int(ops), out.ctypes.data, stream_handle)
    if rc != 0:
        raise RuntimeError(f"random-access probe failed ({rc}): {L.hmprobe_last_error().decode()}")
    return dict(zip(PROBES, out.tolist()))


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def cpu_cores_used() -> int:
    return 1


def host_cpu() -> dict:
    """The host the CPU baselines run on: its core count and CPU model."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None and os.path.exists("/proc/cpuinfo"):
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                model = line.split(":", 1)[1].strip()
                break
    import platform
    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": platform.machine()}


# The paper's own headline (other hardware, its real-world instances and its
# re-randomised rounds): printed beside the numbers as context only.
PAPER_CONTEXT = {
    "claim": "up to 76.6x speedup of the CUDA implementation (HLM:C) over single-core sequential Greedy",
    "range": "3.20x to 76.6x across the paper's hypergraph categories",
    "hardware": "NVIDIA RTX 4090 (GPU) vs one core of an Intel Xeon w5-3435X",
    "where": "Sec. 5.2",
    "note": "other hardware, other instances and per-round random weights: context, not a target",
}


# ------------------------------------------------------------------ reference arm

def run_reference(args, world, rank):
    """The CPU oracle (this project's reference) on this machine's host cores, on
    the bench's own instance (the full workload where it has one; the batch
    and serve workloads use a sample of their generator), one oracle run per
    step. Under torchrun only rank 0 runs it."""
    if rank != 0:
        return
    import oracle
    wl = WORKLOADS[args.workload]
    full = wl["make"] is not None
    hs = wl["make"](args.seed, args.scale) if full else wl["sample"](args.seed)
    hs = hs if isinstance(hs, list) else [hs]
    oracle.build()
    for _ in range(args.warmup):
        for h in hs:
            oracle.match(h, noise=args.noise)
    t0 = time.perf_counter()
    units = 0
    for _ in range(args.steps):
        units = sum(h.kappa * oracle.match(h, noise=args.noise).rounds for h in hs)
    dt = time.perf_counter() - t0
    value = units * args.steps / dt if dt > 0 else 0.0
    if full:
        sample = (f"the bench's own instance{f' scaled 1/{args.scale}' if args.scale > 1 else ''} "
                  f"(kappa={hs[0].kappa}), one oracle run per step")
    else:
        sample = (f"{len(hs)} instances of the {args.workload} generator, kappa={sum(h.kappa for h in hs)}, "
                  f"one oracle run of each per step")
    desc = wl["desc"] + (f" scaled 1/{args.scale}" if full and args.scale > 1 else "")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "pins/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic", "config": {"workload": desc, "sample": sample, "noise": args.noise,
                                        "same_instance_as_gpu_arm": full},
        "cpu_baseline": {"value": value, "unit": "pins/s", "cores": cpu_cores_used(),
                         "kind": "oracle", "sample": sample, "host": host_cpu()},
        "e2e": {"value": value, "unit": "pins/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "paper_context": PAPER_CONTEXT,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ batched arm

def measure_batch(seed: int, count: int, steps: int, warmup: int, one_class: bool = False,
                  plain: bool = True, stream=None) -> dict:
    """The batching workload: `count` independent instances in one
    hm_batch_match (one graph launch, autotuned size classes), timed with
    CUDA events over `steps` launches; then the same instances as one handle
    and one hm_match each (the plain per-instance launch), all launched back
    to back on the same stream and timed the same way. Results of the two
    paths are compared instance by instance."""
    import torch
    import synth
    import paper_2602_22976_gb300 as hm
    stream = stream or torch.cuda.current_stream()
    t0 = time.perf_counter()
    hs = synth.batch(count, seed=seed)
    for h in hs:
        h.seed = 1
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    b = hm.Batch(hs, autotune=True, one_class=one_class)
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t0
    for _ in range(max(warmup, 3)):
        b.match(stream)
    res = b.result()
    units_step = float(sum(h.kappa * r.rounds for h, r in zip(hs, res)))
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    torch.cuda.synchronize()
    for k in range(steps):
        starts[k].record(stream)
        b.match(stream)
        ends[k].record(stream)
    torch.cuda.synchronize()
    step_ms = [x.elapsed_time(y) for x, y in zip(starts, ends)]
    t_ms = float(sum(step_ms))
    ncls, cls, cfg = b.info()
    b.close()
    plain_out = None
    if plain:
        t0 = time.perf_counter()
        mts = [hm.Matcher.from_hypergraph(h) for h in hs]
        t_plain_create = time.perf_counter() - t0
        for mt in mts:
            mt.match(stream)
        torch.cuda.synchronize()
        reps = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for mt in mts:
                mt.match(stream)
            e1.record(stream)
            torch.cuda.synchronize()
            reps.append(e0.elapsed_time(e1))
        same = True
        for mt, r in zip(mts, res):
            rr = mt.result()
            same = same and rr.rounds == r.rounds and np.array_equal(rr.edges, r.edges)
            mt.close()
        plain_ms = statistics.median(reps)
        plain_out = {"ms": plain_ms, "ms_runs": reps, "value": units_step / (plain_ms / 1e3), "unit": "pins/s",
                     "launches": f"{count} hm_match graph launches back to back on one stream",
                     "create_s": t_plain_create, "same_results_as_batch": bool(same),
                     "batched_speedup": plain_ms / (t_ms / steps)}
    return {
        "value": units_step * steps / (t_ms / 1e3), "unit": "pins/s", "steps": steps,
        "ms_per_launch": t_ms / steps,
        "time_to_matching_ms": {"median": statistics.median(step_ms), "mean": t_ms / steps,
                                "p99": float(np.percentile(step_ms, 99))},
        "instances": count, "instances_per_s": count * steps / (t_ms / 1e3),
        "sum_kappa": int(sum(h.kappa for h in hs)), "sum_n": int(sum(h.n for h in hs)),
        "units_per_launch": units_step, "size_classes": int(ncls), "class_launch_configs": cfg.tolist(),
        "classes": "one union (HM_ONE_CLASS)" if one_class else "size classes by kappa (factors of 4)",
        "create_s": t_create, "generate_s": t_gen, "plain_per_instance": plain_out,
    }


def run_batch(args, world, rank, local):
    """One step = one hm_batch_match over all instances (one graph launch);
    compared with one hm_match per instance on the same GPU."""
    import torch
    import paper_2602_22976_gb300 as hm

    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    hm.build()
    count = max(1, 4096 // args.scale)
    clocks = Clocks(local)
    if world > 1:
        dist.barrier()
    clocks.start()
    r = measure_batch(replica_seed(args.seed, rank), count, args.steps, args.warmup, args.one_class,
                      plain=not args.no_plain)
    clk = clocks.stop()
    units_all, t_max = replica_totals(r["units_per_launch"] * args.steps, r["ms_per_launch"] * args.steps, world)
    out = {
        "metric": METRIC, "value": units_all / (t_max / 1e3), "unit": "pins/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": WORKLOADS["batch"]["desc"] + (f" ({count} instances)" if count != 4096 else ""),
                   "l2": "inputs larger than L2", "parallelism": f"replicas x{world}"},
        "batch": r, "clocks": clk, "cpu_baseline": None, "e2e": None,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# ------------------------------------------------------------------ serving arm

def serve_pool(seed: int, scale: int = 1):
    import torch
    import synth
    rng = np.random.default_rng(seed)
    pool_n = max(8, 128 // scale)
    kap = np.exp(rng.uniform(np.log(1e3), np.log(1e7 / scale), size=pool_n)).astype(np.int64)
    pool = [synth.serve_request(int(k), seed=seed * 100_000 + i) for i, k in enumerate(kap)]
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    arrays = [(pin(h.eoff), pin(h.pins), pin(h.weights)) for h in pool]
    return pool, arrays, kap


def measure_serve(seed: int, rates, count_for, scale: int = 1, slots: int = 8, arrival_seed: int = 1) -> dict:
    """Requests drawn from a pool of serving-shaped hypergraphs arrive as a
    Poisson stream at each rate and go through hm_server (continuous
    batching); latency = submit -> done. Then the whole stream at once,
    served with `slots` slots against one slot (one request at a time, each
    through the hm_solve_host path)."""
    import paper_2602_22976_gb300 as hm
    import synth
    pool, arrays, kap = serve_pool(seed, scale)
    pool_n = len(pool)
    units = []  # kappa * rounds of every pool request (from a solo run)
    for h in pool:
        r = hm.solve_host(h)
        units.append(h.kappa * r.rounds)

    def run(rate, count, nslots):
        arr = synth.arrivals(count, rate, seed=arrival_seed + int(min(rate, 1e6)))
        with hm.Server(slots=nslots) as srv:
            t0 = time.perf_counter()
            tickets = []
            for i, ta in enumerate(arr):
                while time.perf_counter() - t0 < ta:
                    pass
                k = i % pool_n
                tickets.append((k, srv.submit(pool[k], arrays[k])))
            lat = []
            for k, t in tickets:
                r, ms = srv.wait(t)
                lat.append(ms)
            wall = time.perf_counter() - t0
            st = srv.stats()
        work = float(sum(units[k] for k, _ in tickets))
        return {"rate_req_s": rate, "requests": count, "slots": nslots,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "pins_per_s": work / wall, "req_per_s": count / wall, "work": work, "wall_s": wall,
                "peak_inflight": st["peak_inflight"], "peak_reserved_gb": st["peak_reserved_bytes"] / 1e9}

    sweep = [run(rate, max(16, count_for(rate) // max(1, scale)), slots) for rate in rates]
    served = run(1e9, 2 * pool_n, slots)
    serial = run(1e9, 2 * pool_n, 1)
    # the plain form: the same 2 * pool requests one at a time, each one
    # hm_solve_host call from its pinned host buffers to its host result
    import torch
    sh = torch.cuda.current_stream().cuda_stream or None
    edges = torch.empty(max(h.m for h in pool), dtype=torch.int32).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(2 * pool_n):
        k = i % pool_n
        h, (e_p, p_p, w_p) = pool[k], arrays[k]
        hm.solve_host_ptrs(h.n, h.m, e_p.data_ptr(), p_p.data_ptr(), w_p.data_ptr(), h.seed, 0,
                           edges.data_ptr(), sh)
    wall = time.perf_counter() - t0
    work = float(sum(units[i % pool_n] for i in range(2 * pool_n)))
    plain = {"requests": 2 * pool_n, "wall_s": wall, "pins_per_s": work / wall, "req_per_s": 2 * pool_n / wall,
             "path": "one hm_solve_host call per request, one after another"}
    return {"pool": pool_n, "kappa_mean": float(kap.mean()), "slots": slots, "sweep": sweep,
            "saturated_served": served, "saturated_one_slot": serial, "plain_one_at_a_time": plain,
            "served_speedup": served["pins_per_s"] / plain["pins_per_s"],
            "one_slot_speedup": serial["pins_per_s"] / plain["pins_per_s"],
            "h2d_bytes_per_request": int(np.mean([h.eoff.nbytes + h.pins.nbytes + h.weights.nbytes
                                                  for h in pool]))}


def run_serve(args, world, rank, local):
    """Requests arrive as a Poisson stream at each rate of the sweep and go
    through hm_server (continuous batching); latency = submit -> done."""
    import torch
    import paper_2602_22976_gb300 as hm

    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    hm.build()
    seed = replica_seed(args.seed, rank)
    clocks = Clocks(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    r = measure_serve(seed, (100, 300, 1000, 3000, 10000), lambda rate: int(min(max(64, rate), 1000)),
                      args.scale, arrival_seed=args.seed)
    clk = clocks.stop()
    served = r["saturated_served"]
    work_all, wall_max = replica_totals(served["work"], served["wall_s"] * 1e3, world)
    out = {
        "metric": METRIC, "value": work_all / (wall_max / 1e3), "unit": "pins/s", "n_gpus": world,
        "steps": served["requests"], "warmup": 0, "ms_per_step": 1e3 / served["req_per_s"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": WORKLOADS["serve"]["desc"], "l2": "inputs larger than L2",
                   "parallelism": f"replicas x{world}"},
        "serve": r, "clocks": clk, "cpu_baseline": None,
        "e2e": {"value": served["pins_per_s"], "unit": "pins/s",
                "h2d_bytes_per_step": r["h2d_bytes_per_request"], "d2h_bytes_per_step": None},
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# ------------------------------------------------------------------ our arm

def run_ours(args, world, rank, local):
    import torch
    import torch.distributed as dist
    import synth
    import paper_2602_22976_gb300 as hm

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    hm.build()
    wl = WORKLOADS[args.workload]
    h = wl["make"](replica_seed(args.seed, rank), args.scale)
    mt = hm.Matcher.from_hypergraph(h)
    if args.noise > 0:
        mt.set_noise(args.noise)
    rnd_mode = args.noise > 0
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    for _ in range(max(args.warmup, 3)):
        mt.match(stream)
    res = mt.result()
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = Clocks(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    for k in range(args.steps):
        flush.zero_()  # L2 flush between steps, outside the step's events
        starts[k].record(stream)
        mt.match(stream)
        ends[k].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    t_ms = float(sum(step_ms))
    res2 = mt.result()
    assert res2.rounds == res.rounds and res2.count == res.count
    units, t_max = replica_totals(float(h.kappa) * res.rounds * args.steps, t_ms, world)
    value = units / (t_max / 1e3)

    # per-kernel replay for the roofline
    prof = mt.profile(stream)
    stats = mt.round_stats()
    create_ms = mt.create_ms()
    max_size = int(np.diff(h.eoff).max()) if h.m else 0
    pairs = h.m > 0 and max_size == 2 and h.kappa == 2 * h.m  # a graph
    kb = kernel_bytes(stats, h.n, h.m, h.kappa, rnd_mode, p16=max_size <= 0xFFFF, pairs=pairs)
    dom = max(("argmax", "win", "kill"), key=lambda k: prof[k][0])
    assert all(isinstance(prof[k], tuple) for k in hm.KERNELS)
    peaks = measured_peaks()
    # achieved bandwidth of the dominant kernel: the method's own per-unit
    # bytes where its step is the argmax of the fixed order, else this
    # design's counts; both are reported
    design_gbs = kb[dom] / (prof[dom][0] / 1e3) / 1e9
    if dom == "argmax" and stats[:, 9].sum() > 0:  # HM_STAT_DEG, filled by the replay
        alg_bytes, bytes_model = method_argmax_bytes(stats), (
            "method step a1: 24 B per active vertex + 8 B per list entry of an active vertex")
    else:
        alg_bytes, bytes_model = kb[dom], "this design's per-unit counts (kernel_bytes)"
    achieved = alg_bytes / (prof[dom][0] / 1e3) / 1e9
    # the DRAM bytes the kernels actually moved (ncu, committed rows) over the same time
    design_pl = {k: kb[k] / max(1, prof[k][1]) for k in ("init", "argmax", "win", "kill")}
    traffic = measured_traffic(dom, rnd_mode, args.workload, design_pl[dom])
    traffic_gbs = traffic * prof[dom][1] / (prof[dom][0] / 1e3) / 1e9 if traffic else None
    per_kernel = {k: {"ms": prof[k][0], "launches": prof[k][1], "alg_bytes": kb[k],
                      "gbs": (kb[k] / (prof[k][0] / 1e3) / 1e9) if prof[k][0] > 0 else None}
                  for k in hm.KERNELS}
    round_ms = [[round(float(x), 4) for x in row[:3]] for row in prof["rounds_ms"]]
    total_bytes = sum(kb.values())
    # random-access ceilings of this GPU for an array the size of the live flags
    ra = probe_random_access(max(h.m, 1 << 20), 200_000_000, stream.cuda_stream or None)
    kills = float(stats[:, hm.STAT_COLUMNS.index("kills")].sum())
    rar = random_access_roofline(stats, prof, ra, rnd_mode)
    loop_ms = sum(prof[k][0] for k in hm.KERNELS)
    rounds_run = int(prof["win"][1])  # one win launch a round
    # the whole match: the method's bytes of steps a1-a4 (the plain
    # formulation), this design's element bytes, and the DRAM bytes ncu
    # counted (committed rows), each over the timed match
    t_match_s = t_max / args.steps / 1e3
    mb = method_match_bytes(stats) if stats[:, 10].sum() > 0 else None  # HM_STAT_LEDGES, from the replay
    dram = {k: measured_traffic(k, rnd_mode, args.workload, design_pl[k]) for k in ("init", "argmax", "win", "kill")}
    dram_total = (sum(dram[k] * prof[k][1] if k != "init" else dram[k] for k in dram)
                  if all(v is not None for v in dram.values()) else None)
    frac = lambda b: None if b is None else b / t_match_s / 1e9 / measured_peaks()["hbm_gbs"]
    whole = {
        "t_match_ms": t_match_s * 1e3,
        "model_bytes": None if mb is None else mb["total"], "model_bytes_by_step": mb,
        "model_frac": frac(None if mb is None else mb["total"]),
        "design_bytes": total_bytes, "design_frac": frac(total_bytes),
        "dram_bytes": dram_total, "dram_frac": frac(dram_total),
        "dram_bytes_by_kernel": {k: (None if dram[k] is None else dram[k] * (prof[k][1] if k != "init" else 1))
                                 for k in dram},
        "peak_gbs": measured_peaks()["hbm_gbs"],
        "note": ("bytes per match over the timed match time and the measured HBM peak: model = the method's "
                 "steps a1-a4 as the plain formulation moves them (per-round units from the replay's "
                 "counters); design = this design's element bytes (kernel_bytes); dram = ncu's "
                 "dram__bytes per launch (profiles/traffic.json) times launches"),
    }
    # init + three kernels per round (argmax, win, kill with the round end);
    # re-randomised: four in round 1 (scan, proposals, win, kill), two in
    # each later round (offers, win test with the round end)
    launches = 1 + ((4 + 2 * (rounds_run - 1)) if rnd_mode else 3 * rounds_run)

    out = {}
    if rank == 0:
        # end to end through hm_solve_host from pinned host memory
        e2e = None
        if args.e2e_steps > 0 and rnd_mode:
            # hm_solve_host runs the fixed order: the public handle calls instead,
            # from pinned host buffers (copy in, hm_create, hm_set_noise,
            # hm_match, hm_result to host)
            pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
            eoff_p, pins_p = pin(h.eoff), pin(h.pins)
            w_p = None if h.weights is None else pin(h.weights)

            def call():
                d_eoff = eoff_p.to("cuda", non_blocking=True)
                d_pins = pins_p.to("cuda", non_blocking=True)
                d_w = None if w_p is None else w_p.to("cuda", non_blocking=True)
                with hm.Matcher(h.n, h.m, d_eoff, d_pins, d_w, seed=h.seed) as m2:
                    m2.set_noise(args.noise)
                    m2.match()
                    return m2.result()
            te, tes, r2 = timed_calls(call, args.e2e_steps)
            assert r2.rounds == res.rounds and r2.count == res.count
            h2d = h.eoff.nbytes + h.pins.nbytes + (0 if h.weights is None else h.weights.nbytes)
            e2e = {"value": h.kappa * res.rounds / te, "unit": "pins/s", "ms_per_step": te * 1e3,
                   "ms_calls": tes, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(res.count * 4 + 64),
                   "path": "hm_create + hm_set_noise + hm_match + hm_result"}
        elif args.e2e_steps > 0:
            pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
            eoff_p, pins_p = pin(h.eoff), pin(h.pins)
            w_p = None if h.weights is None else pin(h.weights)
            edges_p = torch.empty(max(h.m, 1), dtype=torch.int32).pin_memory()
            flags = hm.HM_UNWEIGHTED if h.weights is None else 0
            sh = stream.cuda_stream or None
            call = lambda: hm.solve_host_ptrs(h.n, h.m, eoff_p.data_ptr(), pins_p.data_ptr(),
                                              None if w_p is None else w_p.data_ptr(), h.seed,
                                              flags, edges_p.data_ptr(), sh)
            te, tes, (cnt, rnd, _w) = timed_calls(call, args.e2e_steps)
            assert rnd == res.rounds and cnt == res.count
            h2d = h.eoff.nbytes + h.pins.nbytes + (0 if h.weights is None else h.weights.nbytes)
            e2e = {"value": h.kappa * res.rounds / te, "unit": "pins/s", "ms_per_step": te * 1e3,
                   "ms_calls": tes, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(res.count * 8 + 64)}
        cpu = None
        cpu_greedy = None
        parity = None
        if not args.no_cpu_baseline:
            import oracle
            oracle.build()
            t0 = time.perf_counter()
            o = oracle.match(h, noise=args.noise)
            tc = time.perf_counter() - t0
            parity = bool(np.array_equal(o.edges, res.edges) and o.rounds == res.rounds)
            cpu = {"value": h.kappa * o.rounds / tc, "unit": "pins/s", "cores": cpu_cores_used(),
                   "kind": "oracle", "sample": f"the full instance, one oracle run ({tc:.1f} s)",
                   "active_pins": int(o.round_stats[:, 1].sum()), "host": host_cpu()}
            if not rnd_mode:
                # the paper's single-core Greedy baseline: sort by priority, take an
                # edge when all its pins are free (same order, so the same matching)
                t0 = time.perf_counter()
                g = oracle.greedy(h)
                tg = time.perf_counter() - t0
                gpu_ms = t_max / args.steps
                cpu_greedy = {"ms": tg * 1e3, "cores": 1, "kind": "sequential greedy (oracle)",
                              "same_matching": bool(np.array_equal(np.flatnonzero(g), res.edges)),
                              "speedup_of_match": tg * 1e3 / gpu_ms}
                if e2e:
                    cpu_greedy["speedup_end_to_end"] = tg * 1e3 / e2e["ms_per_step"]
        # the batching and serving workloads, measured in the same run on the
        # same GPU (one GPU only: the scaling runs report the main metric)
        sub_batch = sub_serve = None
        if world == 1 and args.workload == "large" and not rnd_mode and args.scale == 1:
            mt.close()  # the batch below needs the room more than this handle
            clocks2 = Clocks(local)
            clocks2.start()
            if not args.no_batch:
                sub_batch = measure_batch(args.seed, 4096, steps=10, warmup=3, stream=stream)
                sub_batch["note"] = ("4,096 instances in one graph launch (10 timed launches, CUDA events) "
                                     "against the same instances as 4,096 hm_match launches (median of 3)")
            if not args.no_serve:
                sub_serve = measure_serve(args.seed, (1000, 10000), lambda rate: min(rate, 1000),
                                          arrival_seed=args.seed)
                sub_serve["note"] = ("Poisson arrivals at 1,000 and 10,000 req/s (1,000 requests each); "
                                     "saturated = the whole stream submitted at once to the server (8 slots, "
                                     "and 1 slot, which still groups queued requests), against the plain form: "
                                     "the same requests one hm_solve_host call at a time; served_speedup = "
                                     "8-slot server over the plain form")
            clk2 = clocks2.stop()
            for x in (sub_batch, sub_serve):
                if x is not None:
                    x["clocks"] = clk2
        out = {
            "metric": METRIC, "value": value, "unit": "pins/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": wl["desc"] + (f" scaled 1/{args.scale}" if args.scale > 1 else ""),
                       "n": h.n, "m": h.m, "kappa": h.kappa,
                       "rounds": res.rounds, "matched": res.count, "weight": res.weight,
                       "priorities": (f"re-drawn every round, noise amplitude {args.noise}" if rnd_mode
                                      else "one fixed strict order"),
                       "l2": f"{L2_FLUSH_BYTES >> 20} MiB write between steps, outside step events",
                       "parallelism": f"replicas x{world}"},
            "time_to_matching_ms": {"mean": t_ms / args.steps, "median": statistics.median(step_ms),
                                    "p99": float(np.percentile(step_ms, 99))},
            "create_ms": create_ms,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peaks["hbm_gbs"],
                         "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"], "traffic": traffic, "traffic_gbs": traffic_gbs,
                         "traffic_frac": traffic_gbs / peaks["hbm_gbs"] if traffic_gbs else None,
                         "alg_bytes_per_launch": alg_bytes / max(1, prof[dom][1]), "bytes_model": bytes_model,
                         "design_bytes_per_launch": kb[dom] / max(1, prof[dom][1]),
                         "design_frac": design_gbs / peaks["hbm_gbs"],
                         "kernel_source": kernel_source_hash(TRAFFIC_ROWS[(dom, rnd_mode)][1]),
                         "peak_source": peaks["source"],
                         "loop_gbs": total_bytes / (loop_ms / 1e3) / 1e9,
                         "whole_match_model_frac": whole["model_frac"],
                         "whole_match_design_frac": whole["design_frac"],
                         "whole_match_dram_frac": whole["dram_frac"]},
            "random_access": {
                "array_bytes": max(h.m, 1 << 20), "ceiling_gops": ra,
                "kill_entries_gops": kills / (prof["kill"][0] / 1e3) / 1e9,
                "note": "kill reads each target flag (rounds >= 2) and writes the live ones; "
                        "its bound is the random 1-byte load/store rate, not HBM bandwidth"},
            "random_access_roofline": rar,
            "whole_match": whole,
            "kernels": per_kernel,
            "round_ms_argmax_win_kill": round_ms,
            "round_stats": stats.tolist(),
            "cpu_baseline": cpu,
            "cpu_greedy": cpu_greedy,
            "e2e": e2e,
            "clocks": clk,
            "gpu_launches": launches * args.steps,
            "parity_vs_oracle": parity,
            "batch": sub_batch,
            "serve": sub_serve,
            "paper_context": PAPER_CONTEXT,
        }
        if cpu and cpu.get("active_pins"):
            out["active_pins_per_s"] = cpu["active_pins"] * args.steps * world / (t_max / 1e3)
        print(json.dumps(out), flush=True)
    mt.close()  # a no-op when the sub-measurements closed it already
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "batch":
        run_batch(args, world, rank, local)
    elif args.workload == "serve":
        run_serve(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
