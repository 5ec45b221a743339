"""Host logic of bench.py that needs no GPU: the reference arm's JSON line
(it times the CPU oracle), the lookup of committed ncu traffic rows by
kernel, mode, source hash and workload, and the byte count of the method's
argmax step from the per-round counters."""
import hashlib
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_reference_arm_line():
    """--impl reference prints one JSON line with the contract's keys: the
    same metric, unit and workload as the GPU arm, the oracle as its
    cpu_baseline, and an e2e object without host copies."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                         timeout=900, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "pins/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["steps"] == 1 and d["warmup"] == 0
    assert d["config"]["workload"] == bench.WORKLOADS["large"]["desc"]
    assert d["config"]["same_instance_as_gpu_arm"] is True  # the full instance, not a sample
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["cpu_baseline"]["host"]["nproc"] >= 1
    assert "76.6x" in d["paper_context"]["claim"]
    assert d["e2e"] == {"value": d["value"], "unit": "pins/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def _fake_root(tmp_path, source_text, rows):
    csrc = tmp_path / "paper_2602_22976_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "rounds.cu").write_text(source_text)
    (csrc / "rrounds.cu").write_text(source_text + "// other file\n")
    prof = tmp_path / "profiles"
    prof.mkdir()
    doc = {"rows": [dict(kernel=k, mode=m, workload=w, source_hash=h, bytes_per_launch=b, launches=11,
                         scale=sc, design_bytes_per_launch=d) for k, m, w, h, b, sc, d in rows]}
    (prof / "traffic.json").write_text(json.dumps(doc))


def test_traffic_rows_keyed_by_source_workload_and_mode(tmp_path, monkeypatch):
    """A stored DRAM figure is reported only for the source it was measured
    on, in its mode and on its workload; anything else reads as None. A row
    captured at a smaller scale is scaled by this design's bytes per launch
    at the bench's size over those of the captured run; a full-size row is
    preferred to a scaled one."""
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h1 = hashlib.sha256(b"// kernel v1\n").hexdigest()[:16]
    h1r = hashlib.sha256(b"// kernel v1\n// other file\n").hexdigest()[:16]
    _fake_root(tmp_path, "// kernel v1\n", [
        ("k_argmax", "fixed", "large", h1, 1000, 1, None), ("k_argmax", "fixed", "graph", h1, 2000, 1, None),
        ("k_argmax", "fixed", "large", h1, 111, 4, 50.0),
        ("k_kill", "re-randomised", "large", h1, 3000, 1, None),
        ("k_rflat+k_rpropose+k_epush", "re-randomised", "large", h1r, 4000, 1, None),
        ("k_win", "fixed", "large", "0000000000000000", 5000, 1, None),
        ("k_kill", "fixed", "large", h1, 600, 4, 200.0)])
    assert bench.measured_traffic("argmax", False) == 1000.0
    assert bench.measured_traffic("argmax", False, "graph") == 2000.0
    assert bench.measured_traffic("argmax", False, "unweighted") is None
    assert bench.measured_traffic("kill", True) == 3000.0
    assert bench.measured_traffic("argmax", True) == 4000.0
    assert bench.measured_traffic("win", False) is None  # measured on another source
    assert bench.measured_traffic("kill", False) is None  # scaled row, no design bytes to scale by
    assert bench.measured_traffic("kill", False, "large", 800.0) == 600.0 * 800.0 / 200.0
    (tmp_path / "paper_2602_22976_gb300" / "csrc" / "rounds.cu").write_text("// kernel v2\n")
    assert bench.measured_traffic("argmax", False) is None  # the kernel changed since


def test_committed_traffic_file_is_well_formed():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        doc = json.load(f)
    assert doc["rows"]
    for r in doc["rows"]:
        assert r["mode"] in ("fixed", "re-randomised") and r["bytes_per_launch"] > 0
        assert len(r["source_hash"]) == 16 and r.get("scale", 1) >= 1
        assert (r["kernel"], r["mode"] == "re-randomised") in {(v[0], k[1]) for k, v in bench.TRAFFIC_ROWS.items()}


def test_method_match_bytes_from_the_counters():
    """The plain formulation's bytes of steps a1-a4 from the per-round units:
    active vertices (NEXT) and their degrees (DEG), live edges (LEDGES) and
    live pins (LPINS), winners and their pins."""
    stats = np.zeros((2, 12), dtype=np.int64)
    stats[:, 7] = [10, 4]        # active vertices
    stats[:, 9] = [100, 30]      # their degree sums
    stats[:, 10] = [20, 6]       # live edges
    stats[:, 11] = [90, 25]      # live pins
    stats[:, 3] = [5, 2]         # winners
    stats[:, 4] = [20, 7]        # their pins
    stats[:, 1] = 999            # other columns play no part
    b = bench.method_match_bytes(stats)
    assert b["a1"] == 24 * 14 + 8 * 130
    assert b["a2"] == 24 * 26 + 8 * 115 + 27 + 7
    assert b["a3"] == 5 * 115 + 4 * 26
    assert b["a4"] == 8 * (26 + 14)
    assert b["total"] == b["a1"] + b["a2"] + b["a3"] + b["a4"]


def test_host_cpu_reports_cores():
    h = bench.host_cpu()
    assert h["nproc"] >= 1 and h["machine"]


def test_method_argmax_bytes_from_the_counters():
    """24 bytes per active vertex and 8 per list entry of an active vertex,
    from the NEXT and DEG columns of every round."""
    stats = np.zeros((3, 10), dtype=np.int64)
    stats[:, 7] = [10, 4, 1]       # active vertices
    stats[:, 9] = [100, 30, 2]     # their degree sums
    stats[:, 1] = 999              # other columns play no part
    assert bench.method_argmax_bytes(stats) == 24 * 15 + 8 * 132


def test_end_to_end_calls_timed_one_by_one():
    """The end-to-end leg: two untimed calls, then k timed ones; the median
    of the per-call times is reported with every call's milliseconds."""
    n = {"calls": 0}

    def call():
        n["calls"] += 1
        return n["calls"]

    med, ms, last = bench.timed_calls(call, 5)
    assert n["calls"] == 7 and last == 7
    assert len(ms) == 5 and all(t >= 0 for t in ms)
    assert med == pytest.approx(float(np.median(ms)) / 1e3, abs=1e-5)


def test_kernel_bytes_fixed_order_from_the_counters():
    """This design's element bytes per kernel kind, fixed order, hypergraph,
    16-bit counters: the per-unit table of the design written out by hand
    for two rounds."""
    ACT, ADV, PROP, WIN, WPIN, KILL, ITEM, NEXT = range(8)
    stats = np.zeros((2, 12), dtype=np.int64)
    stats[0, [ACT, PROP, WIN, WPIN, KILL, ITEM, NEXT]] = [100, 90, 10, 40, 300, 30, 80]
    stats[1, [ACT, ADV, PROP, WIN, WPIN, KILL, ITEM, NEXT]] = [80, 50, 20, 5, 15, 60, 12, 0]
    b = bench.kernel_bytes(stats, n=100, m=200, random=False, p16=True, pairs=False)
    assert b["init"] == 200 * (1 + 1 + 2 * 2)
    # round 1: first entry + record write per vertex, P read + write per
    # proposal, list write per kept vertex; every round: 12 per winner
    argmax = (100 * 12 + 90 * 4 + 80 * 4) + (80 * 21 + 50 * 5 + 20 * 12 + 0) + 12 * (10 + 5)
    assert b["argmax"] == argmax
    # winner 21 + 4 (list), winner pin 28, kill range 8
    assert b["win"] == (10 * 25 + 40 * 28 + 30 * 8) + (5 * 25 + 15 * 28 + 12 * 8)
    # kill range read 8, killed entry 5
    assert b["kill"] == (30 * 8 + 300 * 5) + (12 * 8 + 60 * 5)


def test_random_access_roofline_from_the_counters():
    """The time each kernel's random accesses take at the measured rates:
    k_argmax one flag load per active vertex and skipped entry from round 2
    on plus one returning atomic per proposal; k_kill one store per target
    in round 1 and one load per target later; over the kernel's time."""
    stats = np.zeros((3, 12), dtype=np.int64)
    stats[:, 0] = [1000, 400, 100]     # active vertices
    stats[:, 1] = [0, 800, 300]        # skipped entries
    stats[:, 2] = [900, 200, 50]       # proposals
    stats[:, 5] = [5000, 2000, 600]    # kill entries
    ra = {"load1B": 100.0, "store1B": 50.0, "atomic4B": 25.0}  # 1e9 per second
    prof = {"argmax": (0.001, 3), "kill": (0.0005, 3)}          # ms, launches
    r = bench.random_access_roofline(stats, prof, ra, random=False)
    argmax_s = (400 + 100 + 800 + 300) / 100e9 + (900 + 200 + 50) / 25e9
    kill_s = (2000 + 600) / 100e9 + 5000 / 50e9
    assert r["argmax"]["bound_ms"] == pytest.approx(argmax_s * 1e3)
    assert r["argmax"]["frac"] == pytest.approx(argmax_s * 1e3 / 0.001)
    assert r["kill"]["bound_ms"] == pytest.approx(kill_s * 1e3)
    assert r["kill"]["frac"] == pytest.approx(kill_s * 1e3 / 0.0005)
    assert bench.random_access_roofline(stats, prof, ra, random=True) is None


def test_kernel_bytes_rerandomised_from_the_counters():
    """Re-randomised rounds, hypergraph: round 1 is the flat scan, the
    proposals, the win and the kill; later rounds are the edge rounds
    (records in and out, the live pins' offers, the win test and the whole
    clear of the other slot buffer), written out by hand for three rounds."""
    ADV, PROP, WIN, WPIN, KILL, ITEM, LIVE, LEDGES = 1, 2, 3, 4, 5, 6, 8, 10
    n, m = 100, 200
    stats = np.zeros((3, 12), dtype=np.int64)
    stats[0, [ADV, PROP, WIN, WPIN, KILL, ITEM]] = [1000, 90, 10, 40, 300, 30]
    stats[1, [ADV, WIN, WPIN, LIVE, LEDGES]] = [600, 8, 20, 600, 120]
    stats[2, [ADV, WIN, WPIN, LIVE, LEDGES]] = [90, 3, 6, 50, 15]
    b = bench.kernel_bytes(stats, n=n, m=m, random=True, p16=True, pairs=False)
    assert b["init"] == m * (1 + 4 + 4 + 1) + n * (1 + 8 + 8)
    argmax = 1000 * 8 + n * 16 + 90 * 24 + 10 * 4                   # round 1
    argmax += m * 16 + m + 0 + 120 * 16 + 600 * (4 + 8)              # round 2: every record and its flag
    argmax += 120 * 16 + 90 * 5 + 15 * 16 + 50 * 8                  # round 3: round 2's live edges
    assert b["argmax"] == argmax
    win = 10 * 25 + 40 * 28 + 30 * 8                                 # round 1
    win += 120 * 16 + 600 * 12 + 8 + 20 + 8 * n                      # round 2
    win += 15 * 16 + 50 * 12 + 3 + 6 + 8 * n                         # round 3
    assert b["win"] == win
    assert b["kill"] == 30 * 8 + 300 * 9
