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
                          "--steps", "1", "--warmup", "1"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "pins/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["n_gpus"] == 1
    assert d["steps"] == 1 and d["warmup"] == 1
    assert d["config"]["workload"] == bench.WORKLOADS["large"]["desc"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "pins/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def _fake_root(tmp_path, source_text, rows):
    csrc = tmp_path / "paper_2602_22976_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "rounds.cu").write_text(source_text)
    (csrc / "rrounds.cu").write_text(source_text + "// other file\n")
    prof = tmp_path / "profiles"
    prof.mkdir()
    table = ["| kernel | mode | source hash | bytes per launch | launches |", "|---|---|---|---|---|"]
    table += [f"| {k} | {m} | {h} | {b} | 11 |" for k, m, h, b in rows]
    (prof / "traffic.md").write_text("\n".join(table) + "\n")


def test_traffic_rows_keyed_by_source_workload_and_mode(tmp_path, monkeypatch):
    """A stored DRAM figure is reported only for the source it was measured
    on, in its mode and on its workload; anything else reads as None."""
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h1 = hashlib.sha256(b"// kernel v1\n").hexdigest()[:16]
    h1r = hashlib.sha256(b"// kernel v1\n// other file\n").hexdigest()[:16]
    _fake_root(tmp_path, "// kernel v1\n", [
        ("k_argmax", "fixed", h1, 1000), ("k_argmax", "fixed, graph", h1, 2000),
        ("k_kill", "re-randomised", h1, 3000), ("k_rargmax+k_rlong+k_rfin", "re-randomised", h1r, 4000),
        ("k_win", "fixed", "0000000000000000", 5000)])
    assert bench.measured_traffic("argmax", False) == 1000.0
    assert bench.measured_traffic("argmax", False, "graph") == 2000.0
    assert bench.measured_traffic("argmax", False, "unweighted") is None
    assert bench.measured_traffic("kill", True) == 3000.0
    assert bench.measured_traffic("argmax", True) == 4000.0
    assert bench.measured_traffic("win", False) is None  # measured on another source
    (tmp_path / "paper_2602_22976_gb300" / "csrc" / "rounds.cu").write_text("// kernel v2\n")
    assert bench.measured_traffic("argmax", False) is None  # the kernel changed since


def test_method_argmax_bytes_from_the_counters():
    """24 bytes per active vertex and 8 per list entry of an active vertex,
    from the NEXT and DEG columns of every round."""
    stats = np.zeros((3, 10), dtype=np.int64)
    stats[:, 7] = [10, 4, 1]       # active vertices
    stats[:, 9] = [100, 30, 2]     # their degree sums
    stats[:, 1] = 999              # other columns play no part
    assert bench.method_argmax_bytes(stats) == 24 * 15 + 8 * 132
