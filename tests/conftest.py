import glob
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN_DIR = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and libhm.so")
    config.addinivalue_line("markers", "slow: full-size workloads (tens of seconds)")


def golden_cases():
    out = []
    for p in sorted(glob.glob(os.path.join(GOLDEN_DIR, "*.json"))):
        with open(p) as f:
            c = json.load(f)
        c["name"] = os.path.splitext(os.path.basename(p))[0]
        out.append(c)
    return out


def golden_hypergraph(c):
    import synth
    return synth.from_edges(c["n"], c["edges"], c["weights"], name=c["name"])
