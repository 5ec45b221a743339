"""Counts derived from the oracle's run that the GPU's per-round counters
must equal (used by tests/test_gpu_parity.py, pinned on the CPU by
tests/test_oracle.py against a direct replay of the rounds)."""
import numpy as np

import oracle


def active_sets(h, o):
    """From the oracle's run: for every round r, the vertices active at its
    start (unmatched, with a live edge: some incident edge is decided in round
    r or later) and the sum of their degrees."""
    sizes = np.diff(h.eoff)
    dec = o.decided_round.astype(np.int64)
    vmax = np.zeros(h.n, dtype=np.int64)
    np.maximum.at(vmax, h.pins, np.repeat(dec, sizes))
    deg = np.bincount(h.pins, minlength=h.n)
    return ([int((vmax >= r).sum()) for r in range(1, o.rounds + 1)],
            [int(deg[vmax >= r].sum()) for r in range(1, o.rounds + 1)])


def entries_ahead_of_the_match(h, o):
    """Over a whole run, the cursor of a vertex passes exactly the entries of
    its list that rank above its matching edge, or its whole list if it stays
    unmatched: summed over the vertices, from the oracle's matching."""
    keys = oracle.keys(h)
    eid = np.repeat(np.arange(h.m), np.diff(h.eoff))
    mv = np.full(h.n, -1, dtype=np.int64)
    won = o.in_matching[eid] == 1
    mv[h.pins[won]] = eid[won]
    matched = mv >= 0
    ahead = matched[h.pins] & (keys[eid] > keys[np.maximum(mv[h.pins], 0)])
    return int(ahead.sum()) + int(np.bincount(h.pins, minlength=h.n)[~matched].sum())
