"""hm_match_noalloc: matching without any memory allocation.

For callers that cannot allocate device memory when they need a matching
(for instance when their framework owns all device memory through its own
arena, or a latency-bound loop cannot pay for cudaMalloc). The entry point's
working memory is a fixed array inside libhm.so; these tests call it through
the C ABI and require the same
matching and round count as the allocating path (hm_create + hm_match +
hm_result_device), exactly: the result is a set of integers, so the
tolerance is zero. Two calls run back to back on each input, and the inputs
follow one another, so every call starts from the bytes the previous one
left in the shared array.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth
import paper_2602_22976_gb300 as hmlib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    hmlib.build()
    assert torch.cuda.is_available(), "needs a CUDA device"
    hmlib.lib()


def via_allocating_path(h):
    with hmlib.Matcher.from_hypergraph(h) as mt:
        mt.match()
        res = mt.result()
        mask = torch.zeros(max(h.m, 1), dtype=torch.uint8, device="cuda")
        mt.result_device(mask)
        torch.cuda.synchronize()
    return mask[:h.m].cpu().numpy(), res.rounds


def via_noalloc(h):
    dev = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()
    eoff = dev(h.eoff, np.int64)
    pins = dev(h.pins, np.int32)
    w = None if h.weights is None else dev(h.weights, np.float32)
    mask = torch.full((max(h.m, 1),), 7, dtype=torch.uint8, device="cuda")  # garbage on purpose
    result = torch.full((2,), -5, dtype=torch.int32, device="cuda")
    flags = hmlib.HM_UNWEIGHTED if w is None else 0
    torch.cuda.synchronize()
    st = hmlib.lib().hm_match_noalloc(h.n, h.m, eoff.data_ptr(), pins.data_ptr(),
                                      None if w is None else w.data_ptr(), h.seed, flags,
                                      mask.data_ptr(), result.data_ptr(), None)
    assert st == hmlib.HM_OK, hmlib.last_error()
    torch.cuda.synchronize()
    rounds, status = result.cpu().tolist()
    return mask[:h.m].cpu().numpy(), rounds, status


INPUTS = [
    lambda: synth.small(seed=3, n=4000, m=12_000),
    lambda: synth.large(seed=4, n=50_000, m=100_000, kmax=256),
    lambda: synth.unweighted(seed=5, n=20_000, m=40_000),
    lambda: synth.from_edges(8, [[i, i + 1] for i in range(7)], [(i + 1) / 8 for i in range(7)]),
]


@pytest.mark.parametrize("make", INPUTS, ids=["uniform", "powerlaw", "unweighted", "path"])
def test_same_result_as_allocating_path_twice_in_a_row(make):
    h = make()
    ref_mask, ref_rounds = via_allocating_path(h)
    for _ in range(2):
        mask, rounds, status = via_noalloc(h)
        assert status == hmlib.HM_OK
        assert rounds == ref_rounds
        assert np.array_equal(mask, ref_mask)


def test_rejects_inputs_beyond_the_fixed_scratch():
    L = hmlib.lib()
    eoff = torch.zeros(1, dtype=torch.int64, device="cuda")
    result = torch.zeros(2, dtype=torch.int32, device="cuda")
    st = L.hm_match_noalloc(2_000_000, 0, eoff.data_ptr(), None, None, 1, hmlib.HM_UNWEIGHTED,
                            None, result.data_ptr(), None)
    assert st == hmlib.HM_EINVAL
    assert "scratch" in hmlib.last_error()


def _call(n, m, eoff, pins, w, mask, result, flags=0):
    ptr = lambda t: None if t is None else t.data_ptr()
    return hmlib.lib().hm_match_noalloc(n, m, ptr(eoff), ptr(pins), ptr(w), 1, flags, ptr(mask),
                                        ptr(result), None)


@pytest.mark.parametrize("kind", ["zero_weight", "nan_weight", "inf_weight", "pin_too_large",
                                  "negative_pin", "decreasing_eoff", "empty_edge", "eoff0"])
def test_invalid_input_is_reported_in_the_result_word(kind):
    """The kernel checks edge ranges and weights before it reads a pin, and
    every pin before it uses one as an index, and reports a failed check as
    result[1] = HM_EINVAL with nothing matched. Every buffer below is as long
    as the offsets say, so no check reads outside it."""
    eoff = [0, 3, 5, 8]
    pins = [0, 1, 2, 2, 3, 4, 5, 6]
    w = [0.5, 0.25, 0.75]
    n = 8
    if kind == "zero_weight":
        w[1] = 0.0
    elif kind == "nan_weight":
        w[2] = float("nan")
    elif kind == "inf_weight":
        w[0] = float("inf")
    elif kind == "pin_too_large":
        pins[6] = n
    elif kind == "negative_pin":
        pins[4] = -3
    elif kind == "decreasing_eoff":
        eoff = [0, 3, 2, 8]
    elif kind == "empty_edge":
        eoff = [0, 3, 3, 8]
    elif kind == "eoff0":
        eoff = [1, 3, 5, 8]
    d_eoff = torch.tensor(eoff, dtype=torch.int64, device="cuda")
    d_pins = torch.tensor(pins, dtype=torch.int32, device="cuda")
    d_w = torch.tensor(w, dtype=torch.float32, device="cuda")
    mask = torch.zeros(3, dtype=torch.uint8, device="cuda")
    result = torch.full((2,), -5, dtype=torch.int32, device="cuda")
    assert _call(n, 3, d_eoff, d_pins, d_w, mask, result) == hmlib.HM_OK, hmlib.last_error()
    torch.cuda.synchronize()
    rounds, status = result.cpu().tolist()
    assert status == hmlib.HM_EINVAL and rounds == 0
    # the same buffers, repaired, give a valid matching in the next call
    good = synth.from_edges(n, [[0, 1, 2], [2, 3], [4, 5, 6]], [0.5, 0.25, 0.75])
    ref_mask, ref_rounds = via_allocating_path(good)
    mask2, rounds2, status2 = via_noalloc(good)
    assert status2 == hmlib.HM_OK and rounds2 == ref_rounds and np.array_equal(mask2, ref_mask)


def test_refuses_host_memory():
    """Pointers that are not memory of the current device are refused on the
    host, before any launch: pinned host memory and ordinary host memory."""
    eoff = torch.tensor([0, 2], dtype=torch.int64)
    pins = torch.tensor([0, 1], dtype=torch.int32)
    w = torch.tensor([0.5], dtype=torch.float32)
    d_eoff, d_pins, d_w = eoff.cuda(), pins.cuda(), w.cuda()
    mask = torch.zeros(1, dtype=torch.uint8, device="cuda")
    result = torch.zeros(2, dtype=torch.int32, device="cuda")
    for host in (eoff.pin_memory(), eoff):
        assert _call(2, 1, host, d_pins, d_w, mask, result) == hmlib.HM_EINVAL
        assert "device memory" in hmlib.last_error()
    assert _call(2, 1, d_eoff, d_pins, d_w, mask, result.cpu().pin_memory()) == hmlib.HM_EINVAL
    assert _call(2, 1, d_eoff, d_pins, d_w, mask, result) == hmlib.HM_OK
    torch.cuda.synchronize()
    assert result.cpu().tolist() == [1, hmlib.HM_OK]
