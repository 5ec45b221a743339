"""hm_match_noalloc: matching without any memory allocation.

For callers that cannot allocate device memory when they need a matching
(for instance while they capture a CUDA graph, or when their framework owns
all device memory). The entry point's working memory is a fixed array inside
libhm.so; these tests call it through the C ABI and require the same
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
