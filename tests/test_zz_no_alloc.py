"""rewl_run_static: the entry point for callers that cannot call cudaMalloc
(a framework's caching allocator owns the device memory, a fixed device-memory
budget, or a loop that cannot take cudaMalloc's device-wide synchronisation).
It keeps the whole run's state in a fixed device array inside the library.

Its results must equal those of the allocating path (rewl_create + rewl_run)
bit for bit -- the tolerance every parity test here uses for ln g -- and a
second call must not see anything the first call left in the shared array.
This file is collected last so that a stop-at-first-failure run has already
run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1312_3004_gb300 import REWL, _lib

pytestmark = pytest.mark.gpu


def reference(args, rounds, spin_bits):
    r = REWL(*args, spin_bits=spin_bits)
    conv = r.run(rounds)
    m = args[4]
    return r.get("lng")[::m].copy(), r.get("mask").copy(), conv


def run_static(args, rounds, spin_bits):
    import torch

    lib = _lib.load()
    q, L, h, o, m, lnf_final, flat, K, seed = args
    p = _lib.Params(q, L, h, o, m, lnf_final, flat, K, seed)
    r = REWL(*args, spin_bits=spin_bits)  # only to learn W; not used for the run
    B = r.B
    r.close()
    lng = torch.full((h * B,), float("nan"), dtype=torch.float64, device="cuda")
    mask = torch.full((h * B,), 7, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    conv = C.c_int(-1)
    st = lib.rewl_run_static(C.byref(p), spin_bits, rounds, C.c_void_p(lng.data_ptr()),
                             C.c_void_p(mask.data_ptr()), h * B, C.byref(conv), None)
    _lib.check(st)
    return lng.cpu().numpy().reshape(h, B), mask.cpu().numpy().reshape(h, B), bool(conv.value)


@pytest.mark.parametrize("args,rounds,bits", [
    ((10, 12, 4, 0.75, 3, 1e-3, 0.8, 3000, 21), 15, 4),
    ((2, 8, 4, 0.75, 2, 1e-6, 0.8, 10_000, 1), 0, 8),   # the L=8 Ising workload, to convergence
])
def test_static_run_matches_allocating_path_twice(args, rounds, bits):
    want_lng, want_mask, want_conv = reference(args, rounds, bits)
    for _ in range(2):  # the second call starts from what the first left behind
        lng, mask, conv = run_static(args, rounds, bits)
        assert conv == want_conv
        assert np.array_equal(lng.view(np.uint64), want_lng.view(np.uint64))
        assert np.array_equal(mask, want_mask)


def test_static_run_after_a_larger_instance():
    big = (10, 40, 16, 0.75, 8, 1e-3, 0.8, 2000, 5)
    small = (3, 6, 3, 0.75, 2, 1e-3, 0.8, 500, 6)
    run_static(big, 3, 4)
    want_lng, want_mask, _ = reference(small, 10, 8)
    lng, mask, _ = run_static(small, 10, 8)
    assert np.array_equal(lng.view(np.uint64), want_lng.view(np.uint64))
    assert np.array_equal(mask, want_mask)


def test_static_run_rejects_instances_beyond_the_array():
    lib = _lib.load()
    # q=10, L=200, 64 windows of 4778 bins, 1024 walkers: ~60 MB of state
    p = _lib.Params(10, 200, 64, 0.75, 16, 1e-6, 0.8, 1000, 1)
    st = lib.rewl_run_static(C.byref(p), 0, 1, C.c_void_p(1), None, 64 * 4778, None, None)
    assert st == 1  # REWL_ERR_ARG, before any device work
    assert b"static scratch" in lib.rewl_last_error()
