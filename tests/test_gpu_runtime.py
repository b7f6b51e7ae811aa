"""Runtime services around the hot path: device memory from a caller's
allocator (and what happens when it fails), and the stall watchdog of
rewl_run.  Failures are made on the host: an allocator that returns NULL, a
run whose windows can never become flat."""
import time

import numpy as np
import pytest

from paper_1312_3004_gb300 import REWL, Batch, RewlError, Server, _lib
from paper_1312_3004_gb300 import rewl as R

pytestmark = pytest.mark.gpu

ARGS = (10, 12, 4, 0.75, 3, 1e-4, 0.8, 3000, 11)
SMALL_JOB = dict(q=2, L=8, h=4, overlap=0.75, m=2, lnf_final=1e-6, flatness=0.8, exchange_interval=1000, seed=1)


def test_allocation_failure_is_reported_by_every_creator():
    calls = []
    R.set_allocator(lambda n: calls.append(n) or 0, None)  # every request fails
    try:
        with pytest.raises(RewlError) as e:
            REWL(*ARGS)
        assert e.value.status == 2  # REWL_ERR_NOMEM
        with pytest.raises(RewlError) as e:
            Batch([SMALL_JOB])
        assert e.value.status == 2
        with pytest.raises(RewlError) as e:
            Server(pool_bytes=1 << 20, max_jobs=2)
        assert e.value.status == 2
        assert len(calls) >= 3
    finally:
        R.set_allocator()
    r = REWL(*ARGS)  # cudaMalloc again
    r.run(2)


def test_caching_allocator_of_torch_supplies_the_state():
    torch = pytest.importorskip("torch")
    live = {}

    def alloc(n):
        p = torch.cuda.caching_allocator_alloc(n)
        live[p] = n
        return p

    def free(p):
        live.pop(p)
        torch.cuda.caching_allocator_delete(p)

    R.set_allocator(alloc, free)
    try:
        a = REWL(*ARGS)
        bt = Batch([SMALL_JOB, dict(SMALL_JOB, seed=2)])
    finally:
        R.set_allocator()
    assert len(live) == 3  # the handle's state; the batch's state and its configuration tables
    b = REWL(*ARGS)
    a.run(5)
    b.run(5)
    for k in ("lng", "spins", "hist", "trips"):
        assert np.array_equal(a.get(k), b.get(k)), k
    bt.run(3)
    a.close()
    bt.close()
    assert not live  # returned through the allocator that gave it


def test_stall_watchdog_stops_a_run_that_makes_no_progress():
    r = REWL(10, 12, 4, 0.75, 3, 1e-4, 0.999999, 3000, 11)  # flatness 0.999999: no window ever flat
    r.set_option(_lib.OPT_STALL_MS, 200)
    assert r.get_option(_lib.OPT_STALL_MS) == 200
    t0 = time.perf_counter()
    with pytest.raises(RewlError) as e:
        r.run(0)  # until converged: never, so only the watchdog can end it
    assert e.value.status == 4  # REWL_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 60
    rounds = r.stats()["rounds"]
    r.set_option(_lib.OPT_STALL_MS, 0)
    r.run(3)  # the state stays usable and the run goes on
    assert r.stats()["rounds"] == rounds + 3
