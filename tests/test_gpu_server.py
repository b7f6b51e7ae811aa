"""Serving: jobs arrive while others run, are admitted as pool memory frees
up, run together with the batched kernels and retire on convergence.  Each
job's result must be exactly what the same job gives when run alone."""
import numpy as np
import pytest

from paper_1312_3004_gb300 import REWL, RewlError, Server

pytestmark = pytest.mark.gpu


def small_jobs():
    return [
        dict(q=2, L=8, h=4, overlap=0.75, m=2, lnf_final=1e-5, flatness=0.8, exchange_interval=5000, seed=1),
        dict(q=3, L=5, h=3, overlap=0.75, m=3, lnf_final=1e-4, flatness=0.8, exchange_interval=777, seed=5),
        dict(q=4, L=6, h=2, overlap=0.75, m=2, lnf_final=1e-4, flatness=0.8, exchange_interval=1000, seed=8),
        dict(q=2, L=8, h=4, overlap=0.75, m=2, lnf_final=1e-5, flatness=0.8, exchange_interval=5000, seed=2),
        dict(q=5, L=4, h=2, overlap=0.75, m=4, lnf_final=1e-4, flatness=0.8, exchange_interval=600, seed=13),
        dict(q=2, L=6, h=3, overlap=0.75, m=2, lnf_final=1e-5, flatness=0.8, exchange_interval=2000, seed=21),
    ]


def alone_result(j):
    r = REWL(j["q"], j["L"], j["h"], j["overlap"], j["m"], j["lnf_final"], j["flatness"],
             j["exchange_interval"], j["seed"])
    assert r.run(0)
    return r.lng()


def same(a, b):
    return np.array_equal(np.isfinite(a), np.isfinite(b)) and np.array_equal(a[np.isfinite(a)], b[np.isfinite(b)])


def test_staggered_arrivals_give_the_alone_results():
    jobs = small_jobs()
    srv = Server(pool_bytes=256 << 20, max_jobs=16)
    ids = {}
    tick = 0
    pending = list(range(len(jobs)))
    while pending or srv.info()["running"] or srv.info()["queued"]:
        if pending and tick % 3 == 0:  # a new arrival every third tick, while others run
            i = pending.pop(0)
            ids[i] = srv.submit(**jobs[i])
        srv.step(rounds=4)
        tick += 1
        assert tick < 100000
    for i, j in enumerate(jobs):
        assert srv.poll(ids[i]) == "done"
        assert same(srv.result(ids[i]), alone_result(j)), i
    info = srv.job_info(ids[0])
    assert info["t_submit"] <= info["t_admit"] <= info["t_done"] and info["rounds"] > 0


def test_small_pool_queues_until_memory_frees():
    jobs = small_jobs()
    probe = Server(pool_bytes=256 << 20, max_jobs=4)
    jid = probe.submit(**jobs[0])
    probe.step(1)
    one = probe.job_info(jid)["bytes"]
    probe.close()
    srv = Server(pool_bytes=2 * one + 1024, max_jobs=16)  # room for about two of the largest
    ids = [srv.submit(**j) for j in jobs]
    peak, waited = 0, 0
    for _ in range(100000):
        running, queued = srv.step(rounds=4)
        peak = max(peak, running)
        waited = max(waited, queued)
        if running == 0 and queued == 0:
            break
    assert waited > 0 and peak < len(jobs)  # admission really queued jobs
    for i, j in enumerate(jobs):
        assert srv.poll(ids[i]) == "done"
        assert same(srv.result(ids[i]), alone_result(j))


def test_cancel_and_errors():
    srv = Server(pool_bytes=64 << 20, max_jobs=2)
    j = small_jobs()[0]
    a = srv.submit(**j)
    b = srv.submit(**j)
    c = srv.submit(**j)  # waits: two slots
    srv.step(1)
    assert srv.poll(c) == "queued"
    srv.cancel(a)
    srv.cancel(c)
    assert srv.poll(a) == "cancelled" and srv.poll(c) == "cancelled"
    with pytest.raises(RewlError):
        srv.result(a)
    with pytest.raises(RewlError):
        srv.result(b)  # still running
    big = dict(j, L=200, h=4)
    with pytest.raises(RewlError):
        srv.submit(**big)  # larger than the pool


def test_release_forgets_finished_jobs():
    srv = Server(pool_bytes=64 << 20, max_jobs=4)
    j = small_jobs()[4]
    jid = srv.submit(**j)
    with pytest.raises(RewlError):
        srv.release(jid)  # queued: not finished
    ticks = 0
    while srv.poll(jid) != "done":
        srv.step(rounds=4)
        ticks += 1
        assert ticks < 100000
    assert same(srv.result(jid), alone_result(j))
    done_before = srv.info()["done"]
    srv.release(jid)
    assert srv.info()["done"] == done_before - 1
    with pytest.raises(RewlError):
        srv.poll(jid)  # the id is unknown now
    with pytest.raises(RewlError):
        srv.release(jid)
    other = srv.submit(**j)
    srv.cancel(other)
    srv.release(other)


def test_many_resident_walkers_switch_mapping_without_changing_results():
    """From 512 resident walkers on the server times lane groups against a
    thread per walker whenever the resident set changes by half, and keeps the
    faster; the jobs' results stay exactly their alone results and the states
    after a fixed number of rounds those of the same rounds alone."""
    jobs = [dict(q=10, L=12, h=16, overlap=0.75, m=8, lnf_final=1e-3, flatness=0.8, exchange_interval=500, seed=s)
            for s in range(1, 5)]  # 4 x 128 walkers
    srv = Server(pool_bytes=512 << 20, max_jobs=8)
    ids = [srv.submit(**j) for j in jobs]
    srv.step(rounds=3)
    lanes, tuned = srv.mapping()
    assert tuned == 512 and lanes in (1, 32)
    ticks = 0
    while srv.info()["running"]:
        srv.step(rounds=4)
        ticks += 1
        assert ticks < 100000
    for i, j in zip(ids, jobs):
        assert srv.poll(i) == "done"
        assert same(srv.result(i), alone_result(j))
