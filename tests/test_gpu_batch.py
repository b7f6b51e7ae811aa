"""Batched instances: one persistent launch per round for many REWL instances
of uneven size.  Each instance must reach exactly the state it reaches alone
(same parameters and seed) -- batching changes the runtime, not the
arithmetic -- and the oracle's state as well."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1312_3004_gb300 import REWL, Batch, RewlError
from paper_1312_3004_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

FIELDS = ("spins", "energy", "replica", "steps", "lng", "hist", "mask", "lnf", "iter", "done", "round", "trips",
          "trip_end")


def jobs_mixed():
    return [
        dict(q=2, L=8, h=4, overlap=0.75, m=2, lnf_final=1e-6, flatness=0.8, exchange_interval=10_000, seed=1),
        dict(q=10, L=20, h=8, overlap=0.75, m=4, lnf_final=1e-8, flatness=0.8, exchange_interval=10_000, seed=3),
        dict(q=4, L=12, h=3, overlap=0.75, m=3, lnf_final=1e-4, flatness=0.8, exchange_interval=777, seed=5),
        dict(q=8, L=16, h=16, overlap=0.75, m=2, lnf_final=1e-6, flatness=0.8, exchange_interval=2000, seed=7),
        dict(q=3, L=5, h=2, overlap=0.75, m=1, lnf_final=1e-3, flatness=0.8, exchange_interval=500, seed=9),
        dict(q=10, L=40, h=4, overlap=0.75, m=4, lnf_final=1e-6, flatness=0.8, exchange_interval=3000, seed=11),
    ]


def alone(j, rounds):
    r = REWL(j["q"], j["L"], j["h"], j["overlap"], j["m"], j["lnf_final"], j["flatness"],
             j["exchange_interval"], j["seed"])
    r.run(rounds)
    return r


@pytest.mark.parametrize("lanes", [32, 1])
def test_batched_instances_equal_their_runs_alone(lanes):
    """Both mappings of walkers to threads: lane groups with shared-memory
    staging, and a thread per walker with every state in global memory."""
    jobs = jobs_mixed()
    b = Batch(jobs, lanes=lanes)
    assert b.info()["instances"] == len(jobs)
    for rounds in (1, 4, 9):
        b.run(rounds)
    for i, j in enumerate(jobs):
        a = alone(j, 14)
        v = b.instance(i)
        for f in FIELDS:
            assert np.array_equal(v.get(f), a.get(f)), (i, f)


@pytest.mark.parametrize("lanes", [32, 1])
def test_batched_instances_equal_the_oracle(lanes):
    jobs = jobs_mixed()[:5]
    b = Batch(jobs, lanes=lanes)
    b.run(6)
    for i, j in enumerate(jobs):
        orc = O.OracleREWL(*WL.rewl_args(j, j["seed"]))
        orc.run(6)
        v = b.instance(i)
        assert np.array_equal(v.get("spins"), orc.sigma())
        assert np.array_equal(v.get("lng").view(np.uint64), orc.lng().view(np.uint64))
        assert np.array_equal(v.get("hist"), orc.H())


def test_batch_runs_to_convergence_and_joins():
    jobs = [dict(q=2, L=8, h=4, overlap=0.75, m=2, lnf_final=1e-6, flatness=0.8, exchange_interval=10_000, seed=s)
            for s in (1, 2, 3)] + [dict(q=3, L=5, h=3, overlap=0.75, m=3, lnf_final=1e-4, flatness=0.8,
                                        exchange_interval=777, seed=5)]
    b = Batch(jobs)
    assert b.run(0) == len(jobs)
    for i, j in enumerate(jobs):
        orc = O.OracleREWL(*WL.rewl_args(j, j["seed"]))
        assert orc.run(0)
        lg = b.instance(i).lng()
        ref = orc.lng_joined()
        fin = np.isfinite(ref)
        assert np.array_equal(np.isfinite(lg), fin)
        assert np.max(np.abs(lg[fin] - ref[fin])) <= 1e-12
    s = b.stats()
    assert s["converged"] == 1 and s["windows_done"] == len(jobs)


def test_batch_views_are_read_only():
    b = Batch(jobs_mixed()[:2])
    v = b.instance(0)
    with pytest.raises(RewlError):
        v.run(1)
    with pytest.raises(RewlError):
        v.run_async(1)
    blob = v.save()
    v.load(blob)  # state access is allowed
    b.run(2)
    assert v.round == 2


def test_generated_batch_workload_builds():
    jobs = WL.batched_instances(64, master_seed=5)
    b = Batch(jobs)
    info = b.info()
    assert info["walkers"] == sum(j["h"] * j["m"] for j in jobs)
    b.run(2)
    assert b.stats()["flips"] == 2 * sum(j["h"] * j["m"] * j["exchange_interval"] for j in jobs)


def test_full_batched_workload_sampled_instances_match_the_oracle():
    """The full 2048-instance batch in the configuration the benchmark times
    (a thread per walker, 56,784 walkers): a sample of instances, each
    recomputed alone by the oracle, agrees bit for bit after two rounds."""
    jobs = WL.batched_instances(2048)
    b = Batch(jobs)
    assert b.info()["walkers"] >= 16384  # the thread-per-walker mapping
    b.run(2)
    rng = np.random.default_rng(11)
    for i in rng.choice(len(jobs), 6, replace=False):
        j = jobs[int(i)]
        orc = O.OracleREWL(*WL.rewl_args(j, j["seed"]))
        orc.run(2)
        v = b.instance(int(i))
        assert np.array_equal(v.get("spins"), orc.sigma()), i
        assert np.array_equal(v.get("lng").view(np.uint64), orc.lng().view(np.uint64)), i
        assert np.array_equal(v.get("hist"), orc.H()), i
        assert np.array_equal(v.get("replica"), orc.rep()), i
        assert np.array_equal(v.get("trips"), orc.rt_trips()), i


def test_autotuner_changes_no_result_and_caches_its_choice():
    """The autotuner runs ordinary rounds in every candidate configuration
    (spin packing 4 / 8 bits, lane groups with three CTA sizes, a thread per
    walker with two CTA sizes), repacking the spins in place between them; the
    instances must still equal their runs alone, and a second batch of the
    same jobs takes the cached choice without timing."""
    jobs = jobs_mixed()
    assert all(j["q"] <= 16 for j in jobs)  # packing free to change
    b = Batch(jobs)
    b.run(2)
    timed, cached = b.autotune(1)
    assert not cached and len(timed) >= 4
    assert {t["spin_bits"] for t in timed} == {4, 8} and {t["lanes"] for t in timed} == {1, 32}
    assert all(t["flips_per_s"] > 0 for t in timed)
    best = max(timed, key=lambda t: t["flips_per_s"])
    cfg = b.config()
    assert (cfg["spin_bits"], cfg["lanes"]) == (best["spin_bits"], best["lanes"])
    rounds = b.stats()["rounds"]
    b.run(3)
    for i, j in enumerate(jobs):
        a = alone(j, rounds + 3)
        v = b.instance(i)
        for f in FIELDS:
            assert np.array_equal(v.get(f), a.get(f)), (i, f)
    b2 = Batch(jobs)
    timed2, cached2 = b2.autotune(0)
    assert cached2 and timed2 == [] and b2.config() == cfg
