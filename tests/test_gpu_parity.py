"""Parity of the CUDA path with the CPU oracle, element by element.

Both implement the same reading of Sec. 2 (arXiv:1312.3004) on the same
Philox4x32-10 streams, so spins, energies, replica ids, step counters, ln g
(bit for bit), histograms, masks and ln f must agree after every round.  A
difference is accepted only when it is traced (tests/tie_trace.py): inverting
near-tie decisions that the library logged (|u - exp(D)| < 1e-14, where exp of
two libraries may round the comparison differently) in a fresh oracle run must
reproduce the CUDA state exactly, and each such decision must be a near tie
for the oracle too.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1312_3004_gb300 import REWL, RewlError
from paper_1312_3004_gb300 import workloads as WL
from tie_trace import TracedPair, differing, gpu_state, gpu_ties, oracle_state, planted_near_tie

pytestmark = pytest.mark.gpu


def make_pair(q, L, h, o, m, lnf_final, flat, K, seed, spin_bits=0):
    gpu = REWL(q, L, h, o, m, lnf_final, flat, K, seed, spin_bits=spin_bits)
    orc = O.OracleREWL(q, L, h, o, m, lnf_final, flat, K, seed)
    return gpu, orc


def traced(q, L, h, o, m, lnf_final, flat, K, seed, spin_bits=0, options=()):
    """A TracedPair of a CUDA run (with the given rewl_set_option pairs) and the oracle."""
    def make_gpu():
        r = REWL(q, L, h, o, m, lnf_final, flat, K, seed, spin_bits=spin_bits)
        for opt, val in options:
            r.set_option(opt, val)
        return r
    return TracedPair(make_gpu, lambda: O.OracleREWL(q, L, h, o, m, lnf_final, flat, K, seed))


def assert_parity(gpu, orc):
    """Strict equality, for tests that steer both sides by hand (set fields):
    a difference there is reported with the library's near-tie log."""
    diff = differing(gpu_state(gpu), oracle_state(orc))
    assert not diff, "state differs in %s (near ties logged by the library: %s)" % (diff, gpu_ties(gpu))


def run_both(gpu, orc, rounds):
    gpu.run(rounds)
    orc.run(rounds)


SMALL = [
    # q, L, h, o, m, lnf_final, flatness, K, seed, spin_bits
    (2, 8, 4, 0.75, 2, 1e-6, 0.8, 10_000, 1, 8),     # 2D Ising L=8 workload
    (2, 8, 4, 0.75, 2, 1e-6, 0.8, 10_000, 1, 4),     # same, 4-bit packing
    (10, 20, 8, 0.75, 4, 1e-8, 0.8, 10_000, 3, 8),   # 10-state Potts L=20 workload
    (3, 5, 3, 0.75, 3, 1e-4, 0.8, 777, 5, 4),        # odd L, m = 3 (ragged merge tree)
    (10, 7, 2, 0.6, 5, 1e-4, 0.7, 1234, 6, 4),       # N = 49: packed tail word
    (4, 3, 1, 0.75, 1, 1e-3, 0.8, 500, 7, 8),        # smallest lattice, one window
    (16, 9, 5, 0.75, 33, 1e-3, 0.8, 300, 8, 4),      # q = 16 (4-bit max), m > 32
    (7, 6, 6, 0.8, 2, 1e-3, 0.8, 1, 9, 8),           # K = 1: exchange every step
]


@pytest.mark.parametrize("case", SMALL)
def test_initial_state_matches(case):
    *args, sb = case
    gpu, orc = make_pair(*args, spin_bits=sb)
    assert_parity(gpu, orc)


@pytest.mark.parametrize("case", SMALL)
def test_rounds_match_bit_for_bit(case):
    *args, sb = case
    tp = traced(*args, spin_bits=sb)
    for n in (1, 2, 5, 12):
        tp.run(n)


SWEEPS = [("reference", 1, 0), ("lanes1", 0, 1), ("lanes2", 0, 2), ("lanes4", 0, 4), ("lanes8", 0, 8),
          ("lanes16", 0, 16), ("lanes32", 0, 32)]


@pytest.mark.parametrize("sweep", SWEEPS, ids=[s[0] for s in SWEEPS])
@pytest.mark.parametrize("case", [SMALL[0], SMALL[2], SMALL[3], SMALL[4], SMALL[6]])
def test_every_sweep_variant_matches(case, sweep):
    """The binary64 reference sweep and the fast sweep at every lane-group
    width produce the oracle's states bit for bit."""
    from paper_1312_3004_gb300 import _lib
    *args, sb = case
    _, kind, lanes = sweep
    opts = [(_lib.OPT_SWEEP_KERNEL, kind)] + ([(_lib.OPT_LANES, lanes)] if kind == 0 else [])
    tp = traced(*args, spin_bits=sb, options=opts)
    for n in (1, 4, 10):
        tp.run(n)


@pytest.mark.parametrize("lanes", [1, 8, 32])
@pytest.mark.parametrize("case", [SMALL[0], SMALL[2], SMALL[4], SMALL[6]])
def test_lattices_in_global_memory_match(case, lanes):
    """The fast sweep with the lattices left in global memory (the placement
    for large lattices, forced here at small sizes) gives the same states."""
    from paper_1312_3004_gb300 import _lib
    *args, sb = case
    tp = traced(*args, spin_bits=sb, options=[(_lib.OPT_LATTICE, 1), (_lib.OPT_LANES, lanes)])
    assert tp.test.get_option(_lib.OPT_LATTICE) == 1
    for n in (1, 4, 10):
        tp.run(n)
    tp.test.set_option(_lib.OPT_LATTICE, 2)  # and back into shared memory mid-run
    assert tp.test.get_option(_lib.OPT_LATTICE) == 0
    tp.run(3)


def test_large_lattices_go_to_global_memory_and_match():
    """q=10, L=130 with 8-bit spins (16.9 KB lattices): the plan keeps them in
    global memory, with hashed conflict marks (N > 8192); rounds against the
    oracle."""
    from paper_1312_3004_gb300 import _lib
    tp = traced(10, 130, 8, 0.75, 1, 1e-6, 0.8, 2000, 3, spin_bits=8)
    assert tp.test.get_option(_lib.OPT_LATTICE) == 1
    for n in (1, 2):
        tp.run(n)


@pytest.mark.parametrize("lanes", [1, 8, 32])
def test_every_lane_width_converges_like_the_oracle(lanes):
    """Whole runs through many ln f halvings and merges (binade changes of ln g,
    exact-add fallbacks): identical final state for each lane-group width."""
    from paper_1312_3004_gb300 import _lib
    args = (3, 5, 3, 0.75, 3, 1e-4, 0.8, 777, 5)
    tp = traced(*args, spin_bits=4, options=[(_lib.OPT_LANES, lanes)])
    tp.run(0)
    assert tp.orc.all_done()


def test_first_million_updates_per_walker_ising_L8():
    """10^6 WL updates per walker (100 rounds of 10^4) on the L=8 Ising workload."""
    p = WL.params("ising_L8")
    for seed in (1, 2):
        tp = traced(*WL.rewl_args(p, seed), spin_bits=p["spin_bits"])
        tp.run(100)
        assert tp.orc.t().min() >= 10 ** 6 or tp.orc.all_done()


def test_first_million_updates_per_walker_potts10_L20():
    p = WL.params("potts10_L20")
    tp = traced(*WL.rewl_args(p, 1), spin_bits=p["spin_bits"])
    tp.run(100)


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_converged_ising_L8_matches_oracle(seed):
    """Full runs to ln f < 1e-6: identical joined ln g and identical state."""
    p = WL.params("ising_L8")
    tp = traced(*WL.rewl_args(p, seed), spin_bits=p["spin_bits"])
    tp.run(0)
    assert tp.orc.all_done()
    a, b = tp.test.lng(), tp.orc.lng_joined()
    fin = np.isfinite(b)
    assert np.array_equal(np.isfinite(a), fin)
    assert np.max(np.abs(a[fin] - b[fin])) <= 1e-12


def test_large_potts10_L80_first_rounds_match():
    """The 1024-walker q=10, L=80 workload in the launch configuration the
    benchmark uses: initial state and two rounds agree with the oracle."""
    p = WL.params("potts10_L80")
    tp = traced(*WL.rewl_args(p, 1), spin_bits=p["spin_bits"])
    tp.check()
    tp.run(2)


def test_rounds_after_convergence_change_nothing():
    gpu = REWL(2, 4, 2, 0.75, 2, 1e-2, 0.8, 2000, 3)
    assert gpu.run(0)
    before = {k: gpu.get(k) for k in ("lng", "spins", "hist", "round", "steps")}
    gpu.run(20)
    for k, v in before.items():
        assert np.array_equal(gpu.get(k), v)


def test_save_load_resume_is_bit_exact():
    args = (10, 12, 4, 0.75, 3, 1e-4, 0.8, 3000, 11)
    a = REWL(*args)
    a.run(10)
    blob = a.save()
    a.run(10)
    b = REWL(*args)
    b.load(blob)
    b.run(10)
    for k in ("lng", "spins", "hist", "mask", "lnf", "replica", "steps", "round"):
        assert np.array_equal(a.get(k), b.get(k)), k
    bad = bytearray(blob)
    bad[-1] ^= 0xFF
    with pytest.raises(RewlError):
        b.load(bytes(bad))
    c = REWL(10, 12, 4, 0.75, 3, 1e-4, 0.8, 3000, 12)  # other seed: other instance
    with pytest.raises(RewlError):
        c.load(blob)


def test_fixed_weights_flat_histogram_on_gpu():
    """ln g = exact ln g and ln f = 0: the GPU walker visits every reachable
    energy equally often, and agrees with the oracle step for step.  (Flatness
    0.999999 keeps the window from ever finishing its iteration.)  The top bin
    (proper 3-colourings) is left rarely, so its count has a long
    autocorrelation: 4e6 steps give a few per cent of noise there."""
    q, L = 3, 3
    ex = O.exact_lng(O.exact_counts_brute(q, L))
    gpu, orc = make_pair(q, L, 1, 0.75, 1, 1e-6, 0.999999, 100_000, 4)
    tab = np.where(np.isfinite(ex), ex, 0.0)[None, :]
    gpu.set("lng", tab)
    gpu.set("lnf", 0.0)
    orc.set_lng(tab)
    orc.set_lnf(0.0)
    run_both(gpu, orc, 40)
    assert_parity(gpu, orc)
    Hg = gpu.get("hist")[0]
    reach = np.isfinite(ex)
    hv = Hg[reach].astype(float)
    assert np.max(np.abs(hv / hv.mean() - 1)) < 0.1


def test_stats_count_every_proposal():
    gpu = REWL(5, 10, 4, 0.75, 3, 1e-6, 0.8, 2500, 2)
    gpu.run(6)
    s = gpu.stats()
    assert s["rounds"] == 6
    assert s["flips"] == 6 * 2500 * 12
    assert 0 < s["accepted"] <= s["flips"]
    assert s["exch_tried"] >= s["exch_accepted"]


def test_partial_results_and_state_errors():
    gpu = REWL(2, 8, 4, 0.75, 2, 1e-6, 0.8, 10_000, 1)
    gpu.run(3)
    with pytest.raises(RewlError):
        gpu.lng(partial=False)
    lg = gpu.lng(partial=True)
    assert np.isfinite(lg).sum() > 10


def test_spins_roundtrip_and_energy_recount():
    gpu = REWL(10, 11, 3, 0.75, 2, 1e-6, 0.8, 100, 5, spin_bits=4)
    s = gpu.get("spins")
    rng = np.random.default_rng(0)
    s2 = rng.integers(0, 10, s.shape).astype(np.uint8)
    gpu.set("spins", s2)
    assert np.array_equal(gpu.get("spins"), s2)
    E = gpu.get("energy")
    for g in range(s2.shape[0]):
        assert E[g] == O.energy(11, s2[g])


def test_many_walkers_run_a_thread_each_with_global_state():
    """Above 80 walkers per SM the plan maps a thread to each walker with its
    whole state in global memory; the states still match the oracle."""
    from paper_1312_3004_gb300 import _lib
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    m = 256
    h = max(2, (80 * sms) // m + 1)
    tp = traced(10, 12, h, 0.75, m, 1e-6, 0.8, 150, 21, spin_bits=8)
    assert tp.test.G > 80 * sms
    assert tp.test.get_option(_lib.OPT_LANES) == 1 and tp.test.get_option(_lib.OPT_LATTICE) == 1
    for n in (1, 2):
        tp.run(n)


def test_paper_size_workload_invariants():
    """q=10, L=300, 717 windows x 3 walkers (2151 walkers, 45 KB lattices in
    global memory), one round in the benchmark's configuration; too big for
    the oracle's window entry, so checked by what holds at any size: every
    energy is the recount of its lattice and lies in its walker's window, and
    with ln f = 1 and no merge yet, ln g equals the visit histogram bin by bin
    and both sum to K per walker."""
    from paper_1312_3004_gb300 import _lib
    p = WL.params("potts10_L300")
    r = REWL(*WL.rewl_args(p, 1), spin_bits=p["spin_bits"])
    assert r.get_option(_lib.OPT_LATTICE) == 1
    r.run(1)
    K = p["exchange_interval"]
    H = r.get("hist")
    lng = r.get("lng")
    assert np.array_equal(H.sum(axis=1), np.full(r.G, K))
    assert np.array_equal(lng, H.astype(np.float64))
    assert np.array_equal(r.get("steps"), np.full(r.G, K, dtype=np.uint64))
    E = r.get("energy")
    e_lo = r.get("e_lo")
    w = np.arange(r.G) // p["m"]
    assert np.all(E >= e_lo[w]) and np.all(E <= e_lo[w] + r.W)
    spins = r.get("spins")
    L = p["L"]
    for g in np.random.default_rng(3).choice(r.G, 24, replace=False):
        s = spins[g].reshape(L, L).astype(np.int32)
        recount = -int((s == np.roll(s, -1, axis=1)).sum() + (s == np.roll(s, -1, axis=0)).sum())
        assert recount == E[g], g


PLANT = (3, 5, 2, 0.75, 2, 1e-3, 0.8, 200, 11)  # q=3, L=5: 2 windows of 2 walkers


@pytest.mark.parametrize("sweep", [("reference", 1, 0), ("lanes1", 0, 1), ("lanes32", 0, 32)],
                         ids=["reference", "lanes1", "lanes32"])
def test_a_planted_near_tie_is_logged_and_traced(sweep):
    """ln g set so that the first proposal of one walker has exp(D) within
    1e-16 of its draw u: the library logs (WL step, walker, step 0), the
    oracle sees the same near tie, and the states agree or differ by exactly
    that decision, in every sweep variant."""
    from paper_1312_3004_gb300 import _lib
    seed = PLANT[-1]
    for g in range(4):
        if planted_near_tie(O.OracleREWL(*PLANT), seed, g):
            break
    else:
        pytest.skip("no walker's first proposal stays in its window")
    _, kind, lanes = sweep

    def make_gpu():
        r = REWL(*PLANT)
        r.set_option(_lib.OPT_SWEEP_KERNEL, kind)
        if kind == 0:
            r.set_option(_lib.OPT_LANES, lanes)
        planted_near_tie(O.OracleREWL(*PLANT), seed, g, setter=lambda lng: r.set("lng", lng))
        return r

    def make_orc():
        o = O.OracleREWL(*PLANT)
        planted_near_tie(o, seed, g)
        return o

    tp = TracedPair(make_gpu, make_orc)
    tp.run(1)
    n, log = gpu_ties(tp.test)
    assert n >= 1 and (0, g, 0) in log
    _, seen = tp.orc.ties()
    assert any(e[:3] == (0, g, 0) and e[3] < 1e-14 for e in seen)
    tp.run(3)


def test_a_planted_exchange_near_tie_is_logged():
    """Two windows of one walker each, both energies in the overlap: ln g of
    walker 0 set so that Eq. 1's ln ratio D of the round-0 exchange equals ln u
    of its draw.  The library logs (exchange, walker 0, round 0), the oracle
    sees the same near tie, and the replica ids agree or differ by that
    decision alone."""
    from paper_1312_3004_gb300 import _lib
    args = (3, 5, 2, 0.75, 1, 1e-3, 0.8, 200, 0)
    for seed in range(1, 40):
        a = args[:-1] + (seed,)
        o = O.OracleREWL(*a)
        E, lo, W = o.E(), o.e_lo(), o.W
        if E[0] != E[1] and lo[1] <= E[0] <= lo[0] + W and lo[0] <= E[1] <= lo[0] + W:
            break
    else:
        pytest.skip("no seed puts both walkers in the overlap")
    r = O.philox4x32_10([0, 0, 0, 4], [seed & 0xffffffff, seed >> 32])
    u = (((int(r[0]) >> 5) << 26) | (int(r[1]) >> 6)) * 2.0 ** -53
    lng = o.lng()
    lng[0, E[1] - lo[0]] = -np.log(u)  # D = (0 - ln g_0(E_1)) + 0 = ln u
    o.set_lng(lng)
    gpu = REWL(*a)
    gpu.set("lng", lng)
    gpu.run_phase(_lib.PHASE_EXCHANGE)
    gpu.sync()
    o.exchange()
    n, log = gpu_ties(gpu)
    assert n == 1 and log == [(1, 0, 0)]
    _, seen = o.ties()
    assert len(seen) == 1 and seen[0][:3] == (1, 0, 0) and seen[0][3] < 1e-14
    got, want = gpu.get("replica"), o.rep()
    if not np.array_equal(got, want):  # the two exps decided differently: the oracle's other choice
        o2 = O.OracleREWL(*a)
        o2.set_lng(lng)
        o2.invert_decision(1, 0, 0)
        o2.exchange()
        assert np.array_equal(got, o2.rep())


@pytest.mark.parametrize("case", [SMALL[0], SMALL[2], SMALL[6]])
def test_autotune_changes_no_result(case):
    """rewl_autotune times every lane width on ordinary rounds and keeps the
    fastest: the state afterwards is the oracle's after as many rounds."""
    from paper_1312_3004_gb300 import _lib
    *args, sb = case
    gpu, orc = make_pair(*args, spin_bits=sb)
    gpu.run(2)
    timed = gpu.autotune(1)
    assert len(timed) >= 1 and all(t["flips_per_s"] > 0 for t in timed)
    best = max(timed, key=lambda t: t["flips_per_s"])
    assert gpu.get_option(_lib.OPT_LANES) == best["lanes"]
    gpu.run(3)
    orc.run(gpu.round)
    assert_parity(gpu, orc)


@pytest.mark.parametrize("case", [
    (10, 1024, 2, 0.75, 1, 1e-6, 0.8, 500, 4, 8),     # the largest L: 2^20 sites, windows of 1.7e6 bins
    (200, 12, 3, 0.75, 2, 1e-3, 0.8, 2000, 5, 8),     # q far above 16: 8-bit spins only
    (2, 3, 1, 0.0, 1, 1e-3, 0.8, 1, 6, 8),            # the smallest lattice, no overlap, K = 1
])
def test_extreme_sizes_match(case):
    """Sizes at the edges of the interface: L = 1024 (the lane group's ln g
    shadow cannot fit in shared memory, so the plan falls back to a thread
    per walker with its state in global memory), q = 200, and L = 3 with one
    window, one walker and an exchange round after every step."""
    from paper_1312_3004_gb300 import _lib
    *args, sb = case
    tp = traced(*args, spin_bits=sb)
    if args[1] == 1024:
        assert tp.test.get_option(_lib.OPT_LANES) == 1 and tp.test.get_option(_lib.OPT_LATTICE) == 1
    for n in (1, 2):
        tp.run(n)
