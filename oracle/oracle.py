"""ctypes front end of the CPU oracle (oracle/rewl_oracle.c, oracle/exact_dos.c).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the
benchmark's CPU-baseline leg use it to produce the values the CUDA path must
reproduce.  Nothing in the product library imports it.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        vp, i32, i64, u64, dbl = C.c_void_p, C.c_int, C.c_int64, C.c_uint64, C.c_double
        L.orc_philox4x32_10.argtypes = [vp, vp, vp]
        L.orc_philox4x32_10.restype = None
        L.orc_window_table.argtypes = [i32, i32, dbl, vp, vp]
        L.orc_window_table.restype = i32
        L.orc_energy.argtypes = [i32, vp]
        L.orc_energy.restype = C.c_int32
        L.orc_create.argtypes = [i32, i32, i32, dbl, i32, dbl, dbl, i64, u64, C.POINTER(C.c_int)]
        L.orc_create.restype = vp
        L.orc_destroy.argtypes = [vp]
        L.orc_destroy.restype = None
        L.orc_wl_steps.argtypes = [vp, i32, i64]
        L.orc_wl_steps.restype = None
        L.orc_sweep.argtypes = [vp]
        L.orc_sweep.restype = None
        L.orc_tree_mean.argtypes = [vp, i32]
        L.orc_tree_mean.restype = dbl
        for name in ("orc_update_mask", "orc_window_iterations", "orc_exchange"):
            getattr(L, name).argtypes = [vp]
            getattr(L, name).restype = None
        L.orc_walker_flat.argtypes = [vp, i32]
        L.orc_walker_flat.restype = i32
        L.orc_barrier.argtypes = [vp]
        L.orc_barrier.restype = i32
        L.orc_all_done.argtypes = [vp]
        L.orc_all_done.restype = i32
        L.orc_run.argtypes = [vp, i64, C.POINTER(C.c_int)]
        L.orc_run.restype = i32
        L.orc_join_pieces.argtypes = [i32, i32, i32, vp, vp, vp, vp]
        L.orc_join_pieces.restype = i32
        L.orc_normalise.argtypes = [i32, i32, vp, i32]
        L.orc_normalise.restype = None
        L.orc_get_lng_joined.argtypes = [vp, vp]
        L.orc_get_lng_joined.restype = i32
        L.orc_dims.argtypes = [vp, vp]
        L.orc_dims.restype = None
        for name in ("orc_get_e_lo", "orc_get_sigma", "orc_get_E", "orc_get_rep", "orc_get_t",
                     "orc_get_lng", "orc_get_H", "orc_get_mask", "orc_get_lnf", "orc_get_iter",
                     "orc_get_done", "orc_get_xstats", "orc_get_rt_end", "orc_get_rt_trips", "orc_get_phase",
                     "orc_set_lng", "orc_set_lnf", "orc_set_H",
                     "orc_set_mask"):
            getattr(L, name).argtypes = [vp, vp]
            getattr(L, name).restype = None
        L.orc_set_config.argtypes = [vp, i32, vp]
        L.orc_set_config.restype = None
        L.orc_set_round.argtypes = [vp, i64]
        L.orc_set_round.restype = None
        L.orc_set_schedule.argtypes = [vp, i32]
        L.orc_set_schedule.restype = None
        L.orc_production_start.argtypes = [vp, i32]
        L.orc_production_start.restype = i32
        L.orc_production_run.argtypes = [vp, i64]
        L.orc_production_run.restype = i32
        L.orc_get_heo.argtypes = [vp, vp]
        L.orc_get_heo.restype = None
        L.orc_majority.argtypes = [vp, i32, i32]
        L.orc_majority.restype = i32
        L.orc_obin.argtypes = [i32, i32, i32, i32]
        L.orc_obin.restype = i32
        L.orc_walker_visited_all.argtypes = [vp, i32]
        L.orc_walker_visited_all.restype = i32
        L.orc_invert_decision.argtypes = [vp, i32, u64, u64]
        L.orc_invert_decision.restype = i32
        L.orc_get_decision_counts.argtypes = [vp, vp]
        L.orc_get_decision_counts.restype = None
        L.orc_get_ties.argtypes = [vp, vp, vp, i32]
        L.orc_get_ties.restype = i64
        L.ex_brute_force.argtypes = [i32, i32, vp]
        L.ex_brute_force.restype = i32
        L.ex_transfer_matrix.argtypes = [i32, i32, i32, vp, vp]
        L.ex_transfer_matrix.restype = i32
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    """One Philox4x32-10 block: ctr = 4 uint32 words, key = 2 uint32 words."""
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def window_table(L, h, overlap):
    """(e_lo[h], W): window i spans energies e_lo[i] .. e_lo[i] + W."""
    e_lo = np.zeros(h, dtype=np.int32)
    W = np.zeros(1, dtype=np.int32)
    if lib().orc_window_table(L, h, overlap, _ptr(e_lo), _ptr(W)):
        raise ValueError("invalid window geometry")
    return e_lo, int(W[0])


def energy(L, sigma):
    s = np.ascontiguousarray(sigma, dtype=np.uint8)
    return int(lib().orc_energy(L, _ptr(s)))


def tree_mean(values):
    v = np.ascontiguousarray(values, dtype=np.float64)
    return float(lib().orc_tree_mean(_ptr(v), len(v)))


def join_pieces(N, e_lo, W, lng_w, mask_w):
    e = np.ascontiguousarray(e_lo, dtype=np.int32)
    lw = np.ascontiguousarray(lng_w, dtype=np.float64)
    mw = np.ascontiguousarray(mask_w, dtype=np.uint8)
    out = np.zeros(2 * N + 1)
    st = lib().orc_join_pieces(N, len(e), W, _ptr(e), _ptr(lw), _ptr(mw), _ptr(out))
    if st:
        raise RuntimeError("join failed (%d)" % st)
    return out


def normalise(q, N, lng):
    v = np.ascontiguousarray(lng, dtype=np.float64).copy()
    lib().orc_normalise(q, N, _ptr(v), len(v))
    return v


# ---------------------------------------------------------------------------
def exact_counts_brute(q, L):
    N = L * L
    out = np.zeros(2 * N + 1, dtype=np.uint64)
    if lib().ex_brute_force(q, L, _ptr(out)):
        raise ValueError("too large for brute force")
    return [int(x) for x in out]


def exact_counts_tm(q, L, symmetry=True):
    N = L * L
    hi = np.zeros(2 * N + 1, dtype=np.uint64)
    lo = np.zeros(2 * N + 1, dtype=np.uint64)
    if lib().ex_transfer_matrix(q, L, 1 if symmetry else 0, _ptr(hi), _ptr(lo)):
        raise ValueError("too large for the transfer matrix")
    return [(int(a) << 64) | int(b) for a, b in zip(hi, lo)]


def exact_lng(counts):
    """ln g(b) for b = 0..2N from exact integer counts (-inf where g = 0)."""
    import math
    return np.array([math.log(c) if c > 0 else -np.inf for c in counts])


# ---------------------------------------------------------------------------
class OracleREWL:
    """One REWL run of the oracle; arrays are copied out on request."""

    def __init__(self, q, L, h, overlap, m, lnf_final, flatness, K, seed):
        st = C.c_int(0)
        self._h = lib().orc_create(q, L, h, overlap, m, lnf_final, flatness, K, seed, C.byref(st))
        if not self._h:
            raise ValueError("orc_create failed with status %d" % st.value)
        d = self.dims()
        self.q, self.L, self.N, self.h, self.m, self.W, self.K = d[:7]
        self.B = self.W + 1
        self.G = self.h * self.m

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_destroy(self._h)
            self._h = None

    def dims(self):
        d = np.zeros(8, dtype=np.int64)
        lib().orc_dims(self._h, _ptr(d))
        return [int(x) for x in d]

    @property
    def round(self):
        return self.dims()[7]

    def _get(self, name, shape, dtype):
        a = np.zeros(shape, dtype=dtype)
        getattr(lib(), name)(self._h, _ptr(a))
        return a

    def e_lo(self): return self._get("orc_get_e_lo", self.h, np.int32)
    def sigma(self): return self._get("orc_get_sigma", (self.G, self.N), np.uint8)
    def E(self): return self._get("orc_get_E", self.G, np.int32)
    def rep(self): return self._get("orc_get_rep", self.G, np.uint32)
    def t(self): return self._get("orc_get_t", self.G, np.uint64)
    def lng(self): return self._get("orc_get_lng", (self.G, self.B), np.float64)
    def H(self): return self._get("orc_get_H", (self.G, self.B), np.uint32)
    def mask(self): return self._get("orc_get_mask", (self.h, self.B), np.uint8)
    def lnf(self): return self._get("orc_get_lnf", self.h, np.float64)
    def iter(self): return self._get("orc_get_iter", self.h, np.int32)
    def done(self): return self._get("orc_get_done", self.h, np.uint8)
    def xstats(self): return self._get("orc_get_xstats", 2, np.uint64)
    def rt_end(self): return self._get("orc_get_rt_end", self.G, np.uint8)
    def rt_trips(self): return self._get("orc_get_rt_trips", self.G, np.uint32)
    def phase(self): return self._get("orc_get_phase", self.h, np.uint8)

    # Decisions are named (kind, who, when): kind 0 a WL step of walker `who` at
    # its step index `when`; kind 1 the exchange of the pair whose lower-window
    # walker is `who`, in round `when`.
    def invert_decision(self, kind, who, when):
        """Invert one acceptance decision when it comes up (test support: to
        reproduce what another implementation decided at a near tie)."""
        if lib().orc_invert_decision(self._h, kind, who, when):
            raise ValueError("too many inverted decisions")

    def ties(self):
        """(count, [(kind, who, when, |u - exp(D)|), ...]) of the draws with
        |u - exp(D)| < 1e-12 so far (the first 64 are listed)."""
        ent = np.zeros((64, 3), dtype=np.uint64)
        gap = np.zeros(64)
        n = int(lib().orc_get_ties(self._h, _ptr(ent), _ptr(gap), 64))
        k = min(n, 64)
        return n, [(int(a), int(b), int(c), float(d)) for (a, b, c), d in zip(ent[:k], gap[:k])]

    def decision_counts(self):
        """(WL decisions made, of which with D < 0): the proposals inside the
        window, and those whose acceptance needed exp(D)."""
        c = np.zeros(2, dtype=np.int64)
        lib().orc_get_decision_counts(self._h, _ptr(c))
        return int(c[0]), int(c[1])

    def set_schedule(self, schedule):
        """0: ln f halves per iteration (Sec. 2); 1: the 1/t rule."""
        lib().orc_set_schedule(self._h, schedule)

    def walker_visited_all(self, g):
        return bool(lib().orc_walker_visited_all(self._h, g))

    def production_start(self, n_obins):
        """Fixed weights from here on (ln f = 0), H(E,O) kept in n_obins classes."""
        if lib().orc_production_start(self._h, n_obins):
            raise ValueError("n_obins outside [1, N - ceil(N/q) + 1]")
        self.n_obins = n_obins

    def production_run(self, rounds):
        if lib().orc_production_run(self._h, rounds):
            raise RuntimeError("not in production")

    def heo(self):
        return self._get("orc_get_heo", (self.h, self.B, self.n_obins), np.uint64)

    def set_lng(self, v):
        a = np.ascontiguousarray(np.broadcast_to(v, (self.G, self.B)), dtype=np.float64)
        lib().orc_set_lng(self._h, _ptr(a))

    def set_lnf(self, v):
        a = np.ascontiguousarray(np.broadcast_to(v, (self.h,)), dtype=np.float64)
        lib().orc_set_lnf(self._h, _ptr(a))

    def set_H(self, v):
        a = np.ascontiguousarray(np.broadcast_to(v, (self.G, self.B)), dtype=np.uint32)
        lib().orc_set_H(self._h, _ptr(a))

    def set_mask(self, v):
        a = np.ascontiguousarray(np.broadcast_to(v, (self.h, self.B)), dtype=np.uint8)
        lib().orc_set_mask(self._h, _ptr(a))

    def set_config(self, g, sigma):
        s = np.ascontiguousarray(sigma, dtype=np.uint8)
        lib().orc_set_config(self._h, g, _ptr(s))

    def set_round(self, r):
        lib().orc_set_round(self._h, r)

    def wl_steps(self, g, n):
        lib().orc_wl_steps(self._h, g, n)

    def sweep(self):
        lib().orc_sweep(self._h)

    def update_mask(self):
        lib().orc_update_mask(self._h)

    def walker_flat(self, g):
        return bool(lib().orc_walker_flat(self._h, g))

    def window_iterations(self):
        lib().orc_window_iterations(self._h)

    def exchange(self):
        lib().orc_exchange(self._h)

    def barrier(self):
        st = lib().orc_barrier(self._h)
        if st:
            raise RuntimeError("barrier status %d" % st)

    def all_done(self):
        return bool(lib().orc_all_done(self._h))

    def run(self, max_rounds=0):
        conv = C.c_int(0)
        st = lib().orc_run(self._h, max_rounds, C.byref(conv))
        if st:
            raise RuntimeError("orc_run status %d" % st)
        return bool(conv.value)

    def lng_joined(self):
        out = np.zeros(2 * self.N + 1)
        st = lib().orc_get_lng_joined(self._h, _ptr(out))
        if st:
            raise RuntimeError("join status %d" % st)
        return out


def majority(sigma, q):
    s = np.ascontiguousarray(sigma, dtype=np.uint8)
    return int(lib().orc_majority(_ptr(s), s.size, q))


def obin(n_max, N, q, n_obins):
    return int(lib().orc_obin(n_max, N, q, n_obins))
