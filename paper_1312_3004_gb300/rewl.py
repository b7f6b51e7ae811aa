"""Python handle over the C ABI (include/rewl.h).

Marshalling only: every step of REWL (arXiv:1312.3004, Sec. 2) runs in the
CUDA library.  Host results come back as numpy arrays.
"""
import ctypes as C

import numpy as np

from . import _lib
from ._lib import check

_FIELD_DTYPES = {
    _lib.FIELD_SPINS: np.uint8, _lib.FIELD_ENERGY: np.int32, _lib.FIELD_REPLICA: np.uint32,
    _lib.FIELD_STEPS: np.uint64, _lib.FIELD_LNG: np.float64, _lib.FIELD_HIST: np.uint32,
    _lib.FIELD_MASK: np.uint8, _lib.FIELD_LNF: np.float64, _lib.FIELD_ITER: np.int32,
    _lib.FIELD_DONE: np.uint8, _lib.FIELD_ELO: np.int32, _lib.FIELD_ROUND: np.int64,
    _lib.FIELD_TRIPS: np.uint32, _lib.FIELD_TRIP_END: np.uint8, _lib.FIELD_PHASE: np.uint8,
    _lib.FIELD_TIES: np.uint64,
}
FIELDS = {"spins": _lib.FIELD_SPINS, "energy": _lib.FIELD_ENERGY, "replica": _lib.FIELD_REPLICA,
          "steps": _lib.FIELD_STEPS, "lng": _lib.FIELD_LNG, "hist": _lib.FIELD_HIST,
          "mask": _lib.FIELD_MASK, "lnf": _lib.FIELD_LNF, "iter": _lib.FIELD_ITER,
          "done": _lib.FIELD_DONE, "e_lo": _lib.FIELD_ELO, "round": _lib.FIELD_ROUND,
          "trips": _lib.FIELD_TRIPS, "trip_end": _lib.FIELD_TRIP_END, "phase": _lib.FIELD_PHASE,
          "ties": _lib.FIELD_TIES}


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


_allocator_refs = None  # keeps the callbacks alive while the library may call them


def set_allocator(alloc=None, free=None):
    """Device memory for the handles, batches and servers created from now on:
    alloc(nbytes) -> device pointer (int, 256-byte aligned) or 0; free(ptr).
    set_allocator() restores cudaMalloc.  Objects free through the allocator
    that gave them their memory."""
    global _allocator_refs
    L = _lib.load()
    if alloc is None:
        L.rewl_set_allocator(_lib.ALLOC_FN(), _lib.FREE_FN(), None)
        return
    a = _lib.ALLOC_FN(lambda n, ctx: alloc(n) or None)
    f = _lib.FREE_FN((lambda p, ctx: free(p)) if free else (lambda p, ctx: None))
    old = _allocator_refs
    _allocator_refs = (a, f, old)  # earlier callbacks stay alive for the objects that use them
    L.rewl_set_allocator(a, f, None)


class REWL:
    """One REWL instance on the current CUDA device.

    Parameters follow Sec. 2: q-state Potts on an L x L torus, h windows with
    overlap o, m walkers per window, stop at ln f < lnf_final, flatness p,
    K = exchange_interval WL steps per walker between exchanges, Philox seed.
    """

    def __init__(self, q, L, h, overlap, m, lnf_final, flatness, exchange_interval, seed,
                 spin_bits=0, stream=None, _view=None):
        self._L = _lib.load()
        self._owner = None
        if _view is not None:  # an instance owned by a Batch
            self._h, self._owner = _view
        else:
            self._h = C.c_void_p()
            p = _lib.Params(q, L, h, overlap, m, lnf_final, flatness, exchange_interval, seed)
            check(self._L.rewl_create_ext(C.byref(p), spin_bits, C.byref(self._h)))
        info = _lib.Info()
        check(self._L.rewl_get_info(self._h, C.byref(info)))
        self.q, self.L, self.h, self.m = q, L, h, m
        self.N, self.W, self.G = info.N, info.W, info.walkers
        self.B = self.W + 1
        self.spin_bits = info.spin_bits
        self.device_bytes = info.device_bytes
        if stream is not None:
            self.set_stream(stream)

    def close(self):
        if getattr(self, "_owner", None) is None and getattr(self, "_h", None) and self._h.value:
            self._L.rewl_destroy(self._h)
        self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
        raw = getattr(stream, "cuda_stream", stream)
        check(self._L.rewl_set_stream(self._h, C.c_void_p(raw) if raw else None))

    def run(self, max_rounds=0):
        conv = C.c_int(0)
        check(self._L.rewl_run(self._h, max_rounds, C.byref(conv)))
        return bool(conv.value)

    def run_async(self, rounds):
        check(self._L.rewl_run_async(self._h, rounds))

    def run_phase(self, phase):
        """Queue one phase (_lib.PHASE_SWEEP / PHASE_CHECK / PHASE_EXCHANGE)."""
        check(self._L.rewl_run_phase(self._h, phase))

    def set_option(self, option, value):
        check(self._L.rewl_set_option(self._h, option, value))

    def get_option(self, option):
        v = C.c_longlong(0)
        check(self._L.rewl_get_option(self._h, option, C.byref(v)))
        return v.value

    def sync(self):
        conv = C.c_int(0)
        check(self._L.rewl_sync(self._h, C.byref(conv)))
        return bool(conv.value)

    def lng(self, partial=False):
        out = np.zeros(2 * self.N + 1)
        check(self._L.rewl_get_lng(self._h, _ptr(out), out.size, 1 if partial else 0))
        return out

    def window_pieces(self):
        """(e_lo[h], W, ln g[h][W+1] of walker 0 of each window, mask[h][W+1]):
        the pieces rewl_join / rewl_bootstrap take."""
        return self.get("e_lo"), self.W, np.ascontiguousarray(self.get("lng")[::self.m]), self.get("mask")

    def window_lng(self, w):
        out = np.zeros(self.B)
        e = C.c_int(0)
        check(self._L.rewl_get_window_lng(self._h, w, _ptr(out), out.size, C.byref(e)))
        return out, e.value

    def stats(self):
        s = _lib.Stats()
        check(self._L.rewl_get_stats(self._h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in _lib.Stats._fields_}

    def _shape(self, field):
        G, B, h, N = self.G, self.B, self.h, self.N
        return {_lib.FIELD_SPINS: (G, N), _lib.FIELD_ENERGY: (G,), _lib.FIELD_REPLICA: (G,),
                _lib.FIELD_STEPS: (G,), _lib.FIELD_LNG: (G, B), _lib.FIELD_HIST: (G, B),
                _lib.FIELD_MASK: (h, B), _lib.FIELD_LNF: (h,), _lib.FIELD_ITER: (h,),
                _lib.FIELD_DONE: (h,), _lib.FIELD_ELO: (h,), _lib.FIELD_ROUND: (1,),
                _lib.FIELD_TRIPS: (G,), _lib.FIELD_TRIP_END: (G,), _lib.FIELD_PHASE: (h,),
                _lib.FIELD_TIES: (32, 2)}[field]

    def get(self, name):
        f = FIELDS[name]
        a = np.zeros(self._shape(f), dtype=_FIELD_DTYPES[f])
        check(self._L.rewl_get_field(self._h, f, _ptr(a), a.nbytes))
        return a

    def set(self, name, values):
        f = FIELDS[name]
        a = np.ascontiguousarray(np.broadcast_to(values, self._shape(f)), dtype=_FIELD_DTYPES[f])
        check(self._L.rewl_set_field(self._h, f, _ptr(a), a.nbytes))

    @property
    def round(self):
        return int(self.get("round")[0])

    def autotune(self, rounds=2):
        """Time the fast sweep's lane widths on the next rounds (rewl_autotune)
        and keep the fastest; returns the timed candidates."""
        ent = (_lib.TuneEntry * 8)()
        n = C.c_int(0)
        check(self._L.rewl_autotune(self._h, rounds, ent, 8, C.byref(n)))
        return [{k: getattr(ent[i], k) for k, _ in _lib.TuneEntry._fields_} for i in range(n.value)]

    def production_start(self, n_obins):
        """Fixed weights 1/g(E) from the current ln g (ln f = 0) and a histogram
        H(E, O) of the majority count in n_obins classes (Sec. 3.2)."""
        check(self._L.rewl_production_start(self._h, n_obins))
        self.n_obins = n_obins

    def production_run(self, rounds):
        check(self._L.rewl_production_run(self._h, rounds))

    def heo(self):
        """H(E, O) per window: uint64 [h][W + 1][n_obins]."""
        a = np.zeros((self.h, self.B, self.n_obins), dtype=np.uint64)
        check(self._L.rewl_production_histogram(self._h, _ptr(a), a.size))
        return a

    def save(self):
        n = C.c_size_t(0)
        check(self._L.rewl_save(self._h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        check(self._L.rewl_save(self._h, buf, C.byref(n)))
        return buf.raw[: n.value]

    def load(self, blob):
        buf = C.create_string_buffer(bytes(blob), len(blob))
        check(self._L.rewl_load(self._h, buf, len(blob)))


class Batch:
    """Many independent REWL instances advanced together (one persistent sweep
    launch, one batched check and one batched exchange launch per round).

    jobs: sequence of dicts with the REWL parameters (q, L, h, overlap, m,
    lnf_final, flatness, exchange_interval, seed).  Each instance computes the
    same states as it would alone.  lanes: 32 (lane groups, shared memory),
    1 (a thread per walker, state in global memory) or 0 (chosen by size).
    """

    def __init__(self, jobs, spin_bits=0, stream=None, lanes=0):
        self._L = _lib.load()
        self._h = C.c_void_p()
        self.jobs = [dict(j) for j in jobs]
        arr = (_lib.Params * len(self.jobs))()
        for i, j in enumerate(self.jobs):
            arr[i] = _lib.Params(j["q"], j["L"], j["h"], j["overlap"], j["m"], j["lnf_final"],
                                 j["flatness"], j["exchange_interval"], j["seed"])
        check(self._L.rewl_batch_create_ext(arr, len(self.jobs), spin_bits, lanes, C.byref(self._h)))
        if stream is not None:
            self.set_stream(stream)
        self._views = {}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            for v in self._views.values():
                v._h = C.c_void_p()
            self._L.rewl_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self):
        return len(self.jobs)

    def set_stream(self, stream):
        raw = getattr(stream, "cuda_stream", stream)
        check(self._L.rewl_batch_set_stream(self._h, C.c_void_p(raw) if raw else None))

    def run(self, max_rounds=0):
        n = C.c_int(0)
        check(self._L.rewl_batch_run(self._h, max_rounds, C.byref(n)))
        return n.value

    def run_async(self, rounds):
        check(self._L.rewl_batch_run_async(self._h, rounds))

    def sync(self):
        n = C.c_int(0)
        check(self._L.rewl_batch_sync(self._h, C.byref(n)))
        return n.value

    def autotune(self, rounds=2):
        """Time the batch's candidate configurations (rewl_batch_autotune) and
        keep the fastest: (list of timed candidates as dicts, from_cache)."""
        ent = (_lib.TuneEntry * 16)()
        n, cached = C.c_int(0), C.c_int(0)
        check(self._L.rewl_batch_autotune(self._h, rounds, ent, 16, C.byref(n), C.byref(cached)))
        return [{k: getattr(ent[i], k) for k, _ in _lib.TuneEntry._fields_} for i in range(n.value)], bool(cached.value)

    def config(self):
        """The batch's configuration: spin bits, lanes, CTA shared memory (KB) or threads per CTA."""
        v = [C.c_int(0) for _ in range(4)]
        check(self._L.rewl_batch_config(self._h, *[C.byref(x) for x in v]))
        return dict(zip(("spin_bits", "lanes", "cta_kb", "threads"), (x.value for x in v)))

    def instance(self, i):
        """Read-only REWL handle of instance i (owned by the batch)."""
        if i not in self._views:
            v = C.c_void_p()
            check(self._L.rewl_batch_instance(self._h, i, C.byref(v)))
            j = self.jobs[i]
            self._views[i] = REWL(j["q"], j["L"], j["h"], j["overlap"], j["m"], j["lnf_final"],
                                  j["flatness"], j["exchange_interval"], j["seed"], _view=(v, self))
        return self._views[i]

    def info(self):
        n, w, b = C.c_int(0), C.c_longlong(0), C.c_size_t(0)
        check(self._L.rewl_batch_info(self._h, C.byref(n), C.byref(w), C.byref(b)))
        return {"instances": n.value, "walkers": w.value, "device_bytes": b.value}

    def stats(self):
        s = _lib.Stats()
        check(self._L.rewl_batch_stats(self._h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in _lib.Stats._fields_}


JOB_STATES = {0: "queued", 1: "running", 2: "done", 3: "failed", 4: "cancelled"}


class Server:
    """Continuous batching of density-of-states jobs in a device memory pool
    (admission by footprint, resident state, retirement on convergence)."""

    def __init__(self, pool_bytes, max_jobs=256):
        self._L = _lib.load()
        self._h = C.c_void_p()
        check(self._L.rewl_server_create(int(pool_bytes), max_jobs, C.byref(self._h)))
        self._N = {}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._L.rewl_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, q, L, h, overlap, m, lnf_final, flatness, exchange_interval, seed, spin_bits=0):
        p = _lib.Params(q, L, h, overlap, m, lnf_final, flatness, exchange_interval, seed)
        jid = C.c_longlong(0)
        check(self._L.rewl_server_submit(self._h, C.byref(p), spin_bits, C.byref(jid)))
        self._N[jid.value] = L * L
        return jid.value

    def step(self, rounds=4):
        r, q = C.c_int(0), C.c_int(0)
        check(self._L.rewl_server_step(self._h, rounds, C.byref(r), C.byref(q)))
        return r.value, q.value

    def poll(self, job):
        st = C.c_int(0)
        check(self._L.rewl_server_poll(self._h, job, C.byref(st)))
        return JOB_STATES[st.value]

    def result(self, job):
        out = np.zeros(2 * self._N[job] + 1)
        check(self._L.rewl_server_result(self._h, job, _ptr(out), out.size))
        return out

    def job_info(self, job):
        t = np.zeros(3)
        c = np.zeros(3, dtype=np.int64)
        check(self._L.rewl_server_job_info(self._h, job, _ptr(t), _ptr(c)))
        return {"t_submit": t[0], "t_admit": t[1], "t_done": t[2], "rounds": int(c[0]), "flips": int(c[1]),
                "bytes": int(c[2])}

    def mapping(self):
        """(lanes, resident walkers when it was chosen): 32 lane groups or 1 thread per walker."""
        ln, w = C.c_int(0), C.c_longlong(0)
        check(self._L.rewl_server_mapping(self._h, C.byref(ln), C.byref(w)))
        return ln.value, w.value

    def cancel(self, job):
        check(self._L.rewl_server_cancel(self._h, job))

    def release(self, job):
        """Forget a finished (or failed / cancelled) job and its kept result."""
        check(self._L.rewl_server_release(self._h, job))

    def info(self):
        c = np.zeros(6, dtype=np.int64)
        f = C.c_size_t(0)
        check(self._L.rewl_server_info(self._h, _ptr(c), C.byref(f)))
        return {"queued": int(c[0]), "running": int(c[1]), "done": int(c[2]), "failed": int(c[3]),
                "rounds": int(c[4]), "flips": int(c[5]), "pool_free": f.value}


# ---- analysis of a joined ln g (host functions of the library) --------------
def _lng_arg(lng):
    return np.ascontiguousarray(lng, dtype=np.float64)


def canonical(lng, T):
    """Per-spin (u, c, f, s) at each temperature of T (Sec. 3.1, Fig. 3b)."""
    v = _lng_arg(lng)
    t = np.ascontiguousarray(np.atleast_1d(T), dtype=np.float64)
    out = np.zeros((t.size, 4))
    check(_lib.load().rewl_canonical(_ptr(v), v.size, _ptr(t), t.size, _ptr(out)))
    return out[:, 0].copy(), out[:, 1].copy(), out[:, 2].copy(), out[:, 3].copy()


def canonical_distribution(lng, T):
    """P(E) at T scaled to 1 at its highest point (Fig. 3b)."""
    v = _lng_arg(lng)
    out = np.zeros(v.size)
    check(_lib.load().rewl_canonical_distribution(_ptr(v), v.size, float(T), _ptr(out)))
    return out


def specific_heat_peak(lng, T_lo, T_hi):
    """(T, c) at the largest specific heat for T in [T_lo, T_hi]."""
    v = _lng_arg(lng)
    T, c = C.c_double(), C.c_double()
    check(_lib.load().rewl_specific_heat_peak(_ptr(v), v.size, float(T_lo), float(T_hi), C.byref(T), C.byref(c)))
    return T.value, c.value


def equal_peak_temperature(lng, T_lo, T_hi):
    """(Tc, E_low, E_high, ln suppression): the two equal canonical peaks of a
    first-order transition (Sec. 3.1)."""
    v = _lng_arg(lng)
    T, a, b, s = C.c_double(), C.c_int(), C.c_int(), C.c_double()
    check(_lib.load().rewl_equal_peak_temperature(_ptr(v), v.size, float(T_lo), float(T_hi), C.byref(T), C.byref(a),
                                                  C.byref(b), C.byref(s)))
    return T.value, a.value, b.value, s.value


def _pieces(e_lo, lng_w, mask_w):
    e = np.ascontiguousarray(e_lo, dtype=np.int32)
    return e, np.ascontiguousarray(lng_w, dtype=np.float64), np.ascontiguousarray(mask_w, dtype=np.uint8)


def join(q, L, e_lo, W, lng_w, mask_w):
    """Joined, normalised ln g from window pieces lng_w, mask_w of shape (h, W+1)."""
    e, lw, mw = _pieces(e_lo, lng_w, mask_w)
    out = np.zeros(2 * L * L + 1)
    check(_lib.load().rewl_join(q, L, e.size, W, _ptr(e), _ptr(lw), _ptr(mw), _ptr(out), out.size))
    return out


def bootstrap(q, L, e_lo, W, lng_runs, mask_runs, draws):
    """One joined, normalised ln g per row of draws: resample k averages the
    window pieces of runs draws[k] (arrays of shape (runs, h, W+1))."""
    e, lw, mw = _pieces(e_lo, lng_runs, mask_runs)
    d = np.ascontiguousarray(np.atleast_2d(draws), dtype=np.int32)
    runs = lw.shape[0]
    if d.shape[1] != runs or lw.shape != (runs, e.size, W + 1) or mw.shape != lw.shape:
        raise ValueError("pieces must be (runs, h, W+1) and every row of draws must name `runs` runs")
    out = np.zeros((d.shape[0], 2 * L * L + 1))
    check(_lib.load().rewl_bootstrap(q, L, e.size, W, _ptr(e), runs, _ptr(lw), _ptr(mw), d.shape[0], _ptr(d),
                                     _ptr(out), out.shape[1]))
    return out


def ising_energy(L, b):
    """Ising energy 2b - 2N of the bin with b broken bonds (q = 2)."""
    e = C.c_longlong()
    check(_lib.load().rewl_ising_energy(int(L), int(b), C.byref(e)))
    return e.value


def measure_pipes():
    """Issue rates of the WL step's pipes on the current device
    (rewl_measure_pipes): lane-operations per clock per SM of f64 add,
    32-bit multiply-add, high multiply, three-input logic, add and shared
    load, the latencies of the dependent f64 add, multiply-add and shared
    load in clocks, the SM count and the maximum SM clock (MHz)."""
    r = _lib.PipeRates()
    check(_lib.load().rewl_measure_pipes(C.byref(r)))
    return {k: getattr(r, k) for k, _ in _lib.PipeRates._fields_}
