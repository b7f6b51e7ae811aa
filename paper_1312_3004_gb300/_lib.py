"""ctypes declarations of the C ABI in include/rewl.h (argument marshalling only).

The shared library is the CUDA implementation; there is no CPU fallback.  If
librewl.so has not been built, load() raises instead of degrading silently.
"""
import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "librewl.so")
# REWL_DEBUG=1 selects the build with the kernels' bounds checks (build.build(debug=True)).
LIB_DEBUG_PATH = os.path.join(HERE, "_build", "librewl_debug.so")

REWL_OK = 0
STATUS_NAMES = {0: "REWL_OK", 1: "REWL_ERR_ARG", 2: "REWL_ERR_NOMEM", 3: "REWL_ERR_CUDA",
                4: "REWL_ERR_TIMEOUT", 5: "REWL_ERR_OVERFLOW", 6: "REWL_ERR_STATE",
                7: "REWL_ERR_CANCELLED"}

FIELD_SPINS, FIELD_ENERGY, FIELD_REPLICA, FIELD_STEPS, FIELD_LNG, FIELD_HIST = 0, 1, 2, 3, 4, 5
PHASE_SWEEP, PHASE_CHECK, PHASE_EXCHANGE = 0, 1, 2
OPT_SWEEP_KERNEL, OPT_LANES, OPT_WALKERS_PER_CTA, OPT_LATTICE, OPT_STALL_MS, OPT_SCHEDULE = 0, 1, 2, 3, 4, 5
SCHEDULE_HALVING, SCHEDULE_INV_T = 0, 1
FIELD_MASK, FIELD_LNF, FIELD_ITER, FIELD_DONE, FIELD_ELO, FIELD_ROUND = 6, 7, 8, 9, 10, 11
FIELD_TRIPS, FIELD_TRIP_END, FIELD_PHASE, FIELD_TIES = 12, 13, 14, 15


class RewlError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), message))
        self.status = status


class Params(C.Structure):
    _fields_ = [("q", C.c_int), ("L", C.c_int), ("h", C.c_int), ("overlap", C.c_double),
                ("m", C.c_int), ("lnf_final", C.c_double), ("flatness", C.c_double),
                ("exchange_interval", C.c_longlong), ("seed", C.c_ulonglong)]


class Info(C.Structure):
    _fields_ = [("N", C.c_int), ("W", C.c_int), ("walkers", C.c_int), ("spin_bits", C.c_int),
                ("device_bytes", C.c_size_t)]


class PipeRates(C.Structure):
    _fields_ = [("dadd", C.c_double), ("imad", C.c_double), ("imad_hi", C.c_double), ("lop3", C.c_double),
                ("iadd", C.c_double), ("lds", C.c_double), ("dadd_latency", C.c_double),
                ("imad_latency", C.c_double), ("lds_latency", C.c_double), ("sms", C.c_int),
                ("max_clock_mhz", C.c_double)]


class TuneEntry(C.Structure):
    _fields_ = [("spin_bits", C.c_int), ("lanes", C.c_int), ("cta_kb", C.c_int), ("threads", C.c_int),
                ("flips_per_s", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("rounds", C.c_longlong), ("flips", C.c_longlong), ("accepted", C.c_longlong),
                ("exch_tried", C.c_longlong), ("exch_accepted", C.c_longlong),
                ("near_ties", C.c_longlong), ("slow_decisions", C.c_longlong),
                ("seq_steps", C.c_longlong), ("windows_done", C.c_int), ("converged", C.c_int),
                ("min_lnf", C.c_double), ("max_lnf", C.c_double)]


_lib = None

# rewl_set_allocator callbacks: alloc(bytes, ctx) -> device pointer or NULL; free(ptr, ctx)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


def load():
    """Load librewl.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = LIB_DEBUG_PATH if os.environ.get("REWL_DEBUG") == "1" else LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("%s is not built; run __graft_entry__.build() (or build.build(debug=True)) first" % path)
    L = C.CDLL(path)
    vp, i32, ll, sz, dbl = C.c_void_p, C.c_int, C.c_longlong, C.c_size_t, C.c_double
    H = C.c_void_p
    st = C.c_int
    L.rewl_create.argtypes = [i32, i32, i32, dbl, i32, dbl, dbl, ll, C.c_ulonglong, C.POINTER(H)]
    L.rewl_create_ext.argtypes = [C.POINTER(Params), i32, C.POINTER(H)]
    L.rewl_set_allocator.argtypes = [ALLOC_FN, FREE_FN, vp]
    L.rewl_set_allocator.restype = None
    L.rewl_set_stream.argtypes = [H, vp]
    L.rewl_run.argtypes = [H, ll, C.POINTER(C.c_int)]
    L.rewl_run_async.argtypes = [H, ll]
    L.rewl_sync.argtypes = [H, C.POINTER(C.c_int)]
    L.rewl_run_phase.argtypes = [H, i32]
    L.rewl_set_option.argtypes = [H, i32, ll]
    L.rewl_get_option.argtypes = [H, i32, C.POINTER(C.c_longlong)]
    L.rewl_get_lng.argtypes = [H, vp, sz, i32]
    L.rewl_get_window_lng.argtypes = [H, i32, vp, sz, C.POINTER(C.c_int)]
    L.rewl_get_info.argtypes = [H, C.POINTER(Info)]
    L.rewl_get_stats.argtypes = [H, C.POINTER(Stats)]
    L.rewl_get_field.argtypes = [H, i32, vp, sz]
    L.rewl_set_field.argtypes = [H, i32, vp, sz]
    L.rewl_save.argtypes = [H, vp, C.POINTER(sz)]
    L.rewl_load.argtypes = [H, vp, sz]
    for name in ("rewl_create", "rewl_create_ext", "rewl_set_stream", "rewl_run", "rewl_run_async",
                 "rewl_sync", "rewl_run_phase", "rewl_set_option", "rewl_get_option", "rewl_get_lng", "rewl_get_window_lng", "rewl_get_info",
                 "rewl_get_stats", "rewl_get_field", "rewl_set_field", "rewl_save", "rewl_load"):
        getattr(L, name).restype = st
    L.rewl_run_static.argtypes = [C.POINTER(Params), i32, ll, vp, vp, sz, C.POINTER(C.c_int), vp]
    L.rewl_run_static.restype = st
    L.rewl_batch_create.argtypes = [C.POINTER(Params), i32, i32, C.POINTER(H)]
    L.rewl_batch_create_ext.argtypes = [C.POINTER(Params), i32, i32, i32, C.POINTER(H)]
    L.rewl_batch_run.argtypes = [H, ll, C.POINTER(C.c_int)]
    L.rewl_batch_run_async.argtypes = [H, ll]
    L.rewl_batch_sync.argtypes = [H, C.POINTER(C.c_int)]
    L.rewl_batch_set_stream.argtypes = [H, vp]
    L.rewl_batch_instance.argtypes = [H, i32, C.POINTER(H)]
    L.rewl_batch_info.argtypes = [H, C.POINTER(C.c_int), C.POINTER(C.c_longlong), C.POINTER(C.c_size_t)]
    L.rewl_batch_stats.argtypes = [H, C.POINTER(Stats)]
    L.rewl_batch_autotune.argtypes = [H, i32, C.POINTER(TuneEntry), i32, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.rewl_batch_autotune.restype = st
    L.rewl_server_mapping.argtypes = [H, C.POINTER(C.c_int), C.POINTER(C.c_longlong)]
    L.rewl_server_mapping.restype = st
    L.rewl_autotune.argtypes = [H, i32, C.POINTER(TuneEntry), i32, C.POINTER(C.c_int)]
    L.rewl_autotune.restype = st
    L.rewl_batch_config.argtypes = [H] + [C.POINTER(C.c_int)] * 4
    L.rewl_batch_config.restype = st
    for name in ("rewl_batch_create", "rewl_batch_create_ext", "rewl_batch_run", "rewl_batch_run_async", "rewl_batch_sync",
                 "rewl_batch_set_stream", "rewl_batch_instance", "rewl_batch_info", "rewl_batch_stats"):
        getattr(L, name).restype = st
    L.rewl_server_create.argtypes = [sz, i32, C.POINTER(H)]
    L.rewl_server_submit.argtypes = [H, C.POINTER(Params), i32, C.POINTER(C.c_longlong)]
    L.rewl_server_step.argtypes = [H, ll, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.rewl_server_poll.argtypes = [H, ll, C.POINTER(C.c_int)]
    L.rewl_server_result.argtypes = [H, ll, vp, sz]
    L.rewl_server_job_info.argtypes = [H, ll, vp, vp]
    L.rewl_server_cancel.argtypes = [H, ll]
    L.rewl_server_release.argtypes = [H, ll]
    L.rewl_server_info.argtypes = [H, vp, C.POINTER(C.c_size_t)]
    for name in ("rewl_server_create", "rewl_server_submit", "rewl_server_step", "rewl_server_poll",
                 "rewl_server_result", "rewl_server_job_info", "rewl_server_cancel", "rewl_server_release",
                 "rewl_server_info"):
        getattr(L, name).restype = st
    L.rewl_server_destroy.argtypes = [H]
    L.rewl_server_destroy.restype = None
    L.rewl_batch_destroy.argtypes = [H]
    L.rewl_batch_destroy.restype = None
    L.rewl_destroy.argtypes = [H]
    L.rewl_destroy.restype = None
    pi = C.POINTER(C.c_int)
    pd = C.POINTER(C.c_double)
    L.rewl_canonical.argtypes = [vp, sz, vp, sz, vp]
    L.rewl_canonical_distribution.argtypes = [vp, sz, C.c_double, vp]
    L.rewl_specific_heat_peak.argtypes = [vp, sz, C.c_double, C.c_double, pd, pd]
    L.rewl_equal_peak_temperature.argtypes = [vp, sz, C.c_double, C.c_double, pd, pi, pi, pd]
    L.rewl_join.argtypes = [i32, i32, i32, i32, vp, vp, vp, vp, sz]
    L.rewl_bootstrap.argtypes = [i32, i32, i32, i32, vp, i32, vp, vp, i32, vp, vp, sz]
    L.rewl_ising_energy.argtypes = [i32, i32, C.POINTER(C.c_longlong)]
    for name in ("rewl_canonical", "rewl_canonical_distribution", "rewl_specific_heat_peak",
                 "rewl_equal_peak_temperature", "rewl_join", "rewl_bootstrap", "rewl_ising_energy"):
        getattr(L, name).restype = st
    L.rewl_last_error.argtypes = []
    L.rewl_last_error.restype = C.c_char_p
    L.rewl_production_start.argtypes = [H, i32]
    L.rewl_production_run.argtypes = [H, C.c_longlong]
    L.rewl_production_histogram.argtypes = [H, vp, sz]
    for name in ("rewl_production_start", "rewl_production_run", "rewl_production_histogram"):
        getattr(L, name).restype = st
    L.rewl_measure_pipes.argtypes = [C.POINTER(PipeRates)]
    L.rewl_measure_pipes.restype = st
    L.rewl_version.argtypes = []
    L.rewl_version.restype = C.c_char_p
    _lib = L
    return L


def check(status):
    if status != REWL_OK:
        msg = load().rewl_last_error().decode("utf-8", "replace")
        raise RewlError(status, msg)
