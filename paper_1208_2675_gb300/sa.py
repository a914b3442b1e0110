"""ctypes binding of libqapsa (include/qap_sa.h): argument marshalling only.

Every function here forwards to the C entry point of the same name; all of the
annealing runs in the CUDA kernels of the library. If ``libqapsa.so`` has not
been built, or no CUDA device is usable, calls raise -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqapsa.so")

QAP_OK = 0
QAP_E_INVAL = -1
QAP_E_RANGE = -2
QAP_E_NOMEM = -3
QAP_E_CUDA = -4
QAP_E_TIMEOUT = -5
QAP_E_STATE = -6
QAP_E_UNSUPPORTED = -7
QAP_T_RELATIVE = 1
QAP_ORDER_RANDOM = 2

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)


class qap_schedule(ctypes.Structure):
    _fields_ = [("t0", ctypes.c_double), ("tf", ctypes.c_double),
                ("total_iters", ctypes.c_uint64), ("flags", ctypes.c_uint32),
                ("stream_id", ctypes.c_uint32)]


class qap_sa_info(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("tier", ctypes.c_int32),
                ("iterations", ctypes.c_uint64), ("accepts", ctypes.c_uint64),
                ("cost", ctypes.c_int64), ("near_ties", ctypes.c_uint64),
                ("exact_evals", ctypes.c_uint64), ("windows", ctypes.c_uint64),
                ("T0", ctypes.c_double), ("Tf", ctypes.c_double),
                ("alpha", ctypes.c_double), ("total_iters", ctypes.c_uint64),
                ("smem_bytes", ctypes.c_uint64), ("direct_iters", ctypes.c_uint64),
                ("direct_accepts", ctypes.c_uint64), ("warp_iters", ctypes.c_uint64),
                ("ctas", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("hot_iters", ctypes.c_uint64), ("hot_accepts", ctypes.c_uint64)]


class qap_peaks(ctypes.Structure):
    _fields_ = [("sm_count", ctypes.c_int32), ("smem_optin_bytes", ctypes.c_int32),
                ("l2_bytes", ctypes.c_int64), ("sm_mhz", ctypes.c_double),
                ("smem_bytes_per_clk_sm", ctypes.c_double), ("smem_gbs_chip", ctypes.c_double),
                ("l2_gbs", ctypes.c_double), ("int32_ops_per_clk_sm", ctypes.c_double),
                ("dp4a_per_clk_sm", ctypes.c_double), ("cta_barrier_ns", ctypes.c_double),
                ("cluster_barrier_ns", ctypes.c_double * 5), ("grid_barrier_ns", ctypes.c_double),
                ("l2_latency_ns", ctypes.c_double), ("dsmem_latency_ns", ctypes.c_double),
                ("smem_latency_ns", ctypes.c_double), ("l2_gbs_sm", ctypes.c_double)]


class qap_knobs(ctypes.Structure):
    _fields_ = [("tier", ctypes.c_int32), ("t3_grid", ctypes.c_int32),
                ("hybrid_rate", ctypes.c_float), ("warp_rate", ctypes.c_float),
                ("cluster_hybrid_rate", ctypes.c_float), ("reserved", ctypes.c_uint32)]


class qap_problem(ctypes.Structure):
    _fields_ = [("A", _i32p), ("B", _i32p), ("p0", _i32p), ("N", ctypes.c_int32),
                ("reserved", ctypes.c_uint32), ("sched", qap_schedule),
                ("seed", ctypes.c_uint64)]


class qap_server_cfg(ctypes.Structure):
    _fields_ = [("max_sms", ctypes.c_int32), ("reserved", ctypes.c_uint32),
                ("mem_budget_bytes", ctypes.c_uint64)]


class qap_result(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int32), ("status", ctypes.c_int32),
                ("cost", ctypes.c_int64), ("accepts", ctypes.c_uint64),
                ("iterations", ctypes.c_uint64), ("queue_s", ctypes.c_double),
                ("latency_s", ctypes.c_double)]


# Every symbol include/qap_sa.h declares, with its ctypes signature.
SIGNATURES = {
    "qap_sa_create": (ctypes.c_int, [_i32p, _i32p, ctypes.c_int32, _i32p,
                                     ctypes.POINTER(qap_schedule), ctypes.c_uint64,
                                     ctypes.POINTER(ctypes.c_void_p)]),
    "qap_sa_create_device": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_int32, ctypes.c_void_p,
                                            ctypes.POINTER(qap_schedule),
                                            ctypes.c_uint64, ctypes.c_void_p,
                                            ctypes.POINTER(ctypes.c_void_p)]),
    "qap_sa_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "qap_sa_run_async": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "qap_sa_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "qap_sa_result": (ctypes.c_int, [ctypes.c_void_p, _i32p, _i64p, _u64p]),
    "qap_sa_result_device": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p]),
    "qap_sa_get_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(qap_sa_info)]),
    "qap_sa_delta": (ctypes.c_int, [ctypes.c_void_p, _i32p]),
    "qap_sa_temperature": (ctypes.c_double, [ctypes.c_void_p, ctypes.c_uint64]),
    "qap_sa_destroy": (None, [ctypes.c_void_p]),
    "qap_sa_set_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "qap_sa_inject_barrier_fault": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "qap_sa_kernel_times": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                           _u64p]),
    "qap_sa_near_tie_log": (ctypes.c_int, [ctypes.c_void_p, _u64p, ctypes.c_int32, _u64p]),
    "qap_sa_accept_probe": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, _u64p, _u64p,
                                           _i32p, _i32p]),
    "qap_batch_create": (ctypes.c_int, [ctypes.POINTER(qap_problem), ctypes.c_int32,
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "qap_batch_run": (ctypes.c_int, [ctypes.c_void_p, _u64p]),
    "qap_batch_result": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, _i32p, _i64p, _u64p]),
    "qap_batch_get_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32,
                                          ctypes.POINTER(qap_sa_info)]),
    "qap_batch_destroy": (None, [ctypes.c_void_p]),
    "qap_server_start": (ctypes.c_int, [ctypes.POINTER(qap_server_cfg),
                                        ctypes.POINTER(ctypes.c_void_p)]),
    "qap_server_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(qap_problem),
                                         ctypes.c_uint64, _u64p]),
    "qap_server_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64,
                                       ctypes.POINTER(qap_result), _i32p]),
    "qap_server_max_running": (ctypes.c_int, [ctypes.c_void_p]),
    "qap_server_stop": (ctypes.c_int, [ctypes.c_void_p]),
    "qap_sa_setup_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p]),
    "qap_peaks_measure": (ctypes.c_int, [ctypes.POINTER(qap_peaks)]),
    "qap_knobs_set": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(qap_knobs)]),
    "qap_tune": (ctypes.c_int, [ctypes.c_int32, ctypes.c_uint64, ctypes.POINTER(qap_knobs),
                                ctypes.POINTER(ctypes.c_double)]),
    "qap_sa_max_n": (ctypes.c_int32, []),
    "qap_sa_max_n_tier": (ctypes.c_int32, [ctypes.c_int32]),
    "qap_sa_strerror": (ctypes.c_char_p, [ctypes.c_int]),
}

_lib = None


def lib() -> ctypes.CDLL:
    """Loads libqapsa.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class QapError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().qap_sa_strerror(status).decode()
        super().__init__(f"{where}: status {status} ({msg})")


def _check(status: int, where: str) -> None:
    if status != QAP_OK:
        raise QapError(status, where)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def make_schedule(t0: float, tf: float, total_iters: int, relative: bool = True,
                  stream_id: int = 0, random_order: bool = False) -> qap_schedule:
    flags = (QAP_T_RELATIVE if relative else 0) | (QAP_ORDER_RANDOM if random_order else 0)
    return qap_schedule(float(t0), float(tf), int(total_iters), flags, int(stream_id))


# ---- C entry points, same names ------------------------------------------- #
def qap_sa_create(A, B, p0, sched: qap_schedule, seed: int) -> ctypes.c_void_p:
    A, B, p0 = _i32(A), _i32(B), _i32(p0)
    h = ctypes.c_void_p()
    _check(lib().qap_sa_create(A.ctypes.data_as(_i32p), B.ctypes.data_as(_i32p),
                               len(p0), p0.ctypes.data_as(_i32p), ctypes.byref(sched),
                               int(seed), ctypes.byref(h)), "qap_sa_create")
    return h


def qap_sa_create_device(A_ptr: int, B_ptr: int, N: int, p0_ptr: int,
                         sched: qap_schedule, seed: int, stream: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().qap_sa_create_device(ctypes.c_void_p(A_ptr), ctypes.c_void_p(B_ptr),
                                      int(N), ctypes.c_void_p(p0_ptr), ctypes.byref(sched),
                                      int(seed), ctypes.c_void_p(stream or None),
                                      ctypes.byref(h)), "qap_sa_create_device")
    return h


def qap_sa_run(h, iters: int) -> None:
    _check(lib().qap_sa_run(h, int(iters)), "qap_sa_run")


def qap_sa_run_async(h, iters: int) -> None:
    _check(lib().qap_sa_run_async(h, int(iters)), "qap_sa_run_async")


def qap_sa_sync(h) -> None:
    _check(lib().qap_sa_sync(h), "qap_sa_sync")


def qap_sa_result(h, N: int):
    p = np.zeros(N, dtype=np.int32)
    cost = ctypes.c_int64()
    acc = ctypes.c_uint64()
    _check(lib().qap_sa_result(h, p.ctypes.data_as(_i32p), ctypes.byref(cost),
                               ctypes.byref(acc)), "qap_sa_result")
    return p, cost.value, acc.value


def qap_sa_result_device(h, p_ptr: int, cost_ptr: int, acc_ptr: int) -> None:
    _check(lib().qap_sa_result_device(h, ctypes.c_void_p(p_ptr or None),
                                      ctypes.c_void_p(cost_ptr or None),
                                      ctypes.c_void_p(acc_ptr or None)),
           "qap_sa_result_device")


def qap_sa_get_info(h) -> dict:
    info = qap_sa_info()
    _check(lib().qap_sa_get_info(h, ctypes.byref(info)), "qap_sa_get_info")
    return {name: getattr(info, name) for name, _ in qap_sa_info._fields_}


KERNEL_KINDS = ("hot", "sa", "aux")  # QAP_KT_HOT, QAP_KT_SA, QAP_KT_AUX


def qap_sa_inject_barrier_fault(h, on: bool) -> None:
    _check(lib().qap_sa_inject_barrier_fault(h, 1 if on else 0), "qap_sa_inject_barrier_fault")


def qap_sa_set_timing(h, on: bool) -> None:
    _check(lib().qap_sa_set_timing(h, 1 if on else 0), "qap_sa_set_timing")


def qap_sa_kernel_times(h) -> dict:
    """{kind: (device seconds, launches)} since timing was switched on or last read."""
    sec = (ctypes.c_double * len(KERNEL_KINDS))()
    n = np.zeros(len(KERNEL_KINDS), dtype=np.uint64)
    _check(lib().qap_sa_kernel_times(h, sec, n.ctypes.data_as(_u64p)), "qap_sa_kernel_times")
    return {k: (float(sec[i]), int(n[i])) for i, k in enumerate(KERNEL_KINDS)}


def qap_sa_delta(h, M: int) -> np.ndarray:
    out = np.zeros(max(M, 1), dtype=np.int32)
    _check(lib().qap_sa_delta(h, out.ctypes.data_as(_i32p)), "qap_sa_delta")
    return out[:M]


def qap_sa_temperature(h, it: int) -> float:
    return float(lib().qap_sa_temperature(h, int(it)))


def qap_sa_near_tie_log(h, cap: int = 8):
    """(iteration indices of the first near-ties, total near-tie count)."""
    out = np.zeros(max(cap, 1), dtype=np.uint64)
    n = ctypes.c_uint64()
    _check(lib().qap_sa_near_tie_log(h, out.ctypes.data_as(_u64p), int(cap), ctypes.byref(n)),
           "qap_sa_near_tie_log")
    return out[:min(cap, 8, n.value)], n.value


def qap_sa_accept_probe(h, it, it0, delta) -> np.ndarray:
    """Eq. (2) decided as the kernels decide it, for probes (it, it0, delta)."""
    it = np.ascontiguousarray(it, dtype=np.uint64)
    it0 = np.ascontiguousarray(it0, dtype=np.uint64)
    dl = np.ascontiguousarray(delta, dtype=np.int32)
    out = np.zeros(len(it), dtype=np.int32)
    _check(lib().qap_sa_accept_probe(h, len(it), it.ctypes.data_as(_u64p),
                                     it0.ctypes.data_as(_u64p), dl.ctypes.data_as(_i32p),
                                     out.ctypes.data_as(_i32p)), "qap_sa_accept_probe")
    return out


def qap_sa_destroy(h) -> None:
    if h:
        lib().qap_sa_destroy(h)


def qap_sa_setup_noalloc(A_ptr: int, B_ptr: int, N: int, p_ptr: int, delta_ptr: int,
                         cost_ptr: int, stream: int = 0) -> None:
    """Step (a) into caller-owned DEVICE buffers, allocating nothing (see the header)."""
    _check(lib().qap_sa_setup_noalloc(ctypes.c_void_p(A_ptr), ctypes.c_void_p(B_ptr), int(N),
                                      ctypes.c_void_p(p_ptr), ctypes.c_void_p(delta_ptr),
                                      ctypes.c_void_p(cost_ptr), ctypes.c_void_p(stream or None)),
           "qap_sa_setup_noalloc")


def qap_peaks_measure() -> dict:
    """Microbenchmarks of the current device (include/qap_peaks.h)."""
    pk = qap_peaks()
    _check(lib().qap_peaks_measure(ctypes.byref(pk)), "qap_peaks_measure")
    out = {name: getattr(pk, name) for name, _ in qap_peaks._fields_}
    out["cluster_barrier_ns"] = dict(zip((2, 4, 8, 13, 16), list(pk.cluster_barrier_ns)))
    return out


KNOB_FIELDS = [name for name, _ in qap_knobs._fields_ if name != "reserved"]


def knobs_struct(d: dict | None) -> qap_knobs:
    """A qap_knobs from a dict (missing fields: the defaults)."""
    d = d or {}
    return qap_knobs(int(d.get("tier", 0)), int(d.get("t3_grid", 0)),
                     float(d.get("hybrid_rate", -1.0)), float(d.get("warp_rate", -1.0)),
                     float(d.get("cluster_hybrid_rate", -1.0)), 0)


def qap_knobs_set(n_lo: int, n_hi: int, knobs: dict | None) -> None:
    """Registers knobs for N in [n_lo, n_hi]; knobs=None clears every range."""
    if knobs is None:
        _check(lib().qap_knobs_set(0, 0, None), "qap_knobs_set")
    else:
        k = knobs_struct(knobs)
        _check(lib().qap_knobs_set(int(n_lo), int(n_hi), ctypes.byref(k)), "qap_knobs_set")


def qap_tune(N: int, iters: int):
    """(best knobs as a dict, seconds of the best trial run)."""
    k = qap_knobs()
    t = ctypes.c_double()
    _check(lib().qap_tune(int(N), int(iters), ctypes.byref(k), ctypes.byref(t)), "qap_tune")
    return {name: getattr(k, name) for name in KNOB_FIELDS}, t.value


def qap_sa_max_n() -> int:
    return int(lib().qap_sa_max_n())


def qap_sa_max_n_tier(tier: int) -> int:
    return int(lib().qap_sa_max_n_tier(int(tier)))


def qap_sa_strerror(status: int) -> str:
    return lib().qap_sa_strerror(int(status)).decode()


def qap_batch_create(problems) -> ctypes.c_void_p:
    """problems: list of dicts with A, B, p0, t0, tf, total_iters, relative,
    stream_id, seed.  Host arrays are kept alive for the duration of the call."""
    keep = []
    arr = (qap_problem * len(problems))()
    for i, pr in enumerate(problems):
        A, B, p0 = _i32(pr["A"]), _i32(pr["B"]), _i32(pr["p0"])
        keep += [A, B, p0]
        arr[i].A = A.ctypes.data_as(_i32p)
        arr[i].B = B.ctypes.data_as(_i32p)
        arr[i].p0 = p0.ctypes.data_as(_i32p)
        arr[i].N = len(p0)
        arr[i].reserved = 0
        arr[i].sched = make_schedule(pr["t0"], pr["tf"], pr["total_iters"],
                                     pr.get("relative", True), pr.get("stream_id", 0))
        arr[i].seed = int(pr.get("seed", 0))
    h = ctypes.c_void_p()
    _check(lib().qap_batch_create(arr, len(problems), ctypes.byref(h)), "qap_batch_create")
    return h


def qap_batch_run(h, iters=None) -> None:
    if iters is None:
        _check(lib().qap_batch_run(h, None), "qap_batch_run")
    else:
        it = np.ascontiguousarray(iters, dtype=np.uint64)
        _check(lib().qap_batch_run(h, it.ctypes.data_as(_u64p)), "qap_batch_run")


def qap_batch_result(h, i: int, N: int):
    p = np.zeros(N, dtype=np.int32)
    cost = ctypes.c_int64()
    acc = ctypes.c_uint64()
    _check(lib().qap_batch_result(h, int(i), p.ctypes.data_as(_i32p), ctypes.byref(cost),
                                  ctypes.byref(acc)), "qap_batch_result")
    return p, cost.value, acc.value


def qap_batch_get_info(h, i: int) -> dict:
    info = qap_sa_info()
    _check(lib().qap_batch_get_info(h, int(i), ctypes.byref(info)), "qap_batch_get_info")
    return {name: getattr(info, name) for name, _ in qap_sa_info._fields_}


def qap_batch_destroy(h) -> None:
    if h:
        lib().qap_batch_destroy(h)


def _problem_struct(pr, keep):
    A, B, p0 = _i32(pr["A"]), _i32(pr["B"]), _i32(pr["p0"])
    keep += [A, B, p0]
    q = qap_problem()
    q.A = A.ctypes.data_as(_i32p)
    q.B = B.ctypes.data_as(_i32p)
    q.p0 = p0.ctypes.data_as(_i32p)
    q.N = len(p0)
    q.reserved = 0
    q.sched = make_schedule(pr["t0"], pr["tf"], pr["total_iters"], pr.get("relative", True),
                            pr.get("stream_id", 0))
    q.seed = int(pr.get("seed", 0))
    return q


def qap_server_start(max_sms: int = 0, mem_budget_bytes: int = 0) -> ctypes.c_void_p:
    cfg = qap_server_cfg(int(max_sms), 0, int(mem_budget_bytes))
    h = ctypes.c_void_p()
    _check(lib().qap_server_start(ctypes.byref(cfg), ctypes.byref(h)), "qap_server_start")
    return h


def qap_server_submit(h, problem: dict, iters: int) -> int:
    keep = []
    q = _problem_struct(problem, keep)
    t = ctypes.c_uint64()
    _check(lib().qap_server_submit(h, ctypes.byref(q), int(iters), ctypes.byref(t)),
           "qap_server_submit")
    return t.value


def qap_server_poll(h, ticket: int, N: int):
    """Returns None while pending, else a dict with the result and p."""
    res = qap_result()
    p = np.zeros(N, dtype=np.int32)
    _check(lib().qap_server_poll(h, int(ticket), ctypes.byref(res), p.ctypes.data_as(_i32p)),
           "qap_server_poll")
    if not res.done:
        return None
    out = {name: getattr(res, name) for name, _ in qap_result._fields_}
    out["p"] = p
    return out


def qap_server_max_running(h) -> int:
    return int(lib().qap_server_max_running(h))


def qap_server_stop(h) -> None:
    if h:
        _check(lib().qap_server_stop(h), "qap_server_stop")


# ---- convenience wrapper ----------------------------------------------------- #
class Chain:
    """One SA chain on the GPU (a qap_sa handle)."""

    def __init__(self, A, B, p0, *, t0: float, tf: float, total_iters: int,
                 relative: bool = True, seed: int = 0, stream_id: int = 0,
                 random_order: bool = False):
        self.N = len(p0)
        self.M = self.N * (self.N - 1) // 2
        self.sched = make_schedule(t0, tf, total_iters, relative, stream_id, random_order)
        self.h = qap_sa_create(A, B, p0, self.sched, seed)

    @classmethod
    def from_device(cls, A_t, B_t, p0_t, *, t0: float, tf: float, total_iters: int,
                    relative: bool = True, seed: int = 0, stream_id: int = 0,
                    stream: int = 0) -> "Chain":
        """A_t, B_t, p0_t: contiguous int32 CUDA tensors (any object with
        data_ptr()); `stream` is a raw cudaStream_t (0 = library-owned)."""
        self = cls.__new__(cls)
        self.N = int(p0_t.shape[0])
        self.M = self.N * (self.N - 1) // 2
        self.sched = make_schedule(t0, tf, total_iters, relative, stream_id)
        self.h = qap_sa_create_device(A_t.data_ptr(), B_t.data_ptr(), self.N,
                                      p0_t.data_ptr(), self.sched, seed, stream)
        return self

    def run(self, iters: int) -> None:
        qap_sa_run(self.h, iters)

    def run_async(self, iters: int) -> None:
        qap_sa_run_async(self.h, iters)

    def sync(self) -> None:
        qap_sa_sync(self.h)

    def result(self):
        return qap_sa_result(self.h, self.N)

    def set_timing(self, on: bool = True) -> None:
        qap_sa_set_timing(self.h, on)

    def kernel_times(self) -> dict:
        return qap_sa_kernel_times(self.h)

    def info(self) -> dict:
        return qap_sa_get_info(self.h)

    def delta(self) -> np.ndarray:
        return qap_sa_delta(self.h, self.M)

    def temperature(self, it: int) -> float:
        return qap_sa_temperature(self.h, it)

    def near_tie_log(self):
        return qap_sa_near_tie_log(self.h)

    def close(self) -> None:
        if getattr(self, "h", None):
            qap_sa_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
