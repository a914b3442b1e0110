"""CPU oracle for Delta-matrix simulated annealing on the QAP (test infrastructure).

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it. The product library (``paper_1208_2675_gb300``) never imports it, and the two
share no code: the oracle is plain C (``qap_oracle.c``) compiled with gcc, the
product is CUDA compiled with nvcc.

Functions follow G. Paul, arXiv:1208.2675: Eq. (1) (cost), Eq. (2) (acceptance),
section 2.2 steps (a)-(e) (the Delta-matrix loop) and section 2.1 (traditional SA).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qap_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile qap_oracle.c into liboracle.so (plain gcc, no FMA contraction)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fvisibility=hidden", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.orc_cost.restype = ctypes.c_int64
        L.orc_cost.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p]
        L.orc_swap_cost_change.restype = ctypes.c_int64
        L.orc_swap_cost_change.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p,
                                           ctypes.c_int32, ctypes.c_int32]
        L.orc_delta_entry.restype = ctypes.c_int64
        L.orc_delta_entry.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p,
                                      ctypes.c_int32, ctypes.c_int32]
        L.orc_delta_matrix.restype = None
        L.orc_delta_matrix.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p, _i64p]
        L.orc_philox4x32_10.restype = None
        L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.orc_rand_word.restype = ctypes.c_uint32
        L.orc_rand_word.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64]
        L.orc_uniform.restype = ctypes.c_double
        L.orc_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64]
        L.orc_chain_create.restype = ctypes.c_void_p
        L.orc_chain_create.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p,
                                       ctypes.c_double, ctypes.c_double,
                                       ctypes.c_uint64, ctypes.c_int32,
                                       ctypes.c_uint64, ctypes.c_uint32]
        L.orc_chain_destroy.restype = None
        L.orc_chain_destroy.argtypes = [ctypes.c_void_p]
        L.orc_chain_set_check.restype = None
        L.orc_chain_set_check.argtypes = [ctypes.c_void_p, ctypes.c_int32]
        L.orc_chain_check_failures.restype = ctypes.c_int64
        L.orc_chain_check_failures.argtypes = [ctypes.c_void_p]
        L.orc_chain_set_log.restype = None
        L.orc_chain_set_log.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
        L.orc_chain_get_log.restype = ctypes.c_uint64
        L.orc_chain_get_log.argtypes = [ctypes.c_void_p, _u64p, ctypes.c_uint64]
        L.orc_chain_set_near_log.restype = None
        L.orc_chain_set_near_log.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
        L.orc_chain_get_near_log.restype = ctypes.c_uint64
        L.orc_chain_get_near_log.argtypes = [ctypes.c_void_p, _u64p, ctypes.c_uint64]
        L.orc_chain_accepts.restype = ctypes.c_int32
        L.orc_chain_accepts.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64]
        L.orc_delta_entry_general.restype = ctypes.c_int64
        L.orc_delta_entry_general.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p,
                                              ctypes.c_int32, ctypes.c_int32]
        L.orc_chain_set_order.restype = None
        L.orc_chain_set_order.argtypes = [ctypes.c_void_p, ctypes.c_int32]
        L.orc_chain_is_general.restype = ctypes.c_int32
        L.orc_chain_is_general.argtypes = [ctypes.c_void_p]
        L.orc_chain_proposal.restype = None
        L.orc_chain_proposal.argtypes = [ctypes.c_void_p, ctypes.c_uint64, _i32p, _i32p]
        L.orc_chain_schedule.restype = None
        L.orc_chain_schedule.argtypes = [ctypes.c_void_p, _f64p, _f64p, _f64p]
        L.orc_chain_temperature.restype = ctypes.c_double
        L.orc_chain_temperature.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
        L.orc_chain_state.restype = None
        L.orc_chain_state.argtypes = [ctypes.c_void_p, _i32p, _i64p, _u64p, _u64p, _u64p]
        L.orc_chain_delta.restype = None
        L.orc_chain_delta.argtypes = [ctypes.c_void_p, _i64p]
        L.orc_chain_run.restype = ctypes.c_int32
        L.orc_chain_run.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32]
        _lib = L
    return _lib


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(t)


# --------------------------------------------------------------------------- #
# Eq. (1) and the swap cost change
# --------------------------------------------------------------------------- #
def cost(A, B, p) -> int:
    """Eq. (1): sum_ij A[i,j] * B[p[i], p[j]]."""
    A, B, p = _i32(A), _i32(B), _i32(p)
    return int(lib().orc_cost(len(p), _ptr(A, _i32p), _ptr(B, _i32p), _ptr(p, _i32p)))


def swap_cost_change(A, B, p, r: int, s: int) -> int:
    """C(p o (r s)) - C(p), Eq. (1) evaluated twice."""
    A, B, p = _i32(A), _i32(B), _i32(p)
    return int(lib().orc_swap_cost_change(len(p), _ptr(A, _i32p), _ptr(B, _i32p),
                                          _ptr(p, _i32p), r, s))


def delta_entry(A, B, p, r: int, s: int) -> int:
    """Closed form of the swap cost change for symmetric, zero-diagonal A, B."""
    A, B, p = _i32(A), _i32(B), _i32(p)
    return int(lib().orc_delta_entry(len(p), _ptr(A, _i32p), _ptr(B, _i32p),
                                     _ptr(p, _i32p), r, s))


def delta_entry_general(A, B, p, r: int, s: int) -> int:
    """The swap cost change for any A, B (asymmetric, nonzero diagonals)."""
    A, B, p = _i32(A), _i32(B), _i32(p)
    return int(lib().orc_delta_entry_general(len(p), _ptr(A, _i32p), _ptr(B, _i32p),
                                             _ptr(p, _i32p), r, s))


def delta_matrix(A, B, p) -> np.ndarray:
    """Step (a) of section 2.2: full symmetric Delta (int64, zero diagonal)."""
    A, B, p = _i32(A), _i32(B), _i32(p)
    N = len(p)
    D = np.zeros((N, N), dtype=np.int64)
    lib().orc_delta_matrix(N, _ptr(A, _i32p), _ptr(B, _i32p), _ptr(p, _i32p),
                           _ptr(D, _i64p))
    return D


# --------------------------------------------------------------------------- #
# Random numbers (Philox4x32-10) and r of Eq. (2)
# --------------------------------------------------------------------------- #
def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c, _u32p), _ptr(k, _u32p), _ptr(out, _u32p))
    return out


def rand_word(seed: int, stream: int, it: int) -> int:
    return int(lib().orc_rand_word(seed, stream, it))


def uniform(seed: int, stream: int, it: int) -> float:
    return float(lib().orc_uniform(seed, stream, it))


# --------------------------------------------------------------------------- #
# One SA chain
# --------------------------------------------------------------------------- #
class Chain:
    """A Delta-matrix SA chain (section 2.2) or a traditional one (section 2.1)."""

    def __init__(self, A, B, p0, *, t0: float, tf: float, total_iters: int,
                 relative: bool = True, seed: int = 0, stream: int = 0,
                 check: bool = False, log_cap: int = 0, random_order: bool = False):
        self.A, self.B = _i32(A), _i32(B)
        p0 = _i32(p0)
        self.N = len(p0)
        h = lib().orc_chain_create(self.N, _ptr(self.A, _i32p), _ptr(self.B, _i32p),
                                   _ptr(p0, _i32p), float(t0), float(tf),
                                   int(total_iters), int(bool(relative)),
                                   int(seed), int(stream))
        if not h:
            raise ValueError("oracle chain rejected its inputs")
        self._h = ctypes.c_void_p(h)
        if check:
            lib().orc_chain_set_check(self._h, 1)
        if log_cap:
            lib().orc_chain_set_log(self._h, int(log_cap))
        self._log_cap = int(log_cap)
        lib().orc_chain_set_near_log(self._h, 8)
        if random_order:
            lib().orc_chain_set_order(self._h, 1)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.orc_chain_destroy(h)
            self._h = None

    def run(self, iters: int, traditional: bool = False) -> None:
        lib().orc_chain_run(self._h, int(iters), int(bool(traditional)))

    def state(self) -> dict:
        p = np.zeros(self.N, dtype=np.int32)
        cost_ = ctypes.c_int64()
        acc = ctypes.c_uint64()
        it = ctypes.c_uint64()
        nt = ctypes.c_uint64()
        lib().orc_chain_state(self._h, _ptr(p, _i32p), ctypes.byref(cost_),
                              ctypes.byref(acc), ctypes.byref(it), ctypes.byref(nt))
        return {"p": p, "cost": cost_.value, "accepts": acc.value,
                "it": it.value, "near_ties": nt.value}

    def delta(self) -> np.ndarray:
        D = np.zeros((self.N, self.N), dtype=np.int64)
        lib().orc_chain_delta(self._h, _ptr(D, _i64p))
        return D

    def schedule(self) -> tuple[float, float, float]:
        T0, Tf, al = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        lib().orc_chain_schedule(self._h, ctypes.byref(T0), ctypes.byref(Tf),
                                 ctypes.byref(al))
        return T0.value, Tf.value, al.value

    def temperature(self, it: int) -> float:
        return float(lib().orc_chain_temperature(self._h, int(it)))

    def check_failures(self) -> int:
        return int(lib().orc_chain_check_failures(self._h))

    def is_general(self) -> bool:
        """True when the general (asymmetric) swap-cost forms are in use."""
        return bool(lib().orc_chain_is_general(self._h))

    def proposal(self, it: int) -> tuple[int, int]:
        """The pair (r, s), r < s, proposed at iteration it."""
        r, s = ctypes.c_int32(), ctypes.c_int32()
        lib().orc_chain_proposal(self._h, int(it), ctypes.byref(r), ctypes.byref(s))
        return r.value, s.value

    def accepts(self, delta: int, it: int) -> bool:
        """Eq. (2) (reading R3) for swap cost delta proposed at iteration it."""
        return bool(lib().orc_chain_accepts(self._h, int(delta), int(it)))

    def near_tie_log(self):
        """(iteration indices of the first near-ties (up to 8), total count)."""
        out = np.zeros(8, dtype=np.uint64)
        n = lib().orc_chain_get_near_log(self._h, _ptr(out, _u64p), 8)
        return out[:min(n, 8)], int(n)

    def accept_log(self) -> np.ndarray:
        cap = max(self._log_cap, 1)
        out = np.zeros(cap, dtype=np.uint64)
        n = lib().orc_chain_get_log(self._h, _ptr(out, _u64p), cap)
        return out[:min(n, cap)]
