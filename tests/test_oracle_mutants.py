"""Planted mistakes in the oracle are caught by its pins.

Each mutant is a copy of oracle/qap_oracle.c with one plausible mistake (a
dropped term, a wrong sign or index, a transposed operand, a wrong constant, a
wrong schedule parameter),
compiled on the CPU into a temporary library.  The checks below use only
formulations independent of the oracle (Eq. (1) over locations, brute-force
swap costs, Eq. (2) in exponential form, published Philox vectors, the
schedule's parameters from their definitions); every
mutant must fail at least one of them, and the unmutated source must pass all.

Not listed: accepting only delta < 0 outright instead of delta <= 0 -- an
equivalent change, since for delta = 0 the binary64 test accepts as well
(log u < 0 for every u of the reading).
"""
import ctypes
import math
import os
import subprocess
import tempfile

import numpy as np
import pytest

from paper_1208_2675_gb300 import instances

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "qap_oracle.c")

MUTANTS = {
    "delta_entry_factor": ("  return 2 * acc;\n}", "  return acc;\n}"),
    "delta_entry_sign": ("int64_t b = (int64_t)B[(int64_t)p[k] * N + p[s]] -\n                B[(int64_t)p[k] * N + p[r]];",
                         "int64_t b = (int64_t)B[(int64_t)p[k] * N + p[r]] -\n                B[(int64_t)p[k] * N + p[s]];"),
    "delta_entry_transposed": ("int64_t a = (int64_t)A[(int64_t)k * N + r] - A[(int64_t)k * N + s];",
                               "int64_t a = (int64_t)A[(int64_t)k * N + r] - A[(int64_t)s * N + r + 0 * k];"),
    "update_dropped_term": ("                  A[(int64_t)s * N + u] + A[(int64_t)s * N + v];",
                            "                  A[(int64_t)s * N + u];"),
    "update_new_p": ("  const int32_t pr = p[r], ps = p[s];", "  const int32_t pr = p[s], ps = p[r];"),
    "update_factor": ("      D[(int64_t)u * N + v] += 2 * a * b;", "      D[(int64_t)u * N + v] += a * b;"),
    "cost_index": ("(int64_t)B[(int64_t)p[i] * N + p[j]];", "(int64_t)B[(int64_t)p[i] * N + j];"),
    "accept_sign": ("  return (double)delta < -prod;", "  return (double)delta < prod;"),
    "uniform_offset": ("return ((double)orc_rand_word(seed, stream, it) + 0.5) * 0x1p-32;",
                       "return ((double)orc_rand_word(seed, stream, it) + 1.0) * 0x1p-32;"),
    "philox_constant": ("const uint32_t W0 = 0x9E3779B9u", "const uint32_t W0 = 0x9E3779B7u"),
    "philox_word": ("  return out[it % 4u];", "  return out[(it + 1) % 4u];"),
    "schedule_order": ("  for (int b = 7; b >= 0; --b) T = T * S->P[b][(it >> (8 * b)) & 0xFFu];",
                       "  for (int b = 7; b >= 0; --b) T = T * S->P[7 - b][(it >> (8 * b)) & 0xFFu];"),
    "cursor_order": ("  c->cur_s++;\n  if (c->cur_s == c->N) {", "  c->cur_s += 2;\n  if (c->cur_s >= c->N) {"),
    "t0_mean_divisor": ("(double)sum / (double)c->M", "(double)sum / (double)c->N"),
    "tf_not_relative": ("    Tf = tf * T0;\n  }", "    Tf = tf;\n  }"),
    "alpha_exponent": ("pow(Tf / T0, 1.0 / (double)(I - 1))", "pow(Tf / T0, 1.0 / (double)(I))"),
    "philox_multiplier": ("const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;",
                          "const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D55u;"),
    "philox_key_word": ("uint32_t n0 = hi1 ^ c1 ^ k0;", "uint32_t n0 = hi1 ^ c1 ^ k1;"),
    # the general (asymmetric) swap cost and its update
    "general_entry_diag_sign": ("(ORC_A(r, r) - ORC_A(s, s)) * (ORC_BP(s, s) - ORC_BP(r, r))",
                                "(ORC_A(r, r) - ORC_A(s, s)) * (ORC_BP(r, r) - ORC_BP(s, s))"),
    "general_entry_pair_transposed": ("(ORC_A(r, s) - ORC_A(s, r)) * (ORC_BP(s, r) - ORC_BP(r, s))",
                                      "(ORC_A(r, s) - ORC_A(s, r)) * (ORC_BP(r, s) - ORC_BP(s, r))"),
    "general_entry_dropped_column_sum": (
        "    d += (ORC_A(r, k) - ORC_A(s, k)) * (ORC_BP(s, k) - ORC_BP(r, k)) +\n"
        "         (ORC_A(k, r) - ORC_A(k, s)) * (ORC_BP(k, s) - ORC_BP(k, r));",
        "    d += 2 * (ORC_A(r, k) - ORC_A(s, k)) * (ORC_BP(s, k) - ORC_BP(r, k));"),
    "general_update_symmetric_shortcut": ("      D[(int64_t)u * N + v] += a1 * b1 + a2 * b2;",
                                          "      D[(int64_t)u * N + v] += 2 * a1 * b1;"),
    "general_update_transposed": (
        "      int64_t a2 = ORC_A(u, r) - ORC_A(v, r) - ORC_A(u, s) + ORC_A(v, s);",
        "      int64_t a2 = ORC_A(r, u) - ORC_A(r, v) - ORC_A(s, u) + ORC_A(s, v);"),
    "general_recompute_symmetric_form": (
        "      int64_t d = orc_delta_entry_general(N, A, B, p, r, v);",
        "      int64_t d = orc_delta_entry(N, A, B, p, r, v);"),
    "family_check_ignores_diagonal": (
        "    if (A[(int64_t)i * N + i] != 0 || B[(int64_t)i * N + i] != 0) return 0;", ""),
    # random proposal order
    "random_pair_word": ("int64_t m = (int64_t)(((uint64_t)out[0] * (uint64_t)c->M) >> 32);",
                         "int64_t m = (int64_t)(((uint64_t)out[1] * (uint64_t)c->M) >> 32);"),
    "random_pair_counter_word": (
        "  uint32_t ctr[4] = {(uint32_t)it, (uint32_t)(it >> 32), c->stream, 1u};",
        "  uint32_t ctr[4] = {(uint32_t)it, (uint32_t)(it >> 32), c->stream, 0u};"),
    "random_pair_scale": ("int64_t m = (int64_t)(((uint64_t)out[0] * (uint64_t)c->M) >> 32);",
                          "int64_t m = (int64_t)(((uint64_t)out[0] * (uint64_t)(c->M - 1)) >> 32);"),
}

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def _build(src_text: str, tmpdir: str, name: str) -> ctypes.CDLL:
    c_path = os.path.join(tmpdir, name + ".c")
    so_path = os.path.join(tmpdir, name + ".so")
    with open(c_path, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                    "-o", so_path, c_path, "-lm"], check=True)
    L = ctypes.CDLL(so_path)
    L.orc_cost.restype = ctypes.c_int64
    L.orc_cost.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p]
    L.orc_delta_matrix.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p, _i64p]
    L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
    L.orc_uniform.restype = ctypes.c_double
    L.orc_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64]
    L.orc_chain_create.restype = ctypes.c_void_p
    L.orc_chain_create.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_uint64, ctypes.c_int32,
                                   ctypes.c_uint64, ctypes.c_uint32]
    L.orc_chain_run.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32]
    L.orc_chain_state.argtypes = [ctypes.c_void_p, _i32p, _i64p, _u64p, _u64p, _u64p]
    L.orc_chain_delta.argtypes = [ctypes.c_void_p, _i64p]
    L.orc_chain_temperature.restype = ctypes.c_double
    L.orc_chain_temperature.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
    L.orc_chain_set_log.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
    L.orc_chain_get_log.restype = ctypes.c_uint64
    L.orc_chain_get_log.argtypes = [ctypes.c_void_p, _u64p, ctypes.c_uint64]
    L.orc_chain_schedule.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.orc_chain_set_order.argtypes = [ctypes.c_void_p, ctypes.c_int32]
    return L


def _loc_cost(A, B, p):
    q = np.argsort(p)
    return int((A[np.ix_(q, q)].astype(np.int64) * B.astype(np.int64)).sum())


def _swapped(p, r, s):
    q = np.array(p, copy=True)
    q[r], q[s] = q[s], q[r]
    return q


def _pins_hold(L) -> bool:
    """True if every independent check passes for this build of the oracle."""
    ptr = lambda a, t: a.ctypes.data_as(t)
    # (1) Eq. (1) against the location form
    A, B, p = instances.taixxa_like(9, 3)
    if L.orc_cost(9, ptr(A, _i32p), ptr(B, _i32p), ptr(p, _i32p)) != _loc_cost(A, B, p):
        return False
    # (2) step (a) against brute-force swap costs
    D = np.zeros((9, 9), dtype=np.int64)
    L.orc_delta_matrix(9, ptr(A, _i32p), ptr(B, _i32p), ptr(p, _i32p), ptr(D, _i64p))
    c0 = _loc_cost(A, B, p)
    for r in range(9):
        for s in range(r + 1, 9):
            if D[r, s] != _loc_cost(A, B, _swapped(p, r, s)) - c0:
                return False
    # (3) Philox known answer
    out = np.zeros(4, dtype=np.uint32)
    L.orc_philox4x32_10(ptr(np.zeros(4, dtype=np.uint32), _u32p),
                        ptr(np.zeros(2, dtype=np.uint32), _u32p), ptr(out, _u32p))
    if [int(x) for x in out] != [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]:
        return False
    # (4) r of Eq. (2) against its reading: (x + 0.5) / 2^32 of the published
    #     counter layout (the unmutated Philox, itself pinned by the vectors)
    import oracle as ref
    for it in [0, 1, 2, 3, 4, 999, 123457]:
        if L.orc_uniform(77, 5, it) != (ref.rand_word(77, 5, it) + 0.5) / 2 ** 32:
            return False
    # (5) a chain: replay every decision against Eq. (2) in exponential form with
    #     brute-force deltas, u from the published counter layout, T against
    #     T0 alpha^it; the final Delta against brute force.  Then the same for
    #     general instances (asymmetric; symmetric with a nonzero diagonal) and
    #     for random proposal order, with the pair drawn by its definition.
    A, B, p0 = instances.taixxa_like(8, 5)
    if not _chain_replay_holds(L, A, B, p0, 3000, 11, check_schedule=True):
        return False
    rng = np.random.default_rng(9)
    Ag = rng.integers(-20, 40, size=(7, 7)).astype(np.int32)
    Bg = rng.integers(-20, 40, size=(7, 7)).astype(np.int32)
    if not _chain_replay_holds(L, Ag, Bg, rng.permutation(7).astype(np.int32), 2000, 12):
        return False
    As, Bs, ps = instances.taixxa_like(7, 6)
    As, Bs = As.copy(), Bs.copy()
    np.fill_diagonal(As, rng.integers(1, 30, size=7))
    np.fill_diagonal(Bs, rng.integers(1, 30, size=7))
    if not _chain_replay_holds(L, As, Bs, ps, 2000, 13):
        return False
    A, B, p0 = instances.taixxa_like(8, 7)
    if not _chain_replay_holds(L, A, B, p0, 2000, 14, random_order=True):
        return False
    return True


def _random_pair(seed, stream, it, M, pairs):
    """The reading of random order: pair number (x M) >> 32, x word 0 of Philox
    at counter (it, stream, 1) -- through the published (pinned) Philox."""
    import oracle as ref
    x = int(ref.philox4x32_10([it & 0xFFFFFFFF, it >> 32, stream, 1],
                              [seed & 0xFFFFFFFF, seed >> 32])[0])
    return pairs[(x * M) >> 32]


def _chain_replay_holds(L, A, B, p0, I, seed, check_schedule=False, random_order=False):
    import oracle as ref
    ptr = lambda a, t: a.ctypes.data_as(t)
    N = len(p0)
    A, B, p0 = (np.ascontiguousarray(x, dtype=np.int32) for x in (A, B, p0))
    h = L.orc_chain_create(N, ptr(A, _i32p), ptr(B, _i32p), ptr(p0, _i32p), 0.5, 1e-2, I, 1,
                           seed, 0)
    if random_order:
        L.orc_chain_set_order(h, 1)
    L.orc_chain_set_log(h, I)
    L.orc_chain_run(h, I, 0)
    log = np.zeros(I, dtype=np.uint64)
    n = L.orc_chain_get_log(h, ptr(log, _u64p), I)
    accepted = set(int(x) for x in log[:n])
    T0, Tf, al = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    L.orc_chain_schedule(h, ctypes.byref(T0), ctypes.byref(Tf), ctypes.byref(al))
    pairs = [(r, s) for r in range(N) for s in range(r + 1, N)]
    c0 = _loc_cost(A, B, p0)
    if check_schedule:
        # the schedule's parameters from their definitions: T0 = 0.5 mean |Delta_0|
        # over the M pairs (brute-force swap costs), Tf = 1e-2 T0,
        # alpha = (Tf/T0)^(1/(I-1))
        sum_abs = sum(abs(_loc_cost(A, B, _swapped(p0, r, s)) - c0) for r, s in pairs)
        if T0.value != 0.5 * (sum_abs / len(pairs)) or Tf.value != 1e-2 * T0.value:
            return False
        if abs(al.value / (Tf.value / T0.value) ** (1.0 / (I - 1)) - 1.0) > 1e-12:
            return False
    q = np.array(p0, copy=True)
    for it in range(I):
        r, s = (_random_pair(seed, 0, it, len(pairs), pairs) if random_order
                else pairs[it % len(pairs)])
        delta = _loc_cost(A, B, _swapped(q, r, s)) - _loc_cost(A, B, q)
        T = L.orc_chain_temperature(h, it)
        if abs(T / (T0.value * al.value ** it) - 1) > 1e-9:
            return False
        u = (ref.rand_word(seed, 0, it) + 0.5) / 2 ** 32
        want = delta <= 0 or math.exp(-delta / T) > u
        if (it in accepted) != want:
            return False
        if want:
            q = _swapped(q, r, s)
    pf = np.zeros(N, dtype=np.int32)
    cost, acc, itv, nt = ctypes.c_int64(), ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    L.orc_chain_state(h, ptr(pf, _i32p), ctypes.byref(cost), ctypes.byref(acc),
                      ctypes.byref(itv), ctypes.byref(nt))
    if not np.array_equal(pf, q) or cost.value != _loc_cost(A, B, q):
        return False
    Dc = np.zeros((N, N), dtype=np.int64)
    L.orc_chain_delta(h, ptr(Dc, _i64p))
    c1 = _loc_cost(A, B, q)
    for r, s in pairs:
        if Dc[r, s] != _loc_cost(A, B, _swapped(q, r, s)) - c1:
            return False
    return True


@pytest.fixture(scope="module")
def source():
    return open(SRC).read()


def test_unmutated_oracle_passes_the_independent_checks(source, tmp_path):
    assert _pins_hold(_build(source, str(tmp_path), "orig"))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, source, tmp_path):
    old, new = MUTANTS[name]
    assert source.count(old) == 1, f"mutation anchor for {name} not found once"
    assert not _pins_hold(_build(source.replace(old, new), str(tmp_path), name))
