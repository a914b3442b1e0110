"""Pins for the CPU oracle against what the paper and the mathematics fix.

Every check here uses a formulation other than the oracle's own: the cost in
location space through p^-1, brute-force enumeration, Eq. (2) in its
exponential form, closed forms of special schedules, published Philox vectors.
A dropped term, a wrong sign or index, or a transposed operand in the oracle
fails at least one of them.
"""
import itertools
import math
import os
from decimal import Decimal, getcontext

import numpy as np
import pytest

import oracle
from paper_1208_2675_gb300 import instances

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- #
# Independent formulations used as pins
# --------------------------------------------------------------------------- #
def cost_location_form(A, B, p):
    """Eq. (1) rewritten over locations: sum_{x,y} A[q(x), q(y)] B[x, y], q = p^-1."""
    q = np.argsort(p)
    return int((A[np.ix_(q, q)].astype(np.int64) * B.astype(np.int64)).sum())


def swapped(p, r, s):
    q = np.array(p, copy=True)
    q[r], q[s] = q[s], q[r]
    return q


def brute_delta(A, B, p):
    N = len(p)
    c0 = cost_location_form(A, B, p)
    D = np.zeros((N, N), dtype=np.int64)
    for r in range(N):
        for s in range(r + 1, N):
            D[r, s] = D[s, r] = cost_location_form(A, B, swapped(p, r, s)) - c0
    return D


def pairs(N):
    return [(r, s) for r in range(N) for s in range(r + 1, N)]


# --------------------------------------------------------------------------- #
# Eq. (1)
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("N", [1, 2, 3, 7, 20])
def test_cost_equals_location_form_general_matrices(N):
    rng = np.random.default_rng(N)
    for _ in range(5):
        A = rng.integers(-50, 100, size=(N, N)).astype(np.int32)  # not symmetric
        B = rng.integers(-50, 100, size=(N, N)).astype(np.int32)
        p = rng.permutation(N).astype(np.int32)
        assert oracle.cost(A, B, p) == cost_location_form(A, B, p)


def test_cost_closed_forms():
    A, B, p = instances.taixxa_like(15, 3)
    ident = np.arange(15, dtype=np.int32)
    # p = identity: C = sum of the elementwise product.
    assert oracle.cost(A, B, ident) == int((A.astype(np.int64) * B).sum())
    # Uniform flows (all ones off the diagonal): C = sum_{x != y} B[x,y] for every p.
    J = (np.ones((15, 15)) - np.eye(15)).astype(np.int32)
    for s in range(5):
        q = np.random.default_rng(s).permutation(15).astype(np.int32)
        assert oracle.cost(J, B, q) == int(B.sum())


def test_enumeration_optimum_and_sa_quality():
    """N = 7: every permutation's cost matches the location form; slow SA finds
    the enumerated optimum for most seeds (a statistical sanity check)."""
    A, B, _ = instances.taixxa_like(7, 11)
    best = None
    for perm in itertools.permutations(range(7)):
        p = np.array(perm, dtype=np.int32)
        c = oracle.cost(A, B, p)
        assert c == cost_location_form(A, B, p)
        best = c if best is None else min(best, c)
    hits = 0
    for seed in range(10):
        p0 = np.random.default_rng(seed).permutation(7).astype(np.int32)
        ch = oracle.Chain(A, B, p0, t0=0.5, tf=1e-3, total_iters=20000, seed=seed)
        ch.run(20000)
        st = ch.state()
        assert st["cost"] == cost_location_form(A, B, st["p"])
        hits += st["cost"] == best
    assert hits >= 6


# --------------------------------------------------------------------------- #
# The swap cost change and step (a)
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("N", [2, 3, 4, 5, 7, 9])
def test_delta_closed_form_equals_bruteforce(N):
    for seed in range(6):
        A, B, p = instances.taixxa_like(N, seed)
        D = oracle.delta_matrix(A, B, p)
        assert np.array_equal(D, brute_delta(A, B, p))
        for r, s in pairs(N):
            assert oracle.swap_cost_change(A, B, p, r, s) == D[r, s]


def test_delta_closed_form_detects_asymmetry_assumption():
    """The closed form is for symmetric zero-diagonal data only; on a
    general instance it must differ from the brute force (the test would catch a
    closed form that silently claimed generality)."""
    rng = np.random.default_rng(5)
    A = rng.integers(0, 10, size=(6, 6)).astype(np.int32)
    B = rng.integers(0, 10, size=(6, 6)).astype(np.int32)
    p = rng.permutation(6).astype(np.int32)
    assert not np.array_equal(oracle.delta_matrix(A, B, p), brute_delta(A, B, p))


# --------------------------------------------------------------------------- #
# Step (d): Delta maintenance
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("N", [3, 4, 6, 9, 13, 16])
def test_delta_maintained_equals_bruteforce_after_every_accept(N):
    A, B, p0 = instances.taixxa_like(N, 100 + N)
    ch = oracle.Chain(A, B, p0, t0=0.5, tf=1e-2, total_iters=3000, seed=N, check=True)
    ch.run(3000)
    st = ch.state()
    assert st["accepts"] > 20
    assert ch.check_failures() == 0
    assert np.array_equal(ch.delta(), brute_delta(A, B, st["p"]))
    assert st["cost"] == cost_location_form(A, B, st["p"])


def test_accept_invariants_step_by_step():
    """C_new = C_old + Delta_rs and Delta_rs(after) = -Delta_rs(before)."""
    N = 8
    A, B, p0 = instances.taixxa_like(N, 4)
    ch = oracle.Chain(A, B, p0, t0=1e300, tf=1e300, total_iters=200, relative=False)
    order = pairs(N)
    for it in range(60):
        D0, st0 = ch.delta(), ch.state()
        ch.run(1)
        D1, st1 = ch.delta(), ch.state()
        r, s = order[it % len(order)]
        assert st1["accepts"] == st0["accepts"] + 1
        assert st1["cost"] == st0["cost"] + D0[r, s]
        assert D1[r, s] == -D0[r, s]
        assert np.array_equal(st1["p"], swapped(st0["p"], r, s))


# --------------------------------------------------------------------------- #
# The loop: traditional SA, special schedules, degenerate sizes
# --------------------------------------------------------------------------- #
@pytest.mark.parametrize("N,seed", [(5, 1), (8, 2), (12, 1), (16, 3)])
def test_traditional_sa_gives_identical_trajectory(N, seed):
    A, B, p0 = instances.taixxa_like(N, seed)
    kw = dict(t0=0.5, tf=1e-3, total_iters=20000, seed=seed, log_cap=20000)
    d = oracle.Chain(A, B, p0, **kw)
    t = oracle.Chain(A, B, p0, **kw)
    d.run(20000)
    t.run(20000, traditional=True)
    sd, st = d.state(), t.state()
    assert st["accepts"] == sd["accepts"] > 0
    assert np.array_equal(d.accept_log(), t.accept_log())
    assert np.array_equal(sd["p"], st["p"]) and sd["cost"] == st["cost"]


def test_hot_limit_accepts_everything():
    """T = 1e300: every proposal passes Eq. (2), so p is the composition of the
    transpositions pair(0), pair(1), ... in order."""
    N, I = 9, 500
    A, B, p0 = instances.taixxa_like(N, 7)
    ch = oracle.Chain(A, B, p0, t0=1e300, tf=1e300, total_iters=I, relative=False)
    ch.run(I)
    st = ch.state()
    q = np.array(p0, copy=True)
    order = pairs(N)
    for it in range(I):
        r, s = order[it % len(order)]
        q = swapped(q, r, s)
    assert st["accepts"] == I
    assert np.array_equal(st["p"], q)
    assert st["cost"] == cost_location_form(A, B, q)


def test_cold_limit_is_a_descent_to_a_two_swap_local_minimum():
    """T = 1e-300: only delta <= 0 is accepted, the cost never rises, and once a
    whole sweep of M proposals passes without an accept no swap improves."""
    N = 10
    M = N * (N - 1) // 2
    for seed in range(4):
        A, B, p0 = instances.taixxa_like(N, 20 + seed)
        I = 60 * M
        ch = oracle.Chain(A, B, p0, t0=1e-300, tf=1e-300, total_iters=I,
                          relative=False, log_cap=I)
        ch.run(I)
        log = ch.accept_log()
        st = ch.state()
        assert st["cost"] <= cost_location_form(A, B, p0)
        # replay: each accepted swap had delta <= 0
        q = np.array(p0, copy=True)
        order = pairs(N)
        for it in log:
            r, s = order[int(it) % M]
            c_before = cost_location_form(A, B, q)
            q = swapped(q, r, s)
            assert cost_location_form(A, B, q) <= c_before
        assert np.array_equal(q, st["p"])
        assert len(log) == 0 or log[-1] < I - M
        D = brute_delta(A, B, st["p"])
        assert D[np.triu_indices(N, 1)].min() > 0


def test_n2_every_iteration_accepts():
    A = np.array([[0, 5], [5, 0]], dtype=np.int32)
    B = np.array([[0, 3], [3, 0]], dtype=np.int32)
    p0 = np.array([1, 0], dtype=np.int32)
    ch = oracle.Chain(A, B, p0, t0=0.5, tf=1e-3, total_iters=1001)
    ch.run(1001)
    st = ch.state()
    assert st["accepts"] == 1001
    assert np.array_equal(st["p"], [0, 1])
    assert st["cost"] == 30


def test_acceptance_matches_eq2_exponential_form():
    """Replay a chain and check each decision against Eq. (2) as printed:
    accept iff delta < 0 or exp(-delta/T) > r."""
    N, I = 9, 4000
    A, B, p0 = instances.taixxa_like(N, 9)
    ch = oracle.Chain(A, B, p0, t0=0.5, tf=1e-2, total_iters=I, seed=77, log_cap=I)
    ch.run(I)
    accepted = set(int(x) for x in ch.accept_log())
    q = np.array(p0, copy=True)
    order = pairs(N)
    M = len(order)
    n_acc = 0
    for it in range(I):
        r, s = order[it % M]
        delta = cost_location_form(A, B, swapped(q, r, s)) - cost_location_form(A, B, q)
        T = ch.temperature(it)
        u = oracle.uniform(77, 0, it)
        want = delta <= 0 or math.exp(-delta / T) > u
        assert (it in accepted) == want, it
        if want:
            q = swapped(q, r, s)
            n_acc += 1
    assert n_acc == len(accepted) > 50


# --------------------------------------------------------------------------- #
# Random numbers
# --------------------------------------------------------------------------- #
def test_philox_known_answers():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(x, 16) for x in line.split()])
    assert len(rows) == 3
    for row in rows:
        out = oracle.philox4x32_10(row[0:4], row[4:6])
        assert [int(x) for x in out] == row[6:10]


def test_counter_layout_and_uniform_range():
    seed = 0x1234_5678_9ABC_DEF0
    for it in [0, 1, 2, 3, 4, 5, 1 << 33, (1 << 40) + 3]:
        blk = it // 4
        out = oracle.philox4x32_10([blk & 0xFFFFFFFF, blk >> 32, 7, 0],
                                   [seed & 0xFFFFFFFF, seed >> 32])
        x = oracle.rand_word(seed, 7, it)
        assert x == int(out[it % 4])
        assert oracle.uniform(seed, 7, it) == (x + 0.5) / 2 ** 32


def test_uniform_statistics():
    n = 40000
    u = np.array([oracle.uniform(5, 3, i) for i in range(n)])
    assert u.min() > 0 and u.max() < 1
    assert abs(u.mean() - 0.5) < 4 * math.sqrt(1 / 12 / n)
    counts, _ = np.histogram(u, bins=50, range=(0, 1))
    chi2 = ((counts - n / 50) ** 2 / (n / 50)).sum()
    assert chi2 < 100  # 49 dof; p ~ 3e-5 tail


# --------------------------------------------------------------------------- #
# Cooling schedule
# --------------------------------------------------------------------------- #
def test_schedule_geometric_and_relative_t0():
    N, I = 12, 10 ** 5
    A, B, p0 = instances.taixxa_like(N, 1)
    ch = oracle.Chain(A, B, p0, t0=0.5, tf=1e-3, total_iters=I)
    T0, Tf, alpha = ch.schedule()
    D = brute_delta(A, B, p0)
    mean_abs = np.abs(D[np.triu_indices(N, 1)]).sum() / (N * (N - 1) // 2)
    assert T0 == 0.5 * mean_abs
    assert Tf == 1e-3 * T0
    assert ch.temperature(0) == T0
    # alpha = pow(...) carries up to one ulp; compounded over I - 1 powers and the
    # table roundings this bounds T(I - 1) / Tf - 1 by about 2 I ulp.
    assert abs(ch.temperature(I - 1) / Tf - 1) < (2 * I + 64) * 2.0 ** -53
    getcontext().prec = 50
    a = Decimal(alpha)
    for it in [1, 2, 255, 256, 257, 65535, 65536, 77777, I - 1]:
        exact = Decimal(T0) * a ** it
        bound = (2 * it + 64) * 2.0 ** -53
        assert abs(Decimal(ch.temperature(it)) / exact - 1) <= Decimal(bound)


def test_schedule_monotone_up_to_rounding_long_run():
    A, B, p0 = instances.taixxa_like(6, 2)
    I = 2 * 10 ** 9
    ch = oracle.Chain(A, B, p0, t0=100.0, tf=0.1, total_iters=I, relative=False)
    rng = np.random.default_rng(0)
    its = list(rng.integers(0, I - 2, size=300)) + [255, 65535, (1 << 24) - 1, (1 << 30) - 1]
    for it in its:
        t0_, t1_ = ch.temperature(int(it)), ch.temperature(int(it) + 1)
        assert t1_ <= t0_ * (1 + 1e-6)
    assert abs(ch.temperature(I - 1) / 0.1 - 1) < 1e-6


def test_zero_delta_instance_uses_absolute_multipliers():
    N = 5
    A = np.zeros((N, N), dtype=np.int32)
    B, _, p0 = instances.taixxa_like(N, 1)
    ch = oracle.Chain(A, B, p0, t0=0.5, tf=1e-3, total_iters=100)
    T0, Tf, _ = ch.schedule()
    assert T0 == 0.5 and Tf == 0.5 * 1e-3
    ch.run(100)
    assert ch.state()["accepts"] == 100
