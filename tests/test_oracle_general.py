"""Pins for the oracle's general-instance and random-order paths.

The general swap cost (asymmetric A or B, nonzero diagonals) and its O(1)
update are derived from Eq. (1); random proposal order is the reading of
section 2.1 (pairs may be drawn at random) stated in the oracle's header (R6).  Every
check uses a formulation other than the oracle's own: Eq. (1) over locations,
brute-force swap costs, the composition of transpositions, the published
Philox primitive, a chi-square test of the pair frequencies.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1208_2675_gb300 import instances


def cost_location_form(A, B, p):
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


def general_instance(N, seed, sym=False):
    rng = np.random.default_rng([seed, N, 0xA5])
    A = rng.integers(-60, 100, size=(N, N)).astype(np.int32)
    B = rng.integers(-60, 100, size=(N, N)).astype(np.int32)
    if sym:
        A = np.triu(A) + np.triu(A, 1).T
        B = np.triu(B) + np.triu(B, 1).T
    return A, B, rng.permutation(N).astype(np.int32)


def pairs(N):
    return [(r, s) for r in range(N) for s in range(r + 1, N)]


@pytest.mark.parametrize("N", [2, 3, 4, 5, 7, 9])
@pytest.mark.parametrize("sym", [False, True])
def test_general_swap_cost_equals_brute_force(N, sym):
    for seed in range(4):
        A, B, p = general_instance(N, seed, sym)
        D = brute_delta(A, B, p)
        for r, s in pairs(N):
            assert oracle.delta_entry_general(A, B, p, r, s) == D[r, s]
            assert oracle.delta_entry_general(A, B, p, s, r) == D[r, s]


def test_general_swap_cost_reduces_to_the_symmetric_form():
    A, B, p = instances.taixxa_like(11, 3)
    for r, s in pairs(11):
        assert oracle.delta_entry_general(A, B, p, r, s) == oracle.delta_entry(A, B, p, r, s)


def test_symmetric_form_fails_for_a_nonzero_diagonal():
    """The symmetric closed form needs zero diagonals: with nonzero diagonals in
    both matrices it differs from brute force, so the chain must use the
    general form there."""
    A, B, p = general_instance(6, 1, sym=True)
    D = brute_delta(A, B, p)
    assert any(oracle.delta_entry(A, B, p, r, s) != D[r, s] for r, s in pairs(6))
    c = oracle.Chain(A, B, p, t0=1.0, tf=0.1, total_iters=10, relative=False)
    assert c.is_general()
    assert not oracle.Chain(*instances.taixxa_like(6, 1), t0=1.0, tf=0.1, total_iters=10,
                            relative=False).is_general()


@pytest.mark.parametrize("N,sym", [(3, False), (5, False), (8, False), (12, False),
                                   (7, True), (16, False)])
def test_general_maintained_delta_matches_brute_force_after_every_accept(N, sym):
    A, B, p0 = general_instance(N, 20 + N, sym)
    I = 1500
    c = oracle.Chain(A, B, p0, t0=0.5, tf=1e-2, total_iters=I, seed=N, check=True,
                     log_cap=I)
    c.run(I)
    assert c.check_failures() == 0
    st = c.state()
    assert st["accepts"] > 10
    assert st["cost"] == cost_location_form(A, B, st["p"])
    assert np.array_equal(c.delta(), brute_delta(A, B, st["p"]))


def test_general_step_by_step_invariants():
    """C_new = C_old + Delta_rs and Delta_rs(after) = -Delta_rs(before) on every
    accepted swap of an asymmetric chain, one iteration at a time."""
    A, B, p0 = general_instance(7, 5)
    I = 600
    c = oracle.Chain(A, B, p0, t0=0.3, tf=1e-2, total_iters=I, seed=3)
    P = pairs(7)
    for it in range(I):
        before = c.state()
        D0 = c.delta()
        r, s = P[it % len(P)]
        c.run(1)
        after = c.state()
        if after["accepts"] > before["accepts"]:
            assert after["cost"] == before["cost"] + D0[r, s]
            assert c.delta()[r, s] == -D0[r, s]
            assert np.array_equal(after["p"], swapped(before["p"], r, s))
        else:
            assert np.array_equal(after["p"], before["p"])


@pytest.mark.parametrize("random_order", [False, True])
def test_general_traditional_sa_gives_the_same_trajectory(random_order):
    A, B, p0 = general_instance(9, 7)
    I = 5000
    kw = dict(t0=0.5, tf=1e-3, total_iters=I, seed=5, log_cap=I, random_order=random_order)
    d = oracle.Chain(A, B, p0, **kw)
    t = oracle.Chain(A, B, p0, **kw)
    d.run(I)
    t.run(I, traditional=True)
    assert np.array_equal(d.accept_log(), t.accept_log())
    sd, stt = d.state(), t.state()
    assert sd["cost"] == stt["cost"] and np.array_equal(sd["p"], stt["p"])


def _pair_by_definition(seed, stream, it, N):
    """Reading R6 written out: word 0 of Philox4x32-10 at counter
    (it low, it high, stream, 1), key (seed low, seed high); m = (x M) >> 32."""
    M = N * (N - 1) // 2
    x = int(oracle.philox4x32_10([it & 0xFFFFFFFF, it >> 32, stream, 1],
                                 [seed & 0xFFFFFFFF, seed >> 32])[0])
    return pairs(N)[(x * M) >> 32]


def test_random_proposals_follow_their_definition():
    A, B, p0 = instances.taixxa_like(13, 2)
    c = oracle.Chain(A, B, p0, t0=1.0, tf=0.1, total_iters=10, seed=2 ** 40 + 9, stream=6,
                     random_order=True)
    for it in [0, 1, 2, 3, 4, 5, 1000, 2 ** 32 - 1, 2 ** 32, 2 ** 33 + 5]:
        assert c.proposal(it) == _pair_by_definition(2 ** 40 + 9, 6, it, 13)
    seq = oracle.Chain(A, B, p0, t0=1.0, tf=0.1, total_iters=10)
    assert [seq.proposal(it) for it in range(80)] == [pairs(13)[it % 78] for it in range(80)]


def test_random_order_hot_limit_composes_the_drawn_transpositions():
    """T = 1e300: every proposal is accepted, so p is the composition of the
    transpositions drawn at it = 0 .. I-1."""
    N, I, seed = 10, 3000, 17
    A, B, p0 = instances.taixxa_like(N, 4)
    c = oracle.Chain(A, B, p0, t0=1e300, tf=1e300, total_iters=I, relative=False,
                     seed=seed, random_order=True)
    c.run(I)
    st = c.state()
    assert st["accepts"] == I
    q = np.array(p0, copy=True)
    for it in range(I):
        r, s = _pair_by_definition(seed, 0, it, N)
        q = swapped(q, r, s)
    assert np.array_equal(st["p"], q)
    assert np.array_equal(c.delta(), brute_delta(A, B, q))


def test_random_pairs_are_uniform():
    """Chi-square of the frequencies of the M = 45 pairs over 90000 draws."""
    N, n = 10, 90000
    c = oracle.Chain(*instances.taixxa_like(N, 1), t0=1.0, tf=0.1, total_iters=10, seed=3,
                     random_order=True)
    M = N * (N - 1) // 2
    index = {pq: k for k, pq in enumerate(pairs(N))}
    counts = np.zeros(M)
    for it in range(n):
        counts[index[c.proposal(it)]] += 1
    expected = n / M
    chi2 = float(((counts - expected) ** 2 / expected).sum())
    # 44 degrees of freedom: the 99.9 % quantile is about 78
    assert chi2 < 78.0
    assert counts.min() > 0


def test_random_order_chain_keeps_delta_exact():
    A, B, p0 = instances.taixxa_like(12, 8)
    I = 4000
    c = oracle.Chain(A, B, p0, t0=0.5, tf=1e-2, total_iters=I, seed=8, check=True,
                     random_order=True)
    c.run(I)
    assert c.check_failures() == 0
    st = c.state()
    assert st["accepts"] > 100 and st["cost"] == cost_location_form(A, B, st["p"])


def test_relative_schedule_of_a_general_instance():
    """T0 = t0 mean |Delta_0| over the M pairs from brute-force swap costs."""
    A, B, p0 = general_instance(8, 2)
    c = oracle.Chain(A, B, p0, t0=0.5, tf=1e-3, total_iters=1000)
    D = brute_delta(A, B, p0)
    mean = sum(abs(D[r, s]) for r, s in pairs(8)) / 28
    T0, Tf, alpha = c.schedule()
    assert T0 == 0.5 * mean and Tf == 1e-3 * T0
    assert math.isclose(alpha, (Tf / T0) ** (1 / 999), rel_tol=1e-15)
