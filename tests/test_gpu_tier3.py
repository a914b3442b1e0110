"""Tier 3 (a persistent grid, Delta in global memory) against the oracle.

Tier 3 takes what the on-chip tiers do not: asymmetric instances and nonzero
diagonals (the general swap cost, reading R7 of the oracle), entries beyond
int8, random proposal order (section 2.1, reading R6), and N beyond a
cluster's capacity.  The bar is the same as everywhere: p, cost, accept count
and the final Delta bit-exact, no near-ties on either side.  Symmetric
instances are also forced onto tier 3 (QAPSA_TIER=3) so that the same
trajectories the other tiers are tested on pass through it, with short windows
(every CTA scans the whole window) and long ones (each CTA scans its own cells,
then a grid barrier).
"""
import numpy as np
import pytest

import oracle
from paper_1208_2675_gb300 import instances
from paper_1208_2675_gb300 import sa

pytestmark = pytest.mark.gpu


def general_instance(N, seed, sym=False, low=-60, high=100):
    rng = np.random.default_rng([seed, N, 0xA5])
    A = rng.integers(low, high, size=(N, N)).astype(np.int32)
    B = rng.integers(low, high, size=(N, N)).astype(np.int32)
    if sym:
        A = np.triu(A) + np.triu(A, 1).T
        B = np.triu(B) + np.triu(B, 1).T
    return A, B, rng.permutation(N).astype(np.int32)


def run_both(A, B, p0, *, I, iters=None, t0=0.5, tf=1e-3, seed=0, stream=0,
             random_order=False, splits=None, relative=True):
    n = I if iters is None else iters
    g = sa.Chain(A, B, p0, t0=t0, tf=tf, total_iters=I, seed=seed, stream_id=stream,
                 random_order=random_order, relative=relative)
    o = oracle.Chain(A, B, p0, t0=t0, tf=tf, total_iters=I, seed=seed, stream=stream,
                     random_order=random_order, relative=relative)
    for k in (splits or [n]):
        g.run(k)
    assert sum(splits or [n]) == n
    o.run(n)
    return g, o


def assert_same(g, o):
    p, cost, acc = g.result()
    st = o.state()
    info = g.info()
    assert info["tier"] == 3
    assert info["iterations"] == st["it"]
    assert acc == st["accepts"]
    assert cost == st["cost"]
    assert np.array_equal(p, st["p"])
    N = len(p)
    D = o.delta()
    assert np.array_equal(g.delta().astype(np.int64), D[np.triu_indices(N, 1)])
    assert info["near_ties"] == 0 and st["near_ties"] == 0
    return st


@pytest.mark.parametrize("N,I,seed", [(2, 3001, 1), (3, 5000, 2), (12, 10 ** 5, 1),
                                      (64, 300000, 5), (100, 10 ** 6, 1), (300, 40000, 32)])
def test_symmetric_instances_forced_onto_tier3(N, I, seed, monkeypatch):
    monkeypatch.setenv("QAPSA_TIER", "3")
    A, B, p0 = instances.taixxa_like(N, seed)
    g, o = run_both(A, B, p0, I=I, seed=seed, stream=seed)
    st = assert_same(g, o)
    assert N <= 3 or st["accepts"] > 100


def test_tier3_long_windows_and_run_splitting(monkeypatch):
    """A cold schedule: windows grow past 1024 proposals, so the CTAs scan
    their own cells and meet at a grid barrier per window; split into uneven
    launches."""
    monkeypatch.setenv("QAPSA_TIER", "3")
    A, B, p0 = instances.taixxa_like(120, 44)
    I = 600000
    g, o = run_both(A, B, p0, I=I, t0=0.05, tf=1e-4, seed=44,
                    splits=[1, 4095, 100000, 295904, 200000])
    st = assert_same(g, o)
    assert st["accepts"] > 200
    assert g.info()["windows"] < I / 200  # most windows were long


@pytest.mark.parametrize("N,I,sym", [(3, 4000, False), (5, 20000, False), (30, 100000, False),
                                     (100, 200000, False), (47, 100000, True),
                                     (257, 30000, False)])
def test_general_instances_match_the_oracle(N, I, sym):
    """Asymmetric A and B with nonzero diagonals (sym=False), and symmetric ones
    with nonzero diagonals (sym=True): the general swap cost."""
    A, B, p0 = general_instance(N, 70 + N, sym)
    g, o = run_both(A, B, p0, I=I, seed=N, stream=2)
    assert o.is_general()
    st = assert_same(g, o)
    assert st["accepts"] > 50


def test_wide_entries_match_the_oracle():
    """Symmetric, zero diagonal, entries up to 1000: beyond the int8 rows of the
    on-chip tiers, within the int32 bound 8 N max|A| max|B| < 2^31."""
    N = 60
    A, B, p0 = instances.taixxa_like(N, 5, low=0, high=1000)
    g, o = run_both(A, B, p0, I=200000, seed=5)
    st = assert_same(g, o)
    assert st["accepts"] > 100


@pytest.mark.parametrize("N,I,gen", [(2, 2001, False), (12, 10 ** 5, False),
                                     (100, 500000, False), (300, 40000, False),
                                     (40, 100000, True)])
def test_random_order_matches_the_oracle(N, I, gen):
    if gen:
        A, B, p0 = general_instance(N, 3, False)
    else:
        A, B, p0 = instances.taixxa_like(N, 17 + N)
    g, o = run_both(A, B, p0, I=I, seed=9, stream=4, random_order=True,
                    splits=[I // 3, I - I // 3])
    st = assert_same(g, o)
    assert st["accepts"] > 50


def test_random_order_hot_limit_accepts_everything():
    A, B, p0 = instances.taixxa_like(25, 6)
    I = 5000
    g, o = run_both(A, B, p0, I=I, t0=1e300, tf=1e300, relative=False, seed=3,
                    random_order=True)
    st = assert_same(g, o)
    assert st["accepts"] == I


def test_beyond_the_cluster_tier_matches_the_oracle():
    """N above the cluster tier's largest size: Delta (about 1.2 M cells) in
    global memory; a prefix of a cold-start schedule against the oracle."""
    N = sa.qap_sa_max_n_tier(2) + 100
    A, B, p0 = instances.taixxa_like(N, 88)
    g, o = run_both(A, B, p0, I=10 ** 9, iters=3000, t0=0.05, seed=88, splits=[1000, 2000])
    st = assert_same(g, o)
    assert st["accepts"] > 100


def test_wide_entries_beyond_the_int32_bound_are_refused():
    A, B, p0 = instances.taixxa_like(60, 5, low=0, high=3000)  # 8 N 3000^2 > 2^31
    with pytest.raises(sa.QapError) as e:
        sa.Chain(A, B, p0, t0=0.5, tf=1e-3, total_iters=10)
    assert e.value.status == sa.QAP_E_RANGE


def test_general_size_limit_and_batch_refusal():
    n4 = sa.qap_sa_max_n_tier(4)
    assert 1000 < n4 <= sa.qap_sa_max_n_tier(3)
    A, B, p0 = general_instance(n4 + 1, 1)
    with pytest.raises(sa.QapError) as e:
        sa.Chain(A, B, p0, t0=0.5, tf=1e-3, total_iters=10)
    assert e.value.status == sa.QAP_E_UNSUPPORTED
    A, B, p0 = general_instance(20, 2)
    with pytest.raises(sa.QapError) as e:
        sa.qap_batch_create([dict(A=A, B=B, p0=p0, t0=0.5, tf=1e-3, total_iters=100)])
    assert e.value.status == sa.QAP_E_UNSUPPORTED


def test_many_ctas_on_a_small_problem_over_a_long_run(monkeypatch):
    """76 CTAs on N = 12 (66 cells, most CTAs own none or one) over 2e7
    iterations: after the grid barrier of an accepted swap some CTAs scan the
    next short window while others have found its swap and update their cells.
    The swap reads one copy of Delta and writes the other, so the slow CTAs
    still read the cells they must; with one copy they would see cells of the
    next swap, take another decision and never meet the others at the barrier."""
    monkeypatch.setenv("QAPSA_TIER", "3")
    monkeypatch.setenv("QAPSA_T3_GRID", "76")
    A, B, p0 = instances.taixxa_like(12, 1)
    I = 2 * 10 ** 7
    g, o = run_both(A, B, p0, I=I, seed=1, stream=1, splits=[I // 2, I - I // 2])
    assert g.info()["ctas"] == 76
    st = assert_same(g, o)
    assert st["accepts"] > 1000


def test_a_grid_barrier_that_cannot_complete_times_out_cleanly(monkeypatch):
    """Failure detection without a fault: the grid barrier is made to expect one
    arrival more than the CTAs make (host-side injection), so every CTA's
    bounded wait (about two seconds) expires, the kernel returns, and the run
    reports QAP_E_TIMEOUT.  The device stays usable: a new chain on the same
    tier then matches the oracle."""
    import time
    monkeypatch.setenv("QAPSA_TIER", "3")
    A, B, p0 = instances.taixxa_like(60, 8)
    g = sa.Chain(A, B, p0, t0=0.5, tf=1e-3, total_iters=10 ** 5, seed=8)
    assert g.info()["tier"] == 3
    sa.qap_sa_inject_barrier_fault(g.h, True)
    t = time.perf_counter()
    with pytest.raises(sa.QapError) as e:
        g.run(10 ** 5)
    assert e.value.status == sa.QAP_E_TIMEOUT
    assert time.perf_counter() - t < 60
    g.close()
    g2, o = run_both(A, B, p0, I=10 ** 5, seed=8)
    st = assert_same(g2, o)
    assert st["accepts"] > 100


def test_the_injection_is_refused_off_the_grid_tier():
    A, B, p0 = instances.taixxa_like(30, 2)
    g = sa.Chain(A, B, p0, t0=0.5, tf=1e-3, total_iters=1000)
    with pytest.raises(sa.QapError) as e:
        sa.qap_sa_inject_barrier_fault(g.h, True)
    assert e.value.status == sa.QAP_E_UNSUPPORTED
