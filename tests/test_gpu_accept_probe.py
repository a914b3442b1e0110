"""Eq. (2) at its edge, as the kernels decide it.

Most acceptance tests in a window are decided by a binary32 interval around the
threshold tau = -T(it) ln u(it); only swap costs inside the interval go on to
the binary64 rule.  Random trajectories rarely bring a swap cost within one
unit of tau, so here every probe does: delta = floor(tau) - 1 ... ceil(tau) + 1
at iterations drawn over the whole schedule (up to 2e9, plus the iterations
with the smallest and largest random words), for schedules with Tf/T0 from 1e-1
to 1e-12 and T0 from 3 to 1e7.  Both binary32 intervals the kernels use (the
prepared per-window tables and the in-window pre-test), the integer pre-filter
and the final decision must agree with the oracle's binary64 decision
everywhere except at near-ties (|delta + T ln u| < 1e-9 T), where two libm logs
may differ.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1208_2675_gb300 import instances
from paper_1208_2675_gb300 import sa

pytestmark = pytest.mark.gpu

SEED, STREAM = 77, 3


def _extreme_word_iterations(count: int):
    """Iterations in [0, 2^18) whose Philox words are the smallest and largest."""
    its = np.arange(1 << 18, dtype=np.uint64)
    words = np.array([oracle.rand_word(SEED, STREAM, int(i)) for i in its], dtype=np.uint64)
    order = np.argsort(words, kind="stable")
    return np.concatenate([its[order[:count]], its[order[-count:]]])


@pytest.fixture(scope="module")
def extreme_its():
    return _extreme_word_iterations(24)


@pytest.mark.parametrize("T0", [3.0, 100.0, 5.0e4, 1.0e7])
@pytest.mark.parametrize("ratio", [1e-1, 1e-3, 1e-6, 1e-12])
@pytest.mark.parametrize("I", [1000, 10 ** 6, 2 * 10 ** 9])
def test_binary32_pretest_never_contradicts_binary64(T0, ratio, I, extreme_its):
    A, B, p0 = instances.taixxa_like(3, 1)
    kw = dict(t0=T0, tf=T0 * ratio, total_iters=I, relative=False, seed=SEED)
    g = sa.Chain(A, B, p0, stream_id=STREAM, **kw)
    o = oracle.Chain(A, B, p0, stream=STREAM, **kw)
    rng = np.random.default_rng([int(math.log10(T0) * 10), int(-math.log10(ratio)), I % 9973])
    its = list(rng.integers(0, I, size=600)) + [0, 1, 2, 3, I - 1, I // 2, I - 4]
    its += [int(x) for x in extreme_its if int(x) < I]
    its = sorted(set(int(x) for x in its))
    p_it, p_it0, p_delta = [], [], []
    for it in its:
        T = o.temperature(it)
        u = oracle.uniform(SEED, STREAM, it)
        tau = -T * math.log(u)
        base = [math.floor(tau) - 1, math.floor(tau), math.ceil(tau), math.ceil(tau) + 1]
        for d in base:
            if not (1 <= d <= 2 ** 31 - 1):
                continue
            if abs(d - tau) < 1e-9 * T:  # a near-tie: either answer is the rule's
                continue
            j = int(rng.integers(0, min(it, 4095) + 1))
            p_it.append(it)
            p_it0.append(it - j)
            p_delta.append(d)
    assert len(p_it) > 100
    out = sa.qap_sa_accept_probe(g.h, p_it, p_it0, p_delta)
    want = np.array([o.accepts(d, it) for d, it in zip(p_delta, p_it)], dtype=np.int32)
    final = out & 1
    table = (out >> 2) & 3
    window = (out >> 4) & 3
    filt = (out >> 6) & 1
    assert np.array_equal(final, want)
    decided = table != 2
    assert np.array_equal(table[decided], want[decided])
    decided = window != 2
    assert np.array_equal(window[decided], want[decided])
    assert not np.any(want[filt == 1])  # the pre-filter rejects only true rejects
    assert not np.any((out >> 7) & 1)   # no probe was a near-tie for CUDA's log either
    g.close()


def test_probe_checks_its_arguments():
    A, B, p0 = instances.taixxa_like(3, 1)
    g = sa.Chain(A, B, p0, t0=10.0, tf=1.0, total_iters=100, relative=False)
    with pytest.raises(sa.QapError) as e:
        sa.qap_sa_accept_probe(g.h, [5], [6], [1])  # window starts after the proposal
    assert e.value.status == sa.QAP_E_RANGE
    assert len(sa.qap_sa_accept_probe(g.h, [], [], [])) == 0
    g.close()
