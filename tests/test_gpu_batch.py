"""Batch of independent chains: every chain's result in the mix equals the
result of the same chain run alone (single-chain path) and the oracle's."""
import numpy as np
import pytest

import oracle
from paper_1208_2675_gb300 import instances
from paper_1208_2675_gb300 import sa

from oracle_pool import run_many

pytestmark = pytest.mark.gpu


def _problems(sizes, I, base_seed):
    probs = []
    for c, N in enumerate(sizes):
        A, B, p0 = instances.taixxa_like(int(N), base_seed + c)
        probs.append(dict(A=A, B=B, p0=p0, t0=0.5, tf=1e-3, total_iters=I,
                          stream_id=c, seed=base_seed + c))
    return probs


def test_batch_equals_single_chain_and_oracle():
    sizes = [5, 12, 37, 64, 100, 129, 160, 200, 256, 12, 100, 3, 2, 77, 150, 230]
    I = 30000
    probs = _problems(sizes, I, 1000)
    b = sa.qap_batch_create(probs)
    try:
        sa.qap_batch_run(b)  # every chain to its total_iters
        for c, pr in enumerate(probs):
            N = len(pr["p0"])
            p, cost, acc = sa.qap_batch_result(b, c, N)
            alone = sa.Chain(pr["A"], pr["B"], pr["p0"], t0=0.5, tf=1e-3, total_iters=I,
                             seed=pr["seed"], stream_id=pr["stream_id"])
            alone.run(I)
            p1, cost1, acc1 = alone.result()
            assert acc == acc1 and cost == cost1 and np.array_equal(p, p1), c
            if N <= 130:
                o = oracle.Chain(pr["A"], pr["B"], pr["p0"], t0=0.5, tf=1e-3, total_iters=I,
                                 seed=pr["seed"], stream=pr["stream_id"])
                o.run(I)
                st = o.state()
                assert acc == st["accepts"] and cost == st["cost"]
                assert np.array_equal(p, st["p"])
            assert sa.qap_batch_get_info(b, c)["iterations"] == I
    finally:
        sa.qap_batch_destroy(b)


def test_batch_mixes_one_sm_chains_and_cluster_chains():
    """N up to 300 (the batch workload's range): chains above one SM's limit run
    on clusters in a second persistent launch of the same graph."""
    sizes = [290, 20, 300, 150, 277, 64, 280]
    I = 6000
    probs = _problems(sizes, I, 500)
    b = sa.qap_batch_create(probs)
    try:
        sa.qap_batch_run(b)
        tiers = set()
        for c, pr in enumerate(probs):
            N = len(pr["p0"])
            p, cost, acc = sa.qap_batch_result(b, c, N)
            tiers.add(sa.qap_batch_get_info(b, c)["tier"])
            o = oracle.Chain(pr["A"], pr["B"], pr["p0"], t0=0.5, tf=1e-3, total_iters=I,
                             seed=pr["seed"], stream=pr["stream_id"])
            o.run(I)
            st = o.state()
            assert acc == st["accepts"] and cost == st["cost"], c
            assert np.array_equal(p, st["p"])
        assert tiers == {1, 2}
    finally:
        sa.qap_batch_destroy(b)


def test_batch_run_in_pieces_and_range_check():
    sizes = [20, 50, 90]
    I = 20000
    probs = _problems(sizes, I, 77)
    b = sa.qap_batch_create(probs)
    try:
        sa.qap_batch_run(b, [5000, 7000, 1])
        sa.qap_batch_run(b, [15000, 13000, 19999])
        with pytest.raises(sa.QapError) as e:
            sa.qap_batch_run(b, [1, 0, 0])
        assert e.value.status == sa.QAP_E_RANGE
        for c, pr in enumerate(probs):
            o = oracle.Chain(pr["A"], pr["B"], pr["p0"], t0=0.5, tf=1e-3, total_iters=I,
                             seed=pr["seed"], stream=pr["stream_id"])
            o.run(I)
            st = o.state()
            p, cost, acc = sa.qap_batch_result(b, c, len(pr["p0"]))
            assert acc == st["accepts"] and cost == st["cost"] and np.array_equal(p, st["p"])
    finally:
        sa.qap_batch_destroy(b)


def test_batch512_workload_against_oracle_and_alone():
    """The 512-chain workload itself -- N ~ U{20..300}, seed 1000 + c, Philox
    stream c, I = 1e7 each -- in one persistent graph launch, with every SM busy
    and chains finishing out of order.  Every chain equals the same chain run
    alone by the single-chain kernel (all 512 run side by side on their own
    streams), and 32 chains spread over the N range equal the oracle's whole
    run."""
    sizes = instances.batch_sizes(512, 20, 300, 4)
    I = 10 ** 7
    probs = _problems(sizes, I, 1000)
    b = sa.qap_batch_create(probs)
    try:
        sa.qap_batch_run(b)
        got = [sa.qap_batch_result(b, c, len(pr["p0"])) for c, pr in enumerate(probs)]
        tiers = {sa.qap_batch_get_info(b, c)["tier"] for c in range(len(probs))}
    finally:
        sa.qap_batch_destroy(b)
    assert tiers == {1, 2}
    alone = [sa.Chain(pr["A"], pr["B"], pr["p0"], t0=0.5, tf=1e-3, total_iters=I,
                      seed=pr["seed"], stream_id=pr["stream_id"]) for pr in probs]
    for h in alone:
        h.run_async(I)
    for c, h in enumerate(alone):
        h.sync()
        p1, cost1, acc1 = h.result()
        p, cost, acc = got[c]
        assert acc == acc1 and cost == cost1 and np.array_equal(p, p1), c
        h.close()
    by_n = np.argsort(sizes, kind="stable")
    pick = [int(by_n[k]) for k in np.linspace(0, len(sizes) - 1, 32).round().astype(int)]
    jobs = [(probs[c]["A"], probs[c]["B"], probs[c]["p0"],
             dict(t0=0.5, tf=1e-3, total_iters=I, seed=probs[c]["seed"],
                  stream=probs[c]["stream_id"]), I) for c in pick]
    for c, st in zip(pick, run_many(jobs)):
        p, cost, acc = got[c]
        assert acc == st["accepts"] and cost == st["cost"], (c, len(probs[c]["p0"]))
        assert np.array_equal(p, st["p"])
        assert st["near_ties"] == 0
