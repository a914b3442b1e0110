"""Knobs change the speed only: the same chain under different knobs (tier,
switch rates, CTAs of the grid tier) is bit-exact against the oracle; qap_tune
returns one of its candidates and checks that all candidates agree."""
import numpy as np
import pytest

import oracle
from paper_1208_2675_gb300 import instances, sa, tuner

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def clear_knobs():
    sa.qap_knobs_set(0, 0, None)
    yield
    sa.qap_knobs_set(0, 0, None)


@pytest.mark.parametrize("N,knobs", [
    (90, {"tier": 3}), (90, {"tier": 3, "t3_grid": 7}), (90, {"hybrid_rate": 2.5e-3}),
    (90, {"warp_rate": 0.05}), (400, {"cluster_hybrid_rate": 0.0}),
    (400, {"cluster_hybrid_rate": 0.01}), (400, {"tier": 3, "t3_grid": 40})])
def test_every_knob_gives_the_oracles_trajectory(N, knobs):
    A, B, p0 = instances.taixxa_like(N, 300 + N)
    I = 200000 if N < 200 else 20000
    sa.qap_knobs_set(N - 5, N + 5, knobs)
    g = sa.Chain(A, B, p0, t0=0.5, tf=1e-3, total_iters=I, seed=N)
    g.run(I // 2)
    g.run(I - I // 2)
    p, cost, acc = g.result()
    info = g.info()
    if knobs.get("tier") == 3:
        assert info["tier"] == 3
        if "t3_grid" in knobs:
            assert info["ctas"] == knobs["t3_grid"]
    o = oracle.Chain(A, B, p0, t0=0.5, tf=1e-3, total_iters=I, seed=N)
    o.run(I)
    st = o.state()
    assert acc == st["accepts"] and cost == st["cost"] and np.array_equal(p, st["p"])
    assert np.array_equal(g.delta().astype(np.int64), o.delta()[np.triu_indices(N, 1)])


def test_knob_ranges_apply_only_inside():
    A, B, p0 = instances.taixxa_like(50, 1)
    sa.qap_knobs_set(40, 60, {"tier": 3})
    assert sa.Chain(A, B, p0, t0=0.5, tf=1e-3, total_iters=10).info()["tier"] == 3
    A2, B2, q2 = instances.taixxa_like(70, 1)
    assert sa.Chain(A2, B2, q2, t0=0.5, tf=1e-3, total_iters=10).info()["tier"] == 1
    sa.qap_knobs_set(0, 0, None)
    assert sa.Chain(A, B, p0, t0=0.5, tf=1e-3, total_iters=10).info()["tier"] == 1


@pytest.mark.parametrize("N", [40, 300])
def test_tune_returns_a_candidate(N):
    knobs, t = sa.qap_tune(N, 200000)
    assert t > 0
    assert knobs["tier"] in (0, 3)
    table = {N: {"knobs": knobs}}
    tuner.apply(table)
    A, B, p0 = instances.taixxa_like(N, 5)
    g = sa.Chain(A, B, p0, t0=0.5, tf=1e-3, total_iters=1000)
    g.run(1000)
    o = oracle.Chain(A, B, p0, t0=0.5, tf=1e-3, total_iters=1000)
    o.run(1000)
    assert g.result()[1] == o.state()["cost"]
