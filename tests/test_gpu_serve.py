"""Serving with continuous batching: requests that arrive while others run are
admitted and overlap on the device, and every result equals the oracle's for
the same request and the result of the same request run alone (bit-exact; the
arithmetic is integer and the trajectory is unique).  The mix includes
requests large enough for the cluster tier, which the server keeps in Delta
mode."""
import time

import numpy as np
import pytest

from paper_1208_2675_gb300 import instances
from paper_1208_2675_gb300 import sa

from oracle_pool import run_many

pytestmark = pytest.mark.gpu


def _requests():
    rng = np.random.default_rng(4)
    sizes = [30, 64, 100, 280, 45, 150, 200, 33, 90, 256, 120, 60, 300, 450, 600]
    reqs = []
    for c, N in enumerate(sizes):
        A, B, p0 = instances.taixxa_like(N, 200 + c)
        if N < 300:
            I, t0 = int(rng.integers(20000, 200000)), 0.5
        else:  # cluster tier: short, cooler runs the oracle finishes in seconds
            I, t0 = 8000, 0.05
        reqs.append(dict(A=A, B=B, p0=p0, t0=t0, tf=1e-3, total_iters=I,
                         stream_id=c, seed=200 + c))
    return reqs


def test_each_result_is_the_oracles_alone_and_in_the_mix():
    reqs = _requests()
    srv = sa.qap_server_start()
    try:
        tickets = []
        for pr in reqs:  # staggered arrivals: later ones come while earlier run
            tickets.append(sa.qap_server_submit(srv, pr, pr["total_iters"]))
            time.sleep(0.002)
        results = [None] * len(reqs)
        deadline = time.time() + 300
        while any(r is None for r in results) and time.time() < deadline:
            for i, t in enumerate(tickets):
                if results[i] is None:
                    results[i] = sa.qap_server_poll(srv, t, len(reqs[i]["p0"]))
            time.sleep(0.005)
        assert all(r is not None for r in results)
        assert sa.qap_server_max_running(srv) > 1  # requests overlapped
    finally:
        sa.qap_server_stop(srv)
    jobs = [(pr["A"], pr["B"], pr["p0"],
             dict(t0=pr["t0"], tf=pr["tf"], total_iters=pr["total_iters"], seed=pr["seed"],
                  stream=pr["stream_id"]), pr["total_iters"]) for pr in reqs]
    want = run_many(jobs)
    for pr, res, st in zip(reqs, results, want):
        assert res["status"] == 0
        assert res["accepts"] == st["accepts"] and res["cost"] == st["cost"], len(pr["p0"])
        assert np.array_equal(res["p"], st["p"])
        assert st["near_ties"] == 0
        alone = sa.Chain(pr["A"], pr["B"], pr["p0"], t0=pr["t0"], tf=pr["tf"],
                         total_iters=pr["total_iters"], seed=pr["seed"],
                         stream_id=pr["stream_id"])
        alone.run(pr["total_iters"])
        p, cost, acc = alone.result()
        alone.close()
        assert res["accepts"] == acc and res["cost"] == cost
        assert np.array_equal(res["p"], p)
        assert res["latency_s"] >= res["queue_s"] >= 0.0
