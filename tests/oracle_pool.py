"""Runs oracle chains in parallel worker processes (test helper).

The workers are started with the "spawn" method, so a test process that has
already used the GPU can use the pool (a process forked after CUDA is
initialised would hang).  Each job is one whole oracle run from its inputs.
"""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp
import os


def _run_one(job):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import oracle
    A, B, p0, kw, iters = job
    o = oracle.Chain(A, B, p0, **kw)
    o.run(iters)
    st = o.state()
    return {"p": st["p"], "cost": st["cost"], "accepts": st["accepts"], "it": st["it"],
            "near_ties": st["near_ties"]}


def run_many(jobs, workers: int | None = None):
    """jobs: (A, B, p0, oracle.Chain keyword arguments, iterations) tuples.
    Returns the final states in the order of the jobs."""
    if not jobs:
        return []
    n = workers or max(1, min(len(jobs), os.cpu_count() or 1))
    with cf.ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_run_one, jobs))
