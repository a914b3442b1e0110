"""Run one SA chain on a seeded synthetic instance and print its result.

    python -m paper_1208_2675_gb300 --n 100 --total 1e8 --iters 2e6
    python -m paper_1208_2675_gb300 --grid 32 --total 2e9 --iters 1e5

The instance is the uniform symmetric one of instances.taixxa_like (or, with
--grid S, the S x S Manhattan-grid one of instances.grid_instance); the
schedule is geometric from T0 = t0 * mean|Delta_0| to Tf = tf * T0 over
--total iterations, of which the first --iters are run.  Prints the tier, the
iterations, the accepted swaps, the final cost and the wall time of the run
call as one JSON line.  Needs the built library and a GPU.
"""
import argparse
import json
import time

from . import instances, sa


def main() -> None:
    ap = argparse.ArgumentParser(prog="python -m paper_1208_2675_gb300")
    ap.add_argument("--n", type=int, default=100, help="problem size (uniform instance)")
    ap.add_argument("--grid", type=int, default=0, help="side of a grid instance (N = side^2)")
    ap.add_argument("--instance-seed", type=int, default=1)
    ap.add_argument("--total", type=float, default=1e8, help="iterations of the schedule")
    ap.add_argument("--iters", type=float, default=None, help="iterations to run (default: all)")
    ap.add_argument("--t0", type=float, default=0.5)
    ap.add_argument("--tf", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=1, help="Philox key of the chain")
    args = ap.parse_args()
    if args.grid:
        A, B, p0 = instances.grid_instance(args.grid, args.instance_seed)
    else:
        A, B, p0 = instances.taixxa_like(args.n, args.instance_seed)
    total = int(args.total)
    iters = total if args.iters is None else int(args.iters)
    g = sa.Chain(A, B, p0, t0=args.t0, tf=args.tf, total_iters=total, seed=args.seed)
    t = time.perf_counter()
    g.run(iters)
    dt = time.perf_counter() - t
    _, cost, acc = g.result()
    info = g.info()
    print(json.dumps({"N": len(p0), "tier": info["tier"], "iterations": info["iterations"],
                      "accepts": acc, "cost": cost, "run_s": dt,
                      "direct_iters": info["direct_iters"], "warp_iters": info["warp_iters"]}))
    g.close()


if __name__ == "__main__":
    main()
