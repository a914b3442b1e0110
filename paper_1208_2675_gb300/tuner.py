"""Autotuner of the library's knobs (none of which changes a trajectory).

The paper leaves the size of the window of proposals tested in parallel as an
adjustable parameter (section 3 (ii)).  This library adapts the window at run
time and has further knobs that change only the speed: the tier of a chain
(on-chip or the grid tier), the acceptance rates at which the one-SM and the
cluster tiers switch between reading swap costs from Delta and evaluating them
directly, the rate from which one warp runs the direct mode alone, and the CTAs
of a grid-tier chain.  ``qap_tune`` (C ABI) times the candidates for one N on the
current GPU; this module tunes a set of sizes, keeps the choices in a JSON table
keyed by N (each entry covers the sizes nearest to it), and installs the table
with ``qap_knobs_set``.

    python -m paper_1208_2675_gb300.tuner --sizes 60,100,150,200,256,300,600,1024 \\
        --out tuned.json
"""
from __future__ import annotations

import argparse
import json
import time

from . import sa


def tuning_iters(N: int) -> int:
    """Iterations of a trial schedule: long enough for the hot start, the
    switch to Delta mode and a cold tail, short enough for seconds per trial."""
    return int(min(2 * 10 ** 7, max(10 ** 6, 4e9 / (N * N))))


def tune(sizes, iters_for=tuning_iters, log=print) -> dict:
    """{N: {"knobs": {...}, "seconds": t, "iters": I}} for each size."""
    table = {}
    for N in sizes:
        I = iters_for(N)
        t = time.perf_counter()
        knobs, best = sa.qap_tune(int(N), I)
        table[int(N)] = {"knobs": knobs, "seconds": best, "iters": I}
        if log:
            log(f"N={N} I={I}: {knobs} best {best:.3f} s (tuning {time.perf_counter() - t:.1f} s)")
    return table


def ranges(table: dict) -> list[tuple[int, int, dict]]:
    """Splits [2, inf) among the tuned sizes: each size covers the N closer to
    it than to its neighbours."""
    sizes = sorted(int(n) for n in table)
    out = []
    for i, n in enumerate(sizes):
        lo = 2 if i == 0 else (sizes[i - 1] + n) // 2 + 1
        hi = 2 ** 31 - 1 if i == len(sizes) - 1 else (n + sizes[i + 1]) // 2
        out.append((lo, hi, table[n]["knobs"] if "knobs" in table[n] else table[n]))
    return out


def save(path: str, table: dict, meta: dict | None = None) -> None:
    with open(path, "w") as f:
        json.dump({"meta": meta or {}, "table": {str(k): v for k, v in table.items()}},
                  f, indent=1, sort_keys=True)


def load(path: str) -> dict:
    with open(path) as f:
        d = json.load(f)
    return {int(k): v for k, v in d["table"].items()}


def apply(table: dict) -> None:
    """Installs the table: qap_knobs_set for every range (earlier ranges cleared)."""
    sa.qap_knobs_set(0, 0, None)
    for lo, hi, knobs in ranges(table):
        sa.qap_knobs_set(lo, hi, knobs)


def main() -> None:
    ap = argparse.ArgumentParser(prog="python -m paper_1208_2675_gb300.tuner")
    ap.add_argument("--sizes", default="60,100,150,200,256,300,600,1024")
    ap.add_argument("--out", required=True)
    args = ap.parse_args()
    sizes = [int(x) for x in args.sizes.split(",")]
    table = tune(sizes)
    save(args.out, table, {"sizes": sizes, "how": "qap_tune, one trial run per candidate"})


if __name__ == "__main__":
    main()
