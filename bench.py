#!/usr/bin/env python
"""Benchmark: Delta-matrix simulated annealing for the QAP on GB300.

Default workload (the largest single-GPU configuration): one chain on the
N = 1024 structured instance -- B the Manhattan distances of a 32 x 32 grid, A
symmetric with 30 % nonzeros in [1, 10] -- over the whole geometric schedule
of I = 2e9 iterations (T0 = 0.5 mean|Delta0|, Tf = 1e-3 T0).  The K timed steps
are K consecutive pieces of that one run (I / K iterations each, the last one
takes the remainder), so the timed region is the whole schedule whatever K is.
The set-up (B', Delta0, C0 -- step (a) of section 2.2) is inside the first
step.  Warm-up steps run 1e6-iteration pieces of a separate chain of the same
instance and schedule.

The same run gives both numbers:
  value  iterations / device time (CUDA events on the chain's stream around
         the set-up and every piece; inputs already in HBM);
  e2e    iterations / host wall time of the same run through the public API,
         including the host-to-device copy of A, B, p0 from pinned memory and a
         device-to-host read of the result (p, cost, accepts) after every step.

Extra fields of the same line: the N = 100 (I = 1e8) and N = 256 (I = 1e9)
single-chain workloads, the 512-chain batch and a bounded serving sample, the
microbenchmarked peaks of this GPU (qap_peaks_measure), and the roofline of
the SA kernel by the method's algorithmic bytes.  With --gpus N (torchrun)
every rank runs an independent replica (own Philox stream); a single chain
does not shard, so work per GPU is fixed ("scaling": "weak").

--impl reference times the CPU oracle (one thread) on a bounded sample of the
same workload: consecutive 100-iteration pieces of the start of the same
schedule on the same instance, one piece per step.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "c3": dict(kind="grid", side=32, N=1024, I=2 * 10 ** 9, seed=1,
               desc="single chain, N=1024: B = Manhattan distances on a 32x32 grid, "
                    "A symmetric with 30% nonzeros uniform int [1,10], random p0, "
                    "geometric cooling T0=0.5*mean|Delta0|, Tf=1e-3*T0, I=2e9",
               cpu_iters=2000, ref_piece=100),
    "n100": dict(kind="uniform", N=100, I=10 ** 8, seed=1,
                 desc="single chain, N=100, A and B symmetric uniform int [0,99], "
                      "zero diagonal, random p0, geometric cooling "
                      "T0=0.5*mean|Delta0|, Tf=1e-3*T0, I=1e8",
                 cpu_iters=10 ** 7, ref_piece=10 ** 6),
    "n256": dict(kind="uniform", N=256, I=10 ** 9, seed=1,
                 desc="single chain, N=256, A and B symmetric uniform int [0,99], "
                      "zero diagonal, random p0, geometric cooling "
                      "T0=0.5*mean|Delta0|, Tf=1e-3*T0, I=1e9",
                 cpu_iters=5 * 10 ** 6, ref_piece=2 * 10 ** 5),
    "batch512": dict(count=512, n_lo=20, n_hi=300, I=10 ** 7, seed=4,
                     desc="512 independent chains, N ~ U{20..300}, uniform symmetric "
                          "int [0,99] instances (seed 1000+c, Philox stream c), "
                          "I=1e7 each, one persistent graph-captured launch"),
    "serve": dict(count=1000, rates=(100, 200, 500, 1000, 2000, 5000), n_lo=30, n_hi=600,
                  i_lo=1e6, i_hi=1e8, seed=5,
                  desc="Poisson solve requests, N log-uniform [30,600], I log-uniform "
                       "[1e6,1e8], uniform symmetric int [0,99] instances, continuous "
                       "batching"),
}
# The bounded serving sample reported beside the default workload.
SERVE_SAMPLE = dict(count=200, rates=(1000,))
WARMUP_PIECE = 10 ** 6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="c3")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the extra single-chain, batch and serving fields")
    return ap.parse_args()


def instance(wl):
    from paper_1208_2675_gb300 import instances
    if wl["kind"] == "grid":
        return instances.grid_instance(wl["side"], wl["seed"])
    return instances.taixxa_like(wl["N"], wl["seed"])


def config_of(wl):
    """The config dict both arms print (identical, so the lines compare)."""
    return {"workload": wl["desc"], "N": wl["N"], "I": wl["I"], "chains_per_gpu": 1,
            "schedule": "geometric, T0=0.5*mean|Delta0|, Tf=1e-3*T0",
            "l2": "inputs and state on chip; the SA kernel moves no DRAM bytes per "
                  "iteration (see roofline.traffic)"}


# --------------------------------------------------------------------------- #
# CPU oracle legs (the only places bench.py touches oracle/)
# --------------------------------------------------------------------------- #
def _oracle_prefix(wl, iters, q):
    import oracle
    A, B, p0 = instance(wl)
    t = time.perf_counter()
    c = oracle.Chain(A, B, p0, t0=0.5, tf=1e-3, total_iters=wl["I"], seed=wl["seed"])
    t_setup = time.perf_counter() - t
    t = time.perf_counter()
    c.run(iters)
    dt = time.perf_counter() - t
    q.put((t_setup, dt, c.state()["accepts"]))


def oracle_prefix_async(wl, iters):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    pr = ctx.Process(target=_oracle_prefix, args=(wl, iters, q))
    pr.start()
    return pr, q


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


# --------------------------------------------------------------------------- #
# clocks
# --------------------------------------------------------------------------- #
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # the samples go to QAPSA_CLOCKS_CSV if set, else to a temporary file
        self.path = os.environ.get("QAPSA_CLOCKS_CSV") or os.path.join(
            tempfile.gettempdir(), f"qapsa_clocks_gpu{gpu_index}_{os.getpid()}.csv")

    def start(self):
        os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- #
# roofline of the dominant kernel
# --------------------------------------------------------------------------- #
def delta_method_roofline(wl, info, accepts, t_kernel, peaks, sms_held):
    """The Delta-matrix method's bytes by its own count: an iteration reads one
    Delta cell (4 B); an accepted swap reads and writes every one of the M
    cells (8 B) and reads A and B' once for rows r,s (2 w B per cell, w = 1 for
    the int8 rows).  Peak: shared memory of the SMs the chain holds, at the
    measured bytes per clock and SM clock of this GPU.  The kernel moves no
    DRAM bytes per iteration: its state stays on chip."""
    N, I = wl["N"], info["iterations"]
    M = N * (N - 1) // 2
    w = 1
    algo = accepts * M * (8 + 2 * w) + 4 * I
    achieved = algo / t_kernel / 1e9
    per_sm = peaks["smem_bytes_per_clk_sm"] * peaks["sm_mhz"] * 1e6 / 1e9
    peak = per_sm * sms_held
    # what the kernels actually moved: a proposal evaluated directly reads rows
    # of A and B (4N on chip, or 2N from L2 in the hot-phase kernel), a direct
    # accept moves O(N) (6N), a proposal read from Delta is 4 B, an accept with
    # Delta maintained is 8M + 2N^2
    d_it, d_acc = info["direct_iters"], info["direct_accepts"]
    moved = d_it * 4 * N + d_acc * 6 * N + (I - d_it) * 4 + (accepts - d_acc) * (8 * M + 2 * N * N)
    nbar = 2  # hardware barriers per accepted swap (CTA or cluster)
    bar_ns = (peaks["cta_barrier_ns"] if sms_held == 1
              else max(v for v in peaks["cluster_barrier_ns"].values()))
    per_acc_ns = t_kernel / max(accepts, 1) * 1e9
    return {
        "bound": "smem", "achieved": achieved, "peak": peak, "unit": "GB/s",
        "frac": achieved / peak, "traffic": None,
        "algorithmic_bytes": algo,
        "bytes_basis": "accepts*M*(8+2w) + 4*I, w=1 (int8 A and B' rows)",
        "peak_basis": f"{sms_held} SM(s) x measured {peaks['smem_bytes_per_clk_sm']:.1f} B/clk "
                      f"x measured {peaks['sm_mhz']:.0f} MHz (qap_peaks_measure)",
        "frac_of_chip": achieved / (per_sm * peaks["sm_count"]),
        "moved_bytes": moved, "moved_frac": moved / t_kernel / 1e9 / peak,
        "latency": {"ns_per_accept": per_acc_ns,
                    "barrier_floor_ns_per_accept": nbar * bar_ns,
                    "frac_of_barrier_floor": nbar * bar_ns / per_acc_ns,
                    "basis": "two hardware barriers per accepted swap at the measured "
                             "barrier latency: the floor a chain of dependent accepts "
                             "cannot go below"},
    }


def roofline(wl, info, accepts, t_kernel, peaks, sms_held, ktimes=None):
    """The roofline of the kernel that takes most of the device time (CUDA
    events around every launch, qap_sa_kernel_times).  For the cluster tier's
    hot-phase kernel (one SM): a proposal streams rows A_s and B_p(s) (int8, 2N
    bytes) from L2 into shared memory and everything else stays on chip, so
    the bound is what one SM draws from L2 (measured, qap_peaks_measure
    l2_gbs_sm); an accepted swap is a dependent chain of two CTA barriers.  For
    the other kernels: the Delta-matrix method's count (delta_method_roofline),
    which is also reported beside the hot kernel's for the whole run."""
    dm = delta_method_roofline(wl, info, accepts, t_kernel, peaks, sms_held)
    if not ktimes or ktimes["hot"][0] <= ktimes["sa"][0]:
        if ktimes:
            dm["kernel"] = "sa_tier1_kernel" if sms_held == 1 else "sa_tier2_kernel"
            dm["share_of_device_time"] = ktimes["sa"][0] / max(1e-12, sum(v[0] for v in ktimes.values()))
        return dm
    N = wl["N"]
    t_hot, n_hot = ktimes["hot"]
    hot_it, hot_acc = info["hot_iters"], info["hot_accepts"]
    algo = hot_it * 2 * N
    achieved = algo / t_hot / 1e9
    peak = peaks["l2_gbs_sm"]
    per_acc_ns = t_hot / max(hot_acc, 1) * 1e9
    floor_ns = 2 * peaks["cta_barrier_ns"]
    total = sum(v[0] for v in ktimes.values())
    return {
        "bound": "l2", "kernel": "sa_hot_kernel", "achieved": achieved, "peak": peak,
        "unit": "GB/s", "frac": achieved / peak, "traffic": None,
        "algorithmic_bytes_per_launch": algo / max(n_hot, 1), "launches": n_hot,
        "avg_launch_s": t_hot / max(n_hot, 1),
        "bytes_basis": "2N per proposal evaluated: rows A_s and B_p(s), int8, streamed "
                       "from L2 (hot_iters x 2N over the kernel's event-timed seconds)",
        "peak_basis": f"measured ld.global.cg from L2 by one CTA of 1024 threads: "
                      f"{peak:.1f} GB/s (qap_peaks_measure l2_gbs_sm)",
        "share_of_device_time": t_hot / max(total, 1e-12),
        "kernel_seconds": {k: v[0] for k, v in ktimes.items()},
        "kernel_launches": {k: v[1] for k, v in ktimes.items()},
        "hot_iters": hot_it, "hot_accepts": hot_acc,
        "latency": {"ns_per_accept": per_acc_ns, "floor_ns_per_accept": floor_ns,
                    "frac_of_floor": floor_ns / per_acc_ns,
                    "basis": "two CTA barriers per accepted swap at the measured barrier "
                             "latency (the pass that finds it, the update)"},
        "delta_method": dm,
    }


# --------------------------------------------------------------------------- #
# our arm
# --------------------------------------------------------------------------- #
def pieces(I, K):
    base = I // K
    out = [base] * K
    out[-1] += I - base * K
    return out


def run_chain_workload(args, wl, rank, world, dev, dist, peaks, timed=True):
    """One whole run of a single-chain workload, in K pieces; returns a dict."""
    import torch
    from paper_1208_2675_gb300 import replicas, sa
    A, B, p0 = instance(wl)
    N, I = wl["N"], wl["I"]
    stream_id = replicas.stream_id_for(rank)
    kw = dict(t0=0.5, tf=1e-3, total_iters=I, seed=wl["seed"], stream_id=stream_id)
    Ah, Bh, ph = (torch.from_numpy(x).pin_memory() for x in (A, B, p0))
    At, Bt, pt = (torch.empty_like(x, device=dev) for x in (Ah, Bh, ph))
    stream = torch.cuda.Stream(dev)
    K = max(1, args.steps)

    # warm-up: 1e6-iteration pieces of a separate chain of the same schedule
    with torch.cuda.stream(stream):
        At.copy_(Ah)
        Bt.copy_(Bh)
        pt.copy_(ph)
    stream.synchronize()
    if args.warmup:
        hw = sa.Chain.from_device(At, Bt, pt, stream=stream.cuda_stream, **kw)
        for _ in range(args.warmup):
            hw.run(min(WARMUP_PIECE, I // (args.warmup + 1)))
        hw.close()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()

    clocks = Clocks(dev.index or 0) if timed else None
    if clocks:
        clocks.start()
    ev_set = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
    results = []
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):  # host -> device copies of the inputs
        At.copy_(Ah, non_blocking=True)
        Bt.copy_(Bh, non_blocking=True)
        pt.copy_(ph, non_blocking=True)
    ev_set[0].record(stream)
    h = sa.Chain.from_device(At, Bt, pt, stream=stream.cuda_stream, **kw)
    ev_set[1].record(stream)
    h.set_timing(True)
    for k, n in enumerate(pieces(I, K)):
        ev[k][0].record(stream)
        h.run_async(n)
        ev[k][1].record(stream)
        results.append(h.result())  # device -> host read of the step's result
    t1 = time.perf_counter()
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    h.sync()
    info = h.info()
    ktimes = h.kernel_times()
    h.close()
    t_setup = ev_set[0].elapsed_time(ev_set[1]) / 1e3
    t_pieces = [e[0].elapsed_time(e[1]) / 1e3 for e in ev]
    t_dev = t_setup + sum(t_pieces)
    t_dev_max = replicas.max_over_ranks(t_dev, dist, dev)
    t_e2e_max = replicas.max_over_ranks(t1 - t0, dist, dev)
    p_fin, cost_fin, acc_fin = results[-1]
    # kernels launched: the set-up (two classify kernels, pack, B', Gram,
    # Delta_0, and B as int8 for the hot kernel), then per launch of 2^26
    # iterations one SA
    # kernel (one SM), or on the cluster tier the hot kernel with its B' and
    # Delta rebuild (4) and two cluster launches each with a Delta rebuild (6)
    chunk = int(os.environ.get("QAPSA_CHUNK_ITERS", str(1 << 26)))
    hot = ktimes["hot"][1] > 0
    per_chunk = (10 if hot else 6) if info["tier"] == 2 else 1
    setup = 7 if hot else 6
    per_piece_launches = [-(-n // chunk) * per_chunk for n in pieces(I, K)]
    return {"N": N, "I": I, "t_dev": t_dev_max, "t_e2e": t_e2e_max, "t_setup": t_setup,
            "t_kernel": sum(t_pieces), "t_pieces": t_pieces, "info": info, "ktimes": ktimes,
            "accepts": acc_fin, "cost": cost_fin, "clocks": clk,
            "launches": setup + sum(per_piece_launches),
            "h2d": 2 * N * N * 4 + 4 * N, "d2h_per_step": 4 * N + 8 + 8}


def gpu_prefix_seconds(wl, iters, dev):
    """The GPU on the same prefix of the schedule the CPU baseline runs."""
    import torch
    from paper_1208_2675_gb300 import sa
    A, B, p0 = instance(wl)
    At, Bt, pt = (torch.from_numpy(x).to(dev) for x in (A, B, p0))
    stream = torch.cuda.Stream(dev)
    kw = dict(t0=0.5, tf=1e-3, total_iters=wl["I"], seed=wl["seed"])
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    h = sa.Chain.from_device(At, Bt, pt, stream=stream.cuda_stream, **kw)
    h.run(min(1000, iters))  # warm
    h.close()
    e[0].record(stream)
    h = sa.Chain.from_device(At, Bt, pt, stream=stream.cuda_stream, **kw)
    h.run_async(iters)
    e[1].record(stream)
    e[1].synchronize()
    _, _, acc = h.result()
    h.close()
    return e[0].elapsed_time(e[1]) / 1e3, acc


def run_ours(args, rank, world, local_rank, dist):
    import torch
    from paper_1208_2675_gb300 import sa
    wl = WORKLOADS[args.workload]
    dev = torch.device(f"cuda:{local_rank}")
    torch.cuda.set_device(dev)
    sa.lib()
    cpu_proc = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_proc, cpu_q = oracle_prefix_async(wl, wl["cpu_iters"])
    peaks = sa.qap_peaks_measure()
    r = run_chain_workload(args, wl, rank, world, dev, dist, peaks)
    info = r["info"]
    sms_held = info["ctas"]
    extras = {}
    if not args.no_extras and args.workload == "c3":
        for name in ("n100", "n256"):
            sub = argparse.Namespace(**{**vars(args), "steps": 1, "warmup": 1})
            x = run_chain_workload(sub, WORKLOADS[name], rank, world, dev, dist, peaks,
                                   timed=False)
            extras[name] = {"workload": WORKLOADS[name]["desc"],
                            "iterations_per_sec": world * x["I"] / x["t_dev"],
                            "e2e_iterations_per_sec": world * x["I"] / x["t_e2e"],
                            "accept_rate": x["accepts"] / x["I"],
                            "s_per_run": x["t_dev"],
                            "roofline": roofline(WORKLOADS[name], x["info"], x["accepts"],
                                                 x["t_kernel"], peaks, 1, x["ktimes"])}
        extras["batch512"] = batch_fields(rank, world, dev, dist, steps=1, warmup=1)
        if rank == 0:
            extras["serve_sample"] = serve_sweep(SERVE_SAMPLE["count"], SERVE_SAMPLE["rates"],
                                                 dev)
    if rank != 0:
        return
    I, N = wl["I"], wl["N"]
    value = world * I / r["t_dev"]
    acc = r["accepts"]
    rl = roofline(wl, info, acc, r["t_kernel"], peaks, sms_held, r["ktimes"])
    traffic = PROFILED_TRAFFIC.get(args.workload)
    if traffic:
        rl["traffic"] = traffic["bytes_per_launch"]
        rl["traffic_basis"] = traffic["basis"]
    M = N * (N - 1) // 2
    line = {
        "metric": "sa_iterations_per_sec",
        "value": value,
        "unit": "iter/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": r["t_dev"] / max(1, args.steps) * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32",
        "data": "synthetic (seeded instance of the configuration's family)",
        "config": config_of(wl),
        "steps_are": f"{args.steps} consecutive pieces of one whole run of I={I} "
                     "(set-up inside the first); warm-up: 1e6-iteration pieces of a "
                     "separate chain",
        "accept_rate": acc / I,
        "accepts": acc,
        "final_cost": r["cost"],
        "delta_cell_updates_per_sec": world * (acc - info["direct_accepts"]) * M / r["t_dev"],
        "direct_proposals_per_sec": world * info["direct_iters"] / r["t_dev"],
        "modes": {"hot_iters": info["hot_iters"], "hot_accepts": info["hot_accepts"],
                  "direct_iters": info["direct_iters"], "direct_accepts": info["direct_accepts"],
                  "delta_iters": I - info["direct_iters"],
                  "delta_accepts": acc - info["direct_accepts"], "tier": info["tier"],
                  "sms_held": sms_held},
        "sa_kernel_s": r["t_kernel"],
        "setup_s": r["t_setup"],
        "e2e": {"value": world * I / r["t_e2e"], "unit": "iter/s",
                "h2d_bytes_per_step": r["h2d"] / max(1, args.steps),
                "d2h_bytes_per_step": r["d2h_per_step"],
                "basis": "host wall time of the same run: pinned host->device copy of "
                         "A, B, p0 before the set-up, qap_sa_result after every step"},
        "gpu_launches": r["launches"],
        "roofline": rl,
        "peaks": peaks,
        "clocks": r["clocks"],
    }
    line.update(extras)
    if cpu_proc is not None:
        cpu_proc.join()
        t_setup_cpu, dt, acc_cpu = cpu_q.get()
        n = wl["cpu_iters"]
        t_gpu, acc_gpu = gpu_prefix_seconds(wl, n, dev)
        per_acc = dt / max(acc_cpu, 1)
        line["cpu_baseline"] = {
            "value": n / dt, "unit": "iter/s", "cores": 1, "kind": "oracle",
            "sample": f"iterations 0..{n - 1} of the same schedule on the same instance "
                      f"({acc_cpu} accepted swaps, a={acc_cpu / n:.3f}); {dt:.1f} s on "
                      f"{cpu_model()}; set-up {t_setup_cpu:.1f} s not included",
            "gpu_same_sample": {"value": n / t_gpu, "unit": "iter/s", "accepts": acc_gpu,
                                "note": "set-up included"},
            "oracle_whole_run_estimate_s": per_acc * acc,
        }
    print(json.dumps(line), flush=True)


# DRAM bytes of one launch of the dominant kernel from an ncu capture (null
# until captured for the current kernel).
PROFILED_TRAFFIC = {
    "c3": {"bytes_per_launch": 2186496,
           "basis": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one sa_hot_kernel "
                    "launch (the first 20000 iterations of the schedule): A and B (int8) "
                    "read into L2 once; the loop's rows stay in L2 and shared memory, so a "
                    "launch of any length moves the same bytes"},
}


# --------------------------------------------------------------------------- #
# reference arm: the CPU oracle
# --------------------------------------------------------------------------- #
def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    wl = WORKLOADS[args.workload]
    if "N" not in wl:
        print(json.dumps({"impl": "reference",
                          "unavailable": "the reference arm times single-chain workloads"}))
        return
    A, B, p0 = instance(wl)
    piece = wl["ref_piece"]
    c = oracle.Chain(A, B, p0, t0=0.5, tf=1e-3, total_iters=wl["I"], seed=wl["seed"])
    for _ in range(args.warmup):
        c.run(piece)
    a0 = c.state()["accepts"]
    ts = []
    for _ in range(args.steps):
        t = time.perf_counter()
        c.run(piece)
        ts.append(time.perf_counter() - t)
    total = sum(ts)
    acc = c.state()["accepts"] - a0
    value = args.steps * piece / total
    start = args.warmup * piece
    sample = (f"iterations {start}..{start + args.steps * piece - 1} of the same schedule "
              f"on the same instance, {piece} per step ({acc} accepted swaps); one thread "
              f"on {cpu_model()}")
    line = {
        "metric": "sa_iterations_per_sec", "value": value, "unit": "iter/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total / max(1, args.steps) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic (seeded instance of the configuration's family)",
        "config": config_of(wl),
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": "iter/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "iter/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- #
# batch of independent chains (one persistent graph-captured launch)
# --------------------------------------------------------------------------- #
def _batch_problems(wl):
    from paper_1208_2675_gb300 import instances
    sizes = instances.batch_sizes(wl["count"], wl["n_lo"], wl["n_hi"], wl["seed"])
    probs = []
    for c, N in enumerate(sizes):
        A, B, p0 = instances.taixxa_like(int(N), 1000 + c)
        probs.append(dict(A=A, B=B, p0=p0, t0=0.5, tf=1e-3, total_iters=wl["I"],
                          stream_id=c, seed=1000 + c))
    return probs


def _oracle_one_chain(job):
    sys.path.insert(0, ROOT)
    import oracle
    A, B, p0, kw, I = job
    c = oracle.Chain(A, B, p0, **kw)
    c.run(I)
    return c.state()["accepts"]


def _oracle_batch_chains(probs, I, q):
    """Whole oracle runs of the given chains, one worker process per core."""
    import concurrent.futures as cf
    jobs = [(pr["A"], pr["B"], pr["p0"], dict(t0=0.5, tf=1e-3, total_iters=I,
             seed=pr["seed"], stream=pr["stream_id"]), I) for pr in probs]
    cores = os.cpu_count() or 1
    t = time.perf_counter()
    with cf.ProcessPoolExecutor(max_workers=min(cores, len(jobs)),
                                mp_context=mp.get_context("spawn")) as ex:
        list(ex.map(_oracle_one_chain, jobs))
    q.put((time.perf_counter() - t, min(cores, len(jobs))))


def batch_fields(rank, world, dev, dist, steps=1, warmup=1):
    import torch  # noqa: F401
    from paper_1208_2675_gb300 import replicas, sa
    wl = WORKLOADS["batch512"]
    all_probs = _batch_problems(wl)
    I = wl["I"]
    parts = replicas.partition_by_cost(
        [replicas.chain_cost(len(pr["p0"]), I) for pr in all_probs], world)
    probs = [all_probs[i] for i in parts[rank]]

    def step():
        t0 = time.perf_counter()
        b = sa.qap_batch_create(probs)
        t1 = time.perf_counter()
        sa.qap_batch_run(b)
        t2 = time.perf_counter()
        acc = sum(sa.qap_batch_result(b, c, len(pr["p0"]))[2] for c, pr in enumerate(probs))
        sa.qap_batch_destroy(b)
        return t2 - t0, t2 - t1, acc

    for _ in range(warmup):
        step()
    if dist:
        dist.barrier()
    res = [step() for _ in range(steps)]
    t_step = replicas.max_over_ranks(statistics.mean(r[0] for r in res), dist, dev)
    t_run = replicas.max_over_ranks(statistics.mean(r[1] for r in res), dist, dev)
    # the plain single-chain path on the same GPU: the largest chains one after another
    single = []
    for pr in sorted(probs, key=lambda x: -len(x["p0"]))[:4]:
        h = sa.Chain(pr["A"], pr["B"], pr["p0"], t0=0.5, tf=1e-3, total_iters=I,
                     seed=pr["seed"], stream_id=pr["stream_id"])
        t = time.perf_counter()
        h.run(I)
        single.append((time.perf_counter() - t, len(pr["p0"])))
        h.close()
    n = len(all_probs)
    out = {"workload": wl["desc"], "chains_per_sec": n / t_step, "unit": "chains/s",
           "run_only_chains_per_sec": n / t_run, "iterations_per_sec": n * I / t_step,
           "accept_rate": statistics.mean(r[2] for r in res) / (len(probs) * I),
           "single_chain_path": {"chains_per_sec": len(single) / sum(t for t, _ in single),
                                 "sample": f"the {len(single)} largest chains run one after "
                                           f"another with qap_sa_run (N = "
                                           f"{[m for _, m in single]})"}}
    return out


def run_batch(args, rank, world, local_rank, dist):
    import torch
    from paper_1208_2675_gb300 import sa
    wl = WORKLOADS["batch512"]
    dev = torch.device(f"cuda:{local_rank}")
    torch.cuda.set_device(dev)
    sa.lib()
    cpu_proc = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        ctx = mp.get_context("spawn")
        cpu_q = ctx.Queue()
        sample = _batch_problems(wl)[:32]
        cpu_proc = ctx.Process(target=_oracle_batch_chains, args=(sample, wl["I"], cpu_q))
        cpu_proc.start()
    clocks = Clocks(local_rank)
    clocks.start()
    f = batch_fields(rank, world, dev, dist, steps=args.steps, warmup=args.warmup)
    clk = clocks.stop()
    if rank != 0:
        return
    line = {
        "metric": "batched_chains_per_sec", "value": f["chains_per_sec"], "unit": "chains/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": len(_batch_problems(wl)) / f["chains_per_sec"] * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (seeded Taixxa-like instances)",
        "config": {"workload": wl["desc"], "chains": wl["count"], "I": wl["I"]},
        **{k: v for k, v in f.items() if k not in ("chains_per_sec", "unit", "workload")},
        "clocks": clk,
    }
    if cpu_proc is not None:
        cpu_proc.join()
        dt, cores = cpu_q.get()
        line["cpu_baseline"] = {"value": 32 / dt, "unit": "chains/s", "cores": cores,
                                "kind": "oracle",
                                "sample": f"chains 0..31 of the same batch, whole runs, one "
                                          f"process per core ({dt:.1f} s)"}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- #
# serving: Poisson request streams through the continuous-batching server
# --------------------------------------------------------------------------- #
def serve_sweep(count, rates, dev):
    import numpy as np
    from paper_1208_2675_gb300 import instances, sa
    wl = WORKLOADS["serve"]
    out = []
    for rate in rates:
        arrival, Ns, Is = instances.request_mix(count, rate, wl["n_lo"], wl["n_hi"],
                                                wl["i_lo"], wl["i_hi"], wl["seed"] + rate)
        reqs = []
        for k in range(count):
            A, B, p0 = instances.taixxa_like(int(Ns[k]), 7000 + k)
            reqs.append(dict(A=A, B=B, p0=p0, t0=0.5, tf=1e-3, total_iters=int(Is[k]),
                             stream_id=k, seed=7000 + k))
        srv = sa.qap_server_start()
        t_start = time.perf_counter()
        tickets = []
        for k, pr in enumerate(reqs):
            delay = t_start + arrival[k] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.append(sa.qap_server_submit(srv, pr, pr["total_iters"]))
        done = [None] * len(reqs)
        while any(d is None for d in done):
            for k, t in enumerate(tickets):
                if done[k] is None:
                    done[k] = sa.qap_server_poll(srv, t, len(reqs[k]["p0"]))
            time.sleep(0.002)
        t_end = time.perf_counter()
        maxrun = sa.qap_server_max_running(srv)
        sa.qap_server_stop(srv)
        lat = np.array([d["latency_s"] for d in done])
        qs = np.array([d["queue_s"] for d in done])
        out.append({"rate_per_s": rate, "requests": len(reqs),
                    "p50_latency_s": float(np.percentile(lat, 50)),
                    "p99_latency_s": float(np.percentile(lat, 99)),
                    "p50_queue_s": float(np.percentile(qs, 50)),
                    "p99_queue_s": float(np.percentile(qs, 99)),
                    "completed_iterations_per_sec": float(sum(Is) / (t_end - t_start)),
                    "max_concurrent_requests": maxrun,
                    "wall_s": t_end - t_start})
    return out


def run_serve(args, rank, world, local_rank):
    if rank != 0:  # the serving sweep runs on one GPU
        return
    import torch
    from paper_1208_2675_gb300 import sa
    wl = WORKLOADS["serve"]
    dev = torch.device(f"cuda:{local_rank}")
    torch.cuda.set_device(dev)
    sa.lib()
    clocks = Clocks(local_rank)
    clocks.start()
    out = serve_sweep(wl["count"], wl["rates"], dev)
    clk = clocks.stop()
    line = {
        "metric": "serve_p99_latency_s", "value": out[-1]["p99_latency_s"], "unit": "s",
        "n_gpus": world, "steps": 1, "warmup": 0, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (seeded Taixxa-like instances, Poisson arrivals)",
        "config": {"workload": wl["desc"], "requests_per_rate": wl["count"]},
        "sweep": out, "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl")
        dist = tdist
    if args.workload == "batch512":
        run_batch(args, rank, world, local_rank, dist)
    elif args.workload == "serve":
        run_serve(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank, dist)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
