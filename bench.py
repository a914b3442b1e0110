#!/usr/bin/env python
"""Benchmark: Delta-matrix simulated annealing for the QAP on GB300.

One step = one whole single-chain SA run of the measured workload: set-up
(B', Delta_0, C0 -- step (a) of section 2.2), I iterations of the window
scan + Delta update (steps (b)-(e)), and the result.  With --gpus N (torchrun)
every rank runs an independent replica of the chain on its own GPU (a single
chain does not shard), so work per GPU is fixed ("scaling": "weak").

--impl reference times the CPU oracle (single thread) on a bounded sample of the
same workload: the full schedule of the same instance at I/10 iterations (I/200
for N = 256), which has the same acceptance rate a(I) as the full-length run.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "n100": dict(N=100, I=10 ** 8, seed=1, cpu_div=10,
                 desc="single chain, N=100, A and B symmetric uniform int [0,99], "
                      "zero diagonal, random p0, geometric cooling "
                      "T0=0.5*mean|Delta0|, Tf=1e-3*T0, I=1e8",
                 # ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch of
                 # sa_tier1_kernel<256> on this instance (2e6 iterations): the chain
                 # state and the code are read once per launch and everything stays
                 # on chip, so a launch of any length moves the same bytes
                 dram_bytes_per_launch=489984,
                 traffic_basis="ncu capture of one 2e6-iteration launch of the same "
                               "kernel on this instance; independent of the launch's "
                               "length (state on chip)"),
    "n256": dict(N=256, I=10 ** 9, seed=1, cpu_div=200,
                 desc="single chain, N=256, A and B symmetric uniform int [0,99], "
                      "zero diagonal, random p0, geometric cooling "
                      "T0=0.5*mean|Delta0|, Tf=1e-3*T0, I=1e9"),
    "batch512": dict(count=512, n_lo=20, n_hi=300, I=10 ** 7, seed=4,
                     desc="512 independent chains, N ~ U{20..300}, uniform symmetric "
                          "int [0,99] instances (seed 1000+c, Philox stream c), "
                          "I=1e7 each, one persistent graph-captured launch"),
    "serve": dict(count=100, rates=(100, 1000, 5000), n_lo=30, n_hi=600,
                  i_lo=1e6, i_hi=1e8, seed=5,
                  desc="Poisson solve requests, N log-uniform [30,600], I log-uniform "
                       "[1e6,1e8], uniform symmetric int [0,99] instances, continuous "
                       "batching; a bounded sample of 100 requests per rate"),
}
SMEM_BYTES_PER_CLK_PER_SM = 128  # 32 banks x 4 bytes


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="n100")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


# --------------------------------------------------------------------------- #
# CPU oracle legs (only place bench.py touches oracle/)
# --------------------------------------------------------------------------- #
def _oracle_sample(N: int, I: int, seed: int, q):
    import oracle
    from paper_1208_2675_gb300 import instances
    A, B, p0 = instances.taixxa_like(N, seed)
    c = oracle.Chain(A, B, p0, t0=0.5, tf=1e-3, total_iters=I, seed=seed)
    t = time.perf_counter()
    c.run(I)
    dt = time.perf_counter() - t
    q.put((dt, c.state()["accepts"]))


def oracle_sample_seconds(N: int, I: int, seed: int):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    pr = ctx.Process(target=_oracle_sample, args=(N, I, seed, q))
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
# our arm
# --------------------------------------------------------------------------- #
def run_ours(args, rank: int, world: int, local_rank: int, dist):
    import torch
    from paper_1208_2675_gb300 import instances, replicas, sa

    wl = WORKLOADS[args.workload]
    N, I, seed = wl["N"], wl["I"], wl["seed"]
    M = N * (N - 1) // 2
    dev = torch.device(f"cuda:{local_rank}")
    torch.cuda.set_device(dev)
    sa.lib()

    # CPU oracle baseline (rank 0, N=1): started first, runs beside the GPU work.
    cpu_proc = None
    I_sample = I // wl["cpu_div"]
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_proc, cpu_q = oracle_sample_seconds(N, I_sample, seed)

    A, B, p0 = instances.taixxa_like(N, seed)
    stream_id = replicas.stream_id_for(rank)  # independent replicas
    kw = dict(t0=0.5, tf=1e-3, total_iters=I, seed=seed, stream_id=stream_id)
    At, Bt, pt = (torch.from_numpy(x).to(dev) for x in (A, B, p0))
    p_out = torch.zeros(N, dtype=torch.int32, device=dev)
    c_out = torch.zeros(1, dtype=torch.int64, device=dev)
    a_out = torch.zeros(1, dtype=torch.int64, device=dev)
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.int32, device=dev)  # 256 MB > L2
    chunk = int(os.environ.get("QAPSA_CHUNK_ITERS", str(1 << 26)))
    sa_launches = -(-I // chunk)

    def step():
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        with torch.cuda.stream(stream):
            flush.fill_(1)
        ev[0].record(stream)
        h = sa.Chain.from_device(At, Bt, pt, stream=stream.cuda_stream, **kw)
        ev[1].record(stream)
        h.run_async(I)
        ev[2].record(stream)
        sa.qap_sa_result_device(h.h, p_out.data_ptr(), c_out.data_ptr(), a_out.data_ptr())
        ev[3].record(stream)
        ev[3].synchronize()
        h.sync()
        acc = int(a_out.item())
        info = h.info()
        h.close()
        return (ev[0].elapsed_time(ev[3]) / 1e3, ev[1].elapsed_time(ev[2]) / 1e3, acc,
                info["direct_iters"], info["direct_accepts"])

    for _ in range(args.warmup):
        step()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else local_rank)
    clocks.start()
    t_steps, t_sa, accs, dits, daccs = [], [], [], [], []
    for _ in range(args.steps):
        a, b, c, d, e = step()
        t_steps.append(a)
        t_sa.append(b)
        accs.append(c)
        dits.append(d)
        daccs.append(e)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total = sum(t_steps)
    total_max = replicas.max_over_ranks(total, dist, dev)

    # ---- end to end through the host-pointer API (pinned host buffers) ----
    Ah = torch.from_numpy(A).pin_memory()
    Bh = torch.from_numpy(B).pin_memory()
    ph = torch.from_numpy(p0).pin_memory()
    e2e_times = []
    for k in range(max(1, min(args.steps, 3)) + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = sa.Chain(Ah.numpy(), Bh.numpy(), ph.numpy(), **kw)
        h.run(I)
        p_res, cost_res, acc_res = h.result()
        dt = time.perf_counter() - t0
        h.close()
        if k:  # first one warms the host path
            e2e_times.append(dt)
    e2e_value = I / statistics.median(e2e_times)

    if rank != 0:
        return
    acc_mean = statistics.mean(accs)
    per_step = total_max / args.steps
    value = world * args.steps * I / total_max
    # roofline of sa_tier1_kernel: algorithmic shared-memory bytes of the work
    # done in a step -- a proposal evaluated directly reads rows r,s of A and B'
    # (4N), a directly handled accept moves O(N) (6N: rows r,s read, B' swapped),
    # a proposal read from Delta is 4 bytes, an accept with Delta maintained
    # reads and writes every cell (8M) and reads A and B' once (2N^2)
    d_it, d_acc = statistics.mean(dits), statistics.mean(daccs)
    bytes_step = (d_it * 4 * N + d_acc * 6 * N + (I - d_it) * 4 +
                  (acc_mean - d_acc) * (8 * M + 2 * N * N))
    t_kernel = statistics.mean(t_sa)
    achieved = bytes_step / t_kernel / 1e9
    mhz = clk.get("sm_mhz") or 2070.0
    peak = SMEM_BYTES_PER_CLK_PER_SM * mhz * 1e6 / 1e9  # one SM
    traffic = wl.get("dram_bytes_per_launch")
    line = {
        "metric": "sa_iterations_per_sec",
        "value": value,
        "unit": "iter/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": per_step * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "int32",
        "data": "synthetic (seeded Taixxa-like instance)",
        "config": {"workload": wl["desc"], "N": N, "I": I, "chains_per_gpu": 1,
                   "l2": "flushed between steps (256 MB write)",
                   "parallelism": f"replicas x{world}"},
        "delta_cell_updates_per_sec": world * acc_mean * M / per_step,
        "accept_rate": acc_mean / I,
        "direct_mode": {"iterations": d_it, "accepts": d_acc,
                        "note": "proposals evaluated directly while acceptance was high; "
                                "Delta maintained for the rest"},
        "sa_kernel_s_per_step": t_kernel,
        "e2e": {"value": e2e_value, "unit": "iter/s",
                "h2d_bytes_per_step": 2 * N * N * 4 + 4 * N,
                "d2h_bytes_per_step": 4 * N + 8 + 8},
        "gpu_launches": args.steps * (4 + sa_launches),
        "roofline": {"bound": "smem", "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "traffic_basis": wl.get("traffic_basis"),
                     "peak_basis": "one SM: 128 B/clk x median SM clock under load "
                                   "(derived; the kernel runs on one CTA)",
                     "frac_of_chip": achieved / (peak * 152)},
        "clocks": clk,
    }
    if cpu_proc is not None:
        cpu_proc.join()
        dt, acc_cpu = cpu_q.get()
        line["cpu_baseline"] = {
            "value": I_sample / dt, "unit": "iter/s", "cores": 1, "kind": "oracle",
            "sample": f"full schedule of the same N={N} instance at I={I_sample} "
                      f"(a(I)={acc_cpu / I_sample:.4f} vs {acc_mean / I:.4f} at I={I}); "
                      f"{dt:.1f} s on {cpu_model()}"}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- #
# reference arm: the CPU oracle
# --------------------------------------------------------------------------- #
def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    import oracle
    from paper_1208_2675_gb300 import instances
    wl = WORKLOADS[args.workload]
    N, seed = wl["N"], wl["seed"]
    I = wl["I"] // wl.get("cpu_div", 10)
    A, B, p0 = instances.taixxa_like(N, seed)

    def step():
        c = oracle.Chain(A, B, p0, t0=0.5, tf=1e-3, total_iters=I, seed=seed)
        t = time.perf_counter()
        c.run(I)
        return time.perf_counter() - t

    for _ in range(args.warmup):
        step()
    ts = [step() for _ in range(args.steps)]
    total = sum(ts)
    value = args.steps * I / total
    line = {
        "metric": "sa_iterations_per_sec", "value": value, "unit": "iter/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic (seeded Taixxa-like instance)",
        "config": {"workload": wl["desc"], "N": N, "I": wl["I"], "chains_per_gpu": 1,
                   "parallelism": "single CPU thread"},
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": "iter/s", "cores": 1, "kind": "oracle",
                         "sample": f"full schedule of the same instance at I={I} per step"},
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


def run_batch(args, rank, world, local_rank, dist):
    import torch
    from paper_1208_2675_gb300 import replicas, sa
    wl = WORKLOADS["batch512"]
    dev = torch.device(f"cuda:{local_rank}")
    torch.cuda.set_device(dev)
    all_probs = _batch_problems(wl)
    I = wl["I"]
    # replicas: this rank's share of the chains, balanced by estimated work
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

    for _ in range(args.warmup):
        step()
    if dist:
        dist.barrier()
    clocks = Clocks(local_rank)
    clocks.start()
    res = [step() for _ in range(args.steps)]
    clk = clocks.stop()
    t_step = replicas.max_over_ranks(statistics.mean(r[0] for r in res), dist, dev)
    t_run = replicas.max_over_ranks(statistics.mean(r[1] for r in res), dist, dev)
    # the plain single-chain path on the same GPU: chains one after another
    single = []
    for pr in probs[:6]:
        h = sa.Chain(pr["A"], pr["B"], pr["p0"], t0=0.5, tf=1e-3, total_iters=I,
                     seed=pr["seed"], stream_id=pr["stream_id"])
        t = time.perf_counter()
        h.run(I)
        single.append((time.perf_counter() - t, len(pr["p0"])))
        h.close()
    n = len(all_probs)
    per_chain = statistics.mean(t for t, _ in single)
    line = {
        "metric": "batched_chains_per_sec", "value": n / t_step, "unit": "chains/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic (seeded Taixxa-like instances)",
        "config": {"workload": wl["desc"], "chains": n, "I": I,
                   "sizes": "N ~ U{20..300}", "parallelism": f"replicas x{world}"},
        "run_only_chains_per_sec": n / t_run,
        "iterations_per_sec": n * I / t_step,
        "accept_rate": statistics.mean(r[2] for r in res) / (len(probs) * I),
        "single_chain_path": {"chains_per_sec": 1.0 / per_chain,
                              "sample": f"first {len(single)} chains run one after another "
                                        f"with qap_sa_run (N = {[m for _, m in single]})"},
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- #
# serving: Poisson request streams through the continuous-batching server
# --------------------------------------------------------------------------- #
def run_serve(args, rank, world, local_rank):
    if rank != 0:  # the serving sample runs on one GPU
        return
    import numpy as np
    import torch
    from paper_1208_2675_gb300 import instances, sa
    wl = WORKLOADS["serve"]
    dev = torch.device(f"cuda:{local_rank}")
    torch.cuda.set_device(dev)
    sa.lib()
    out = []
    for rate in wl["rates"]:
        arrival, Ns, Is = instances.request_mix(wl["count"], rate, wl["n_lo"], wl["n_hi"],
                                                wl["i_lo"], wl["i_hi"], wl["seed"] + rate)
        reqs = []
        for k in range(wl["count"]):
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
                    "completed_iterations_per_sec": float(sum(Is) / (t_end - t_start)),
                    "max_concurrent_requests": maxrun,
                    "wall_s": t_end - t_start})
    line = {
        "metric": "serve_p99_latency_s", "value": out[-1]["p99_latency_s"], "unit": "s",
        "n_gpus": world, "steps": 1, "warmup": 0, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (seeded Taixxa-like instances, Poisson arrivals)",
        "config": {"workload": wl["desc"]}, "sweep": out,
    }
    if rank == 0:
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
