"""The benchmark's JSON line, on the CPU: the reference arm (the oracle timed on
the host cores) prints one line with the keys a caller of bench.py reads, and
the workload table names what the bench measures."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def reference_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=600, check=True, cwd=ROOT)
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_reference_arm_prints_the_contract_keys(reference_line):
    d = reference_line
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["metric"] == "sa_iterations_per_sec" and d["unit"] == "iter/s"
    assert d["higher_is_better"] is True and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_workloads_name_the_measured_configurations(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    w = bench.WORKLOADS
    assert w["c3"]["N"] == 1024 and w["c3"]["I"] == 2 * 10 ** 9 and w["c3"]["side"] == 32
    assert w["n100"]["N"] == 100 and w["n100"]["I"] == 10 ** 8
    assert w["n256"]["N"] == 256 and w["n256"]["I"] == 10 ** 9
    assert w["batch512"]["count"] == 512
    assert (w["batch512"]["n_lo"], w["batch512"]["n_hi"]) == (20, 300)
    assert (w["serve"]["n_lo"], w["serve"]["n_hi"]) == (30, 600)
    assert w["serve"]["rates"] == (100, 200, 500, 1000, 2000, 5000)
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    args = bench.parse()  # no flags: one GPU, the N = 1024 chain, >= 3 warm-up steps
    assert args.gpus == 1 and args.workload == "c3" and args.warmup >= 3


def test_steps_cover_the_whole_schedule():
    sys.path.insert(0, ROOT)
    import bench
    for K in (1, 3, 7, 20, 1000):
        p = bench.pieces(2 * 10 ** 9, K)
        assert len(p) == K and sum(p) == 2 * 10 ** 9 and min(p) > 0


def test_reference_arm_config_equals_ours(reference_line):
    sys.path.insert(0, ROOT)
    import bench
    assert reference_line["config"] == bench.config_of(bench.WORKLOADS["c3"])


def _peaks():
    return {"smem_bytes_per_clk_sm": 128.0, "sm_mhz": 2000.0, "sm_count": 152,
            "l2_gbs_sm": 200.0, "cta_barrier_ns": 50.0,
            "cluster_barrier_ns": {2: 180.0, 4: 175.0, 8: 185.0, 13: 183.0, 16: 188.0}}


def test_roofline_follows_the_dominant_kernel():
    """The roofline is computed for the kernel with the most event-timed device
    time: the hot-phase kernel by its own bytes (2N per proposal from L2, over
    the one-SM L2 rate), with the Delta-method count of the whole run beside it;
    otherwise the Delta-method count of the tier's SA kernel."""
    sys.path.insert(0, ROOT)
    import bench
    wl = {"N": 1000, "I": 10 ** 6}
    M = 1000 * 999 // 2
    info = {"iterations": 10 ** 6, "direct_iters": 6 * 10 ** 5, "direct_accepts": 9 * 10 ** 4,
            "hot_iters": 5 * 10 ** 5, "hot_accepts": 8 * 10 ** 4}
    accepts = 10 ** 5
    kt = {"hot": (4.0, 2), "sa": (1.0, 4), "aux": (0.01, 6)}
    rl = bench.roofline(wl, info, accepts, 5.0, _peaks(), 13, kt)
    assert rl["kernel"] == "sa_hot_kernel" and rl["bound"] == "l2"
    assert rl["achieved"] == pytest.approx(5 * 10 ** 5 * 2 * 1000 / 4.0 / 1e9)
    assert rl["frac"] == pytest.approx(rl["achieved"] / 200.0)
    assert rl["algorithmic_bytes_per_launch"] == pytest.approx(5 * 10 ** 5 * 2 * 1000 / 2)
    assert rl["share_of_device_time"] == pytest.approx(4.0 / 5.01)
    assert rl["latency"]["ns_per_accept"] == pytest.approx(4.0 / 8e4 * 1e9)
    dm = rl["delta_method"]
    algo = accepts * M * 10 + 4 * 10 ** 6
    assert dm["algorithmic_bytes"] == algo
    assert dm["frac"] == pytest.approx(algo / 5.0 / 1e9 / (128.0 * 2000.0 * 1e6 / 1e9 * 13))
    kt2 = {"hot": (0.5, 2), "sa": (4.0, 4), "aux": (0.01, 6)}
    rl2 = bench.roofline(wl, info, accepts, 5.0, _peaks(), 13, kt2)
    assert rl2["kernel"] == "sa_tier2_kernel" and rl2["bound"] == "smem"
    assert rl2["frac"] == pytest.approx(dm["frac"])
    rl1 = bench.roofline(wl, info, accepts, 5.0, _peaks(), 1, {"hot": (0.0, 0), "sa": (5.0, 1),
                                                             "aux": (0.0, 0)})
    assert rl1["kernel"] == "sa_tier1_kernel"
