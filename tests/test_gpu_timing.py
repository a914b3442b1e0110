"""Per-kernel device time of a chain's runs (qap_sa_set_timing /
qap_sa_kernel_times): CUDA events around every launch, counted by kind."""
import pytest

from paper_1208_2675_gb300 import instances
from paper_1208_2675_gb300 import sa

pytestmark = pytest.mark.gpu


def test_cluster_tier_times_the_hot_phase_the_cluster_kernel_and_the_rebuilds():
    A, B, p0 = instances.taixxa_like(300, 35)
    g = sa.Chain(A, B, p0, t0=0.5, tf=1e-3, total_iters=300000, seed=3, stream_id=1)
    g.set_timing(True)
    g.run(100000)
    g.run(200000)
    kt = g.kernel_times()
    info = g.info()
    assert info["tier"] == 2
    # one piece of each run: the hot kernel with its rebuild, two cluster launches
    # each followed by a Delta rebuild
    assert kt["hot"][1] == 2 and kt["sa"][1] == 4 and kt["aux"][1] == 6
    assert all(v[0] > 0.0 for v in kt.values())
    assert 0 < info["hot_accepts"] <= info["accepts"]
    assert 0 < info["hot_iters"] <= info["direct_iters"]
    assert g.kernel_times() == {"hot": (0.0, 0), "sa": (0.0, 0), "aux": (0.0, 0)}  # read once


def test_one_sm_tier_and_timing_off():
    A, B, p0 = instances.taixxa_like(100, 1)
    g = sa.Chain(A, B, p0, t0=0.5, tf=1e-3, total_iters=10 ** 6, seed=1)
    g.set_timing(True)
    g.run(500000)
    kt = g.kernel_times()
    assert kt["hot"] == (0.0, 0) and kt["aux"] == (0.0, 0)
    assert kt["sa"][1] == 1 and kt["sa"][0] > 0.0
    assert g.info()["hot_iters"] == 0
    g.set_timing(False)
    g.run(500000)
    assert g.kernel_times() == {"hot": (0.0, 0), "sa": (0.0, 0), "aux": (0.0, 0)}
