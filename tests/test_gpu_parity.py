"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

The bar is bit-exact: Delta (int32 vs the oracle's int64), the permutation, the
int64 cost, the accept count and the binary64 schedule must be identical, and
both sides must report zero near-ties (|delta + T ln u| < 1e-9 T) -- a flip of
the Eq. (2) decision between CUDA's and libm's log could only happen there.
"""
import numpy as np
import pytest

import oracle
from paper_1208_2675_gb300 import instances
from paper_1208_2675_gb300 import sa

pytestmark = pytest.mark.gpu


def packed_upper(D):
    N = D.shape[0]
    return D[np.triu_indices(N, 1)]


def run_both(A, B, p0, *, t0, tf, I, relative=True, seed=0, stream=0, splits=None,
             oracle_iters=None):
    """Runs I iterations (or oracle_iters of them) on both sides; returns
    (gpu_state, oracle_state, gpu_delta_packed, oracle_delta_packed)."""
    n_run = I if oracle_iters is None else oracle_iters
    g = sa.Chain(A, B, p0, t0=t0, tf=tf, total_iters=I, relative=relative,
                 seed=seed, stream_id=stream)
    o = oracle.Chain(A, B, p0, t0=t0, tf=tf, total_iters=I, relative=relative,
                     seed=seed, stream=stream)
    if splits:
        done = 0
        for k in splits:
            g.run(k)
            done += k
        assert done == n_run
    else:
        g.run(n_run)
    o.run(n_run)
    p, cost, acc = g.result()
    info = g.info()
    gs = {"p": p, "cost": cost, "accepts": acc, "it": info["iterations"],
          "near_ties": info["near_ties"], "info": info,
          "near_log": [int(x) for x in g.near_tie_log()[0]]}
    os_ = o.state()
    os_["near_log"] = [int(x) for x in o.near_tie_log()[0]]
    out = (gs, os_, g.delta(), packed_upper(o.delta()), g, o)
    return out


def assert_same(gs, os_, gd, od):
    assert gs["it"] == os_["it"]
    assert gs["accepts"] == os_["accepts"]
    assert gs["cost"] == os_["cost"]
    assert np.array_equal(gs["p"], os_["p"])
    assert np.array_equal(gd.astype(np.int64), od)
    # a flip of an Eq. (2) decision between CUDA's and libm's log could only
    # occur at a near-tie; both sides log the iterations of theirs
    assert gs["near_log"] == os_["near_log"]
    assert gs["near_ties"] == 0 and os_["near_ties"] == 0


@pytest.mark.parametrize("N", [2, 3, 4, 12, 37, 100, 129, 200])
def test_setup_matches_oracle(N):
    A, B, p0 = instances.taixxa_like(N, 5 + N)
    g = sa.Chain(A, B, p0, t0=0.5, tf=1e-3, total_iters=1000)
    o = oracle.Chain(A, B, p0, t0=0.5, tf=1e-3, total_iters=1000)
    _, cost, acc = g.result()
    assert cost == o.state()["cost"] and acc == 0
    assert np.array_equal(g.delta().astype(np.int64), packed_upper(o.delta()))
    info = g.info()
    T0, Tf, alpha = o.schedule()
    assert (info["T0"], info["Tf"], info["alpha"]) == (T0, Tf, alpha)
    for it in [0, 1, 255, 256, 999]:
        assert g.temperature(it) == o.temperature(it)


def test_config_n12_full_run():
    """N = 12, uniform [0,99] symmetric, seed 1, random p0, T0 = 0.5 mean|Delta0|,
    Tf = 1e-3 T0, I = 1e5."""
    A, B, p0 = instances.taixxa_like(12, 1)
    gs, os_, gd, od, g, _ = run_both(A, B, p0, t0=0.5, tf=1e-3, I=10 ** 5)
    assert os_["accepts"] > 100
    assert_same(gs, os_, gd, od)


@pytest.mark.parametrize("N,I,seed", [(5, 20000, 2), (16, 100000, 3), (33, 200000, 4),
                                      (64, 300000, 5), (100, 1000000, 1),
                                      (129, 400000, 6), (160, 300000, 10), (200, 300000, 7)])
def test_trajectory_matches_oracle(N, I, seed):
    A, B, p0 = instances.taixxa_like(N, seed)
    gs, os_, gd, od, _, _ = run_both(A, B, p0, t0=0.5, tf=1e-3, I=I, seed=seed,
                                     stream=seed)
    assert os_["accepts"] > 0
    assert_same(gs, os_, gd, od)


def test_largest_tier1_size_partial_run():
    N = sa.qap_sa_max_n_tier(1)
    assert N >= 200
    A, B, p0 = instances.taixxa_like(N, 9)
    gs, os_, gd, od, g, _ = run_both(A, B, p0, t0=0.5, tf=1e-3, I=10 ** 7, seed=9,
                                     oracle_iters=60000)
    assert g.info()["tier"] == 1
    assert os_["accepts"] > 1000
    assert_same(gs, os_, gd, od)


def test_run_splitting_is_invisible():
    A, B, p0 = instances.taixxa_like(50, 8)
    I = 200000
    splits = [1, 2, 3, 1000, 4093, 77777, I - 1 - 2 - 3 - 1000 - 4093 - 77777]
    gs, os_, gd, od, _, _ = run_both(A, B, p0, t0=0.5, tf=1e-3, I=I, seed=8,
                                     splits=splits)
    assert_same(gs, os_, gd, od)


def test_handles_of_different_sizes_interleave():
    """A handle created after another, with a smaller (or larger) shared-memory
    footprint on the same kernel, must not affect the other's launches."""
    sizes = [230, 20, 320, 40]  # one-SM tier and cluster tier, large before small
    I = 20000
    chains, oracles = [], []
    for k, N in enumerate(sizes):
        A, B, p0 = instances.taixxa_like(N, 30 + k)
        chains.append(sa.Chain(A, B, p0, t0=0.5, tf=1e-3, total_iters=I, seed=k))
        oracles.append(oracle.Chain(A, B, p0, t0=0.5, tf=1e-3, total_iters=I, seed=k))
    for half in range(2):
        for g, o in zip(chains, oracles):
            g.run(I // 2)
            o.run(I // 2)
    for g, o in zip(chains, oracles):
        p, cost, acc = g.result()
        st = o.state()
        assert acc == st["accepts"] and cost == st["cost"]
        assert np.array_equal(p, st["p"])
        assert np.array_equal(g.delta().astype(np.int64), packed_upper(o.delta()))
        g.close()


def test_hot_limit_every_proposal_accepted():
    A, B, p0 = instances.taixxa_like(20, 3)
    I = 3000
    gs, os_, gd, od, _, _ = run_both(A, B, p0, t0=1e300, tf=1e300, I=I,
                                     relative=False)
    assert gs["accepts"] == I
    assert_same(gs, os_, gd, od)


def test_cold_limit_descent():
    A, B, p0 = instances.taixxa_like(40, 4)
    I = 200000
    gs, os_, gd, od, _, _ = run_both(A, B, p0, t0=1e-300, tf=1e-300, I=I,
                                     relative=False)
    assert_same(gs, os_, gd, od)
    assert gd.min() > 0  # a 2-swap local minimum


def test_n2_and_n3_degenerate():
    for N, seed in [(2, 1), (3, 2)]:
        A, B, p0 = instances.taixxa_like(N, seed)
        gs, os_, gd, od, _, _ = run_both(A, B, p0, t0=0.5, tf=1e-3, I=5001)
        assert_same(gs, os_, gd, od)
    A = np.array([[0, 5], [5, 0]], dtype=np.int32)
    B = np.array([[0, 3], [3, 0]], dtype=np.int32)
    g = sa.Chain(A, B, np.array([1, 0], dtype=np.int32), t0=0.5, tf=1e-3,
                 total_iters=1001)
    g.run(1001)
    p, cost, acc = g.result()
    assert acc == 1001 and list(p) == [0, 1] and cost == 30


def test_negative_entries_and_zero_matrix():
    rng = np.random.default_rng(3)
    N = 30
    A = np.zeros((N, N), dtype=np.int32)
    iu = np.triu_indices(N, 1)
    A[iu] = rng.integers(-127, 128, size=len(iu[0]))
    A = A + A.T
    B = np.zeros((N, N), dtype=np.int32)
    B[iu] = rng.integers(-127, 128, size=len(iu[0]))
    B = B + B.T
    p0 = rng.permutation(N).astype(np.int32)
    gs, os_, gd, od, _, _ = run_both(A, B, p0, t0=0.5, tf=1e-3, I=100000, seed=3)
    assert_same(gs, os_, gd, od)
    Z = np.zeros((N, N), dtype=np.int32)
    gs, os_, gd, od, _, _ = run_both(Z, B, p0, t0=0.5, tf=1e-3, I=1000)
    assert gs["accepts"] == 1000
    assert_same(gs, os_, gd, od)


def test_invalid_inputs_are_rejected():
    A, B, p0 = instances.taixxa_like(10, 1)
    kw = dict(t0=0.5, tf=1e-3, total_iters=100)
    # asymmetric A, a nonzero diagonal, entries beyond int8: accepted, on tier 3
    bad = A.copy()
    bad[0, 1] += 1
    assert sa.Chain(bad, B, p0, **kw).info()["tier"] == 3
    bad = B.copy()
    bad[3, 3] = 1
    assert sa.Chain(A, bad, p0, **kw).info()["tier"] == 3
    q = p0.copy()
    q[0] = q[1]
    with pytest.raises(sa.QapError) as e:
        sa.Chain(A, B, q, **kw)
    assert e.value.status == sa.QAP_E_INVAL
    big = A.copy()
    big[0, 1] = big[1, 0] = 128
    assert sa.Chain(big, B, p0, **kw).info()["tier"] == 3
    big[0, 1] = big[1, 0] = 1 << 20  # 8 N max|A| max|B| beyond 2^31 - 1
    with pytest.raises(sa.QapError) as e:
        sa.Chain(big, B, p0, **kw)
    assert e.value.status == sa.QAP_E_RANGE
    with pytest.raises(sa.QapError) as e:  # an unknown schedule flag
        sa.qap_sa_create(A, B, p0, sa.qap_schedule(0.5, 0.1, 100, 8, 0), 0)
    assert e.value.status == sa.QAP_E_INVAL
    with pytest.raises(sa.QapError) as e:
        sa.Chain(A, B, p0, t0=0.5, tf=0.0, total_iters=100)
    assert e.value.status == sa.QAP_E_INVAL
    g = sa.Chain(A, B, p0, **kw)
    g.run(60)
    with pytest.raises(sa.QapError) as e:
        g.run(41)
    assert e.value.status == sa.QAP_E_RANGE
    g.run(40)
    n = sa.qap_sa_max_n()
    A2, B2, p2 = instances.taixxa_like(n + 1, 1)
    with pytest.raises(sa.QapError) as e:
        sa.Chain(A2, B2, p2, **kw)
    assert e.value.status == sa.QAP_E_UNSUPPORTED


def test_device_pointer_entry_points_match_host_ones():
    torch = pytest.importorskip("torch")
    A, B, p0 = instances.taixxa_like(77, 12)
    kw = dict(t0=0.5, tf=1e-3, total_iters=300000, seed=12)
    h = sa.Chain(A, B, p0, **kw)
    h.run(300000)
    dev = torch.device("cuda:0")
    At, Bt, pt = (torch.from_numpy(x).to(dev) for x in (A, B, p0))
    s = torch.cuda.Stream()
    d = sa.Chain.from_device(At, Bt, pt, stream=s.cuda_stream, **kw)
    d.run(300000)
    p_out = torch.zeros(77, dtype=torch.int32, device=dev)
    c_out = torch.zeros(1, dtype=torch.int64, device=dev)
    a_out = torch.zeros(1, dtype=torch.int64, device=dev)
    sa.qap_sa_result_device(d.h, p_out.data_ptr(), c_out.data_ptr(), a_out.data_ptr())
    s.synchronize()
    hp, hc, ha = h.result()
    assert np.array_equal(p_out.cpu().numpy(), hp)
    assert int(c_out.item()) == hc and int(a_out.item()) == ha


@pytest.mark.parametrize("N,I", [(100, 10 ** 8)])
def test_full_size_single_chain_n100(N, I):
    """The N = 100, I = 1e8 single-chain workload, whole run, against the oracle."""
    A, B, p0 = instances.taixxa_like(N, 1)
    gs, os_, gd, od, _, _ = run_both(A, B, p0, t0=0.5, tf=1e-3, I=I, seed=1)
    assert_same(gs, os_, gd, od)


def test_n256_workload_prefix_matches_oracle():
    """N = 256 under the I = 1e9 schedule: the first 3e5 iterations (the
    high-acceptance start, where the 640-thread kernel's warp-only mode carries
    the chain) against the oracle, in three launches."""
    A, B, p0 = instances.taixxa_like(256, 1)
    gs, os_, gd, od, _, _ = run_both(A, B, p0, t0=0.5, tf=1e-3, I=10 ** 9, seed=1,
                                     oracle_iters=300000, splits=[100000, 100000, 100000])
    assert os_["accepts"] > 50000
    assert gs["info"]["warp_iters"] > 100000
    assert_same(gs, os_, gd, od)


@pytest.mark.parametrize("N,I,iters,seed", [(277, 10 ** 7, 40000, 31), (300, 10 ** 7, 30000, 32),
                                            (513, 10 ** 8, 8000, 33)])
def test_cluster_tier_matches_oracle(N, I, iters, seed):
    """Sizes beyond one SM: the chain runs on a thread-block cluster."""
    A, B, p0 = instances.taixxa_like(N, seed)
    gs, os_, gd, od, g, _ = run_both(A, B, p0, t0=0.5, tf=1e-3, I=I, seed=seed,
                                     stream=seed, oracle_iters=iters)
    assert g.info()["tier"] == 2
    assert os_["accepts"] > 500
    assert_same(gs, os_, gd, od)


def test_n1024_grid_workload_prefix_matches_oracle():
    """N = 1024: B = Manhattan distances on a 32 x 32 grid, A with 30 % nonzeros
    in [1, 10], I = 2e9 schedule; the first 4000 iterations against the oracle,
    run in two pieces."""
    A, B, p0 = instances.grid_instance(32, 1)
    gs, os_, gd, od, g, _ = run_both(A, B, p0, t0=0.5, tf=1e-3, I=2 * 10 ** 9, seed=1,
                                     oracle_iters=4000, splits=[1500, 2500])
    assert g.info()["tier"] == 2
    assert os_["accepts"] > 300
    assert_same(gs, os_, gd, od)


@pytest.mark.parametrize("N,rate", [(300, "0"), (300, "1e-9"), (300, "2e-3"), (300, "1.0"),
                                    (600, "1.0"), (600, "2e-3"), (280, "1e-9")])
def test_cluster_direct_and_delta_modes_give_the_same_trajectory(N, rate, monkeypatch):
    """The cluster tier's direct mode (each CTA evaluates the window's proposals
    whose row lies in its slice; Delta not maintained, rebuilt between launches)
    against the oracle.  rate = 0: Delta throughout; 1e-9: direct throughout;
    2e-3: the default; 1.0: direct for the first block, then Delta (the launch
    stops, Delta is rebuilt, a second launch continues).  Runs split across
    launches; Delta compared at the end."""
    monkeypatch.setenv("QAPSA_CLUSTER_HYBRID_RATE", rate)
    A, B, p0 = instances.taixxa_like(N, 47)
    I = 10 ** 7
    gs, os_, gd, od, g, _ = run_both(A, B, p0, t0=0.5, tf=1e-3, I=I, seed=47, stream=3,
                                     oracle_iters=60000, splits=[1, 29999, 30000])
    info = g.info()
    assert info["tier"] == 2
    assert os_["accepts"] > 1000
    assert_same(gs, os_, gd, od)
    if rate == "0":
        assert info["direct_iters"] == 0
    elif rate == "1.0":
        assert 0 < info["direct_iters"] < 60000
    else:
        assert info["direct_iters"] > 30000


def test_cluster_direct_mode_cold_run_matches_oracle(monkeypatch):
    """A whole short schedule on the cluster tier with the default switch point:
    direct mode through the hot part, Delta mode (after a rebuild) through the
    cold part, the final state and Delta against the oracle."""
    A, B, p0 = instances.taixxa_like(290, 48)
    I = 200000
    gs, os_, gd, od, g, _ = run_both(A, B, p0, t0=0.5, tf=1e-3, I=I, seed=48,
                                     splits=[70000, 70000, I - 140000])
    info = g.info()
    assert info["tier"] == 2 and 0 < info["direct_iters"] < I
    assert_same(gs, os_, gd, od)


@pytest.mark.parametrize("rate", ["0", "1e-9", "5e-4", "1.0"])
def test_direct_and_delta_modes_give_the_same_trajectory(rate, monkeypatch):
    """Proposals evaluated directly or read from the maintained Delta: the same
    exact integer either way.  rate = 0: Delta throughout; 1e-9: direct
    throughout; 5e-4: the default switch point; 1.0: switch after the first block."""
    monkeypatch.setenv("QAPSA_HYBRID_RATE", rate)
    A, B, p0 = instances.taixxa_like(64, 41)
    gs, os_, gd, od, g, _ = run_both(A, B, p0, t0=0.5, tf=1e-3, I=400000, seed=41,
                                     splits=[150000, 250000])
    assert os_["accepts"] > 1000
    assert_same(gs, os_, gd, od)


@pytest.mark.parametrize("N,warp_rate", [(64, "1e-9"), (64, "0"), (100, "1e-9"), (150, "1e-9"),
                                         (230, "1e-9"), (276, "1e-9"), (12, "1e-9"), (2, "1e-9"),
                                         (3, "1e-9")])
def test_warp_only_direct_mode_gives_the_same_trajectory(N, warp_rate, monkeypatch):
    """One warp evaluating proposals and applying swaps alone (windows of 32 to
    128, no block barrier) against the oracle; warp_rate 1e-9: whenever the
    chain is in direct mode, 0: never.  Runs split across launches.  The sizes
    cover the 256-thread kernel (one lane per proposal) and the 640-thread one
    (two lanes per proposal)."""
    monkeypatch.setenv("QAPSA_HYBRID_RATE", "5e-4")
    monkeypatch.setenv("QAPSA_WARP_RATE", warp_rate)
    A, B, p0 = instances.taixxa_like(N, 43)
    I = 300000
    gs, os_, gd, od, g, _ = run_both(A, B, p0, t0=0.5, tf=1e-3, I=I, seed=43,
                                     splits=[1, 99999, I - 100000])
    assert_same(gs, os_, gd, od)
    if warp_rate == "0":
        assert gs["info"]["warp_iters"] == 0
    elif N > 3:
        assert gs["info"]["warp_iters"] > 10000


def test_warp_mode_default_threshold_runs_and_matches():
    """The default thresholds on the N = 100 workload's schedule: the warp-only
    mode carries the hot start, the CTA modes the rest, one trajectory."""
    A, B, p0 = instances.taixxa_like(100, 1)
    gs, os_, gd, od, _, _ = run_both(A, B, p0, t0=0.5, tf=1e-3, I=10 ** 8, seed=1,
                                     oracle_iters=300000)
    assert_same(gs, os_, gd, od)
    assert gs["info"]["warp_iters"] > 100000


def test_n1024_grid_delta_mode_matches_oracle(monkeypatch):
    """N = 1024 grid instance on its 13-CTA cluster with Delta maintained from
    the first iteration (Delta tiles in the cluster's Tensor Memory, rows
    posted over distributed shared memory): 8000 iterations of a schedule
    over I = 2e9 from T0 = 0.05 mean|Delta0| (about 950 accepted swaps), in
    three launches, the final Delta element by element."""
    monkeypatch.setenv("QAPSA_CLUSTER_HYBRID_RATE", "0")
    A, B, p0 = instances.grid_instance(32, 1)
    gs, os_, gd, od, g, _ = run_both(A, B, p0, t0=0.05, tf=1e-3, I=2 * 10 ** 9, seed=1,
                                     oracle_iters=8000, splits=[1, 3999, 4000])
    info = g.info()
    assert info["tier"] == 2 and info["direct_iters"] == 0
    assert os_["accepts"] > 500
    assert_same(gs, os_, gd, od)


def test_largest_cluster_delta_mode_matches_oracle(monkeypatch):
    """The largest size the cluster tier takes (16 CTAs) in Delta mode, against
    the oracle after 10000 iterations, Delta element by element."""
    monkeypatch.setenv("QAPSA_CLUSTER_HYBRID_RATE", "0")
    N = sa.qap_sa_max_n_tier(2)
    assert N >= 1100
    A, B, p0 = instances.taixxa_like(N, 61)
    gs, os_, gd, od, g, _ = run_both(A, B, p0, t0=0.05, tf=1e-3, I=10 ** 9, seed=61,
                                     stream=5, oracle_iters=10000, splits=[4000, 6000])
    assert g.info()["tier"] == 2
    assert os_["accepts"] > 500
    assert_same(gs, os_, gd, od)


def test_n1024_grid_direct_then_delta_mode_matches_oracle(monkeypatch):
    """N = 1024 grid instance, a whole schedule of I = 40000 that crosses the
    cluster tier's mode switch: direct mode through the first block of 16384
    iterations (acceptance about 0.1), then below the threshold of 0.05 a stop,
    the Delta rebuild and Delta mode to the end; state and Delta against the
    oracle."""
    monkeypatch.setenv("QAPSA_CLUSTER_HYBRID_RATE", "0.05")
    A, B, p0 = instances.grid_instance(32, 2)
    I = 40000
    gs, os_, gd, od, g, _ = run_both(A, B, p0, t0=0.05, tf=1e-4, I=I, seed=2,
                                     splits=[20000, 20000])
    info = g.info()
    assert info["tier"] == 2 and 16384 <= info["direct_iters"] < I
    assert_same(gs, os_, gd, od)


@pytest.mark.parametrize("N,hot,rate,warps,I,iters,splits", [
    (300, "1", None, None, 300000, 300000, [100000, 200000]),
    (300, "0", None, None, 300000, 300000, [100000, 200000]),
    (300, "1", "0.1", "1", 300000, 300000, [100000, 200000]),
    (300, "1", "0.1", "16", 300000, 300000, [100000, 200000]),
    (300, "1", "1e-9", "5", 300000, 300000, [1, 149999, 150000]),
    (1024, "1", None, None, 2 * 10 ** 9, 4000, [1500, 2500]),
    (0, "1", None, "12", 10 ** 9, 2000, [700, 1300]),
])
def test_cluster_hot_phase_kernel_gives_the_same_trajectory(N, hot, rate, warps, I, iters,
                                                            splits, monkeypatch):
    """The hot-phase kernel of the cluster tier (one SM, rows of A and B' in L2
    staged by cp.async) forced on and off, on 1 to 16 warps; state and Delta
    against the oracle.  N = 300 under a schedule of 3e5 iterations, whose
    blocks of 16384 iterations accept 0.17, 0.062, 0.015, 0.0063, ... of their
    proposals: at the default rate 0.009 the kernel hands over after four
    blocks (Delta rebuilt, the cluster kernel in direct mode), at 0.1 after two;
    at 1e-9 it keeps the chain until the acceptance falls below the cluster
    tier's switch to Delta mode (2e-3, about the seventh block) and hands over
    in Delta mode.  N = 1024 (grid instance) and the largest cluster size
    (N = 0 here) under their long schedules: the hot kernel all along."""
    monkeypatch.setenv("QAPSA_HOT", hot)
    if rate:
        monkeypatch.setenv("QAPSA_HOT_RATE", rate)
    if warps:
        monkeypatch.setenv("QAPSA_HOT_WARPS", warps)
    if N == 1024:
        A, B, p0 = instances.grid_instance(32, 1)
    else:
        A, B, p0 = instances.taixxa_like(N or sa.qap_sa_max_n_tier(2), 35)
    gs, os_, gd, od, g, _ = run_both(A, B, p0, t0=0.5, tf=1e-3, I=I, seed=3, stream=1,
                                     oracle_iters=iters, splits=splits)
    info = g.info()
    assert info["tier"] == 2
    assert os_["accepts"] > 200
    assert_same(gs, os_, gd, od)
    blk, pas = 16384, 64  # a block ends with the pass that reaches 16384 iterations
    if hot == "0":
        assert info["hot_iters"] == 0
    elif N != 300:
        assert info["hot_iters"] == iters
    elif rate is None:
        assert 4 * blk <= info["hot_iters"] < 4 * (blk + pas)
    elif rate == "0.1":
        assert 2 * blk <= info["hot_iters"] < 2 * (blk + pas)
    else:
        assert 5 * blk < info["hot_iters"] < iters
