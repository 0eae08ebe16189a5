"""The register-resident chain kernel (FP32 mRNA/protein log-likelihood):
bit-identical to the shared-memory chain kernel on single-member observation
groups (same operation order per state), and within the FP32 tolerance of the
oracle, over box shapes that exercise ragged column quads, odd row counts and
clusters of 1, 2, 3, 4 and 8 CTAs; every state of a band observed (each
thread summing an observation per register slot); ten runs of the same launch
identical bit for bit; the hand-over of the rows that cross a CTA boundary
reports a wait that runs out."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

PER_OBS_FP32 = 5e-5  # per observation, derived in test_parity_gpu.py


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_05647_gb300 import build as lib_build
    lib_build.build()
    torch.cuda.set_device(0)


def _case(dims, theta, times, cells, seed):
    snaps = synth.gillespie_snapshots(synth.MRNA_PROT2D, dims, theta, times, cells, synth.rng(2, seed))
    obs = synth.snapshot_obs(synth.MRNA_PROT2D, dims, snaps)
    n = dims[0] * dims[1]
    return obs, synth.delta(n, 0)


def _loglik(dims, theta, thetas, times, obs, rho0, chain, threads=0):
    import paper_2312_05647_gb300 as mjp
    m = mjp.Model(synth.MRNA_PROT2D, dims, theta, mjp.FP32)
    m.set_option(mjp.OPT_CHAIN, chain)
    if threads:
        m.set_option(mjp.OPT_THREADS, threads)
    o = mjp.Obs(dims[0] * dims[1], times, obs, rho0)
    ll = mjp.loglik(m, o, thetas)
    m.check()
    return ll


@pytest.mark.parametrize("dims,theta", [
    ((30, 40), (8.0, 1.0, 1.0, 0.3)),        # 1 CTA, two padding columns in the last quad
    ((37, 53), (10.0, 1.0, 1.5, 0.4)),       # odd rows, three padding columns
    ((200, 200), (20.0, 1.0, 5.0, 0.1)),     # the benchmark box: 2 CTAs, 10 rows per thread
    ((120, 330), (15.0, 1.0, 2.0, 0.2)),     # 2 CTAs, uneven split
    ((136, 401), (12.0, 1.0, 2.0, 0.15)),    # 3 CTAs, odd rows, short last CTA
])
def test_register_chain_is_bitwise_equal_to_shared_memory_chain(dims, theta):
    times = np.array([0.05, 0.2, 0.6, 1.5])
    obs, rho0 = _case(dims, theta, times, 30, seed=sum(dims))
    thetas = synth.jitter(theta, 3, 0.2, synth.rng(2, 7))
    a = _loglik(dims, theta, thetas, times, obs, rho0, 1)
    b = _loglik(dims, theta, thetas, times, obs, rho0, 2)
    assert np.all(np.isfinite(a))
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("dims,theta", [((200, 200), (20.0, 1.0, 5.0, 0.1)), ((136, 401), (12.0, 1.0, 2.0, 0.15))])
def test_register_chain_two_ctas_per_sm_variant_is_bitwise_equal(dims, theta):
    # OPT_THREADS = 256 selects 256-thread CTAs (two per SM, more CTAs per cluster).
    times = np.array([0.05, 0.2, 0.6])
    obs, rho0 = _case(dims, theta, times, 30, seed=sum(dims) + 1)
    thetas = synth.jitter(theta, 2, 0.2, synth.rng(2, 17))
    a = _loglik(dims, theta, thetas, times, obs, rho0, 1)
    b = _loglik(dims, theta, thetas, times, obs, rho0, 2, threads=256)
    np.testing.assert_array_equal(a, b)


def test_register_chain_refuses_other_thread_counts():
    # The register-resident chain runs 512- or 256-thread CTAs only.
    import paper_2312_05647_gb300 as mjp
    from paper_2312_05647_gb300.capi import MJPError
    dims, theta = (37, 53), (10.0, 1.0, 1.5, 0.4)
    times = np.array([0.05, 0.2])
    obs, rho0 = _case(dims, theta, times, 10, seed=5)
    with pytest.raises(MJPError):
        _loglik(dims, theta, np.array([theta]), times, obs, rho0, 2, threads=128)


@pytest.mark.parametrize("dims,theta", [((37, 53), (10.0, 1.0, 1.5, 0.4)), ((200, 200), (20.0, 1.0, 5.0, 0.1))])
def test_register_chain_matches_oracle(dims, theta):
    times = np.array([0.1, 0.5, 1.2])
    obs, rho0 = _case(dims, theta, times, 40, seed=3)
    thetas = synth.jitter(theta, 2, 0.2, synth.rng(2, 8))
    ll = _loglik(dims, theta, thetas, times, obs, rho0, 2)
    nobs = sum(c.sum() for _, c in obs)
    for b in range(len(thetas)):
        ref = oracle.loglik(oracle.build_model(synth.MRNA_PROT2D, list(dims), thetas[b]), rho0, times, obs)
        assert abs(ll[b] - ref) <= PER_OBS_FP32 * nobs


def test_register_chain_groups_of_many_states():
    # Groups of 1, 3 and 5 states: each member accumulates in its owner thread.
    import paper_2312_05647_gb300 as mjp
    dims, theta = (30, 40), [6.0, 1.0, 1.5, 0.3]
    n = 1200
    times = np.array([0.4, 1.5])
    gen = np.random.default_rng(21)
    obs = []
    for _ in times:
        mem, cnt = [], []
        for size in (1, 3, 5, 3, 1):
            mem.append(gen.choice(n // 4, size=size, replace=False))
            cnt.append(float(gen.integers(1, 9)))
        obs.append((mem, np.array(cnt)))
    rho0 = synth.delta(n, 0)
    ll = _loglik(dims, theta, np.array([theta]), times, obs, rho0, 2)
    ref = oracle.loglik(oracle.build_model(synth.MRNA_PROT2D, list(dims), theta), rho0, times, obs)
    nobs = sum(c.sum() for _, c in obs)
    assert abs(ll[0] - ref) <= PER_OBS_FP32 * nobs


def test_register_chain_option_rejects_other_models():
    import paper_2312_05647_gb300 as mjp
    from paper_2312_05647_gb300.capi import MJPError
    m = mjp.Model(synth.MRNA_PROT2D, [20, 20], [5.0, 1.0, 1.0, 0.2], mjp.FP64)
    m.set_option(mjp.OPT_CHAIN, 2)
    o = mjp.Obs(400, [0.5], [([np.array([0])], np.array([1.0]))], synth.delta(400, 0))
    with pytest.raises(MJPError):
        mjp.loglik(m, o, np.array([[5.0, 1.0, 1.0, 0.2]]))


def _spread_obs(dims, times, ngroups, seed):
    # Single-state groups anywhere in the box (rho_0 below is uniform, so
    # every state has mass).
    n = dims[0] * dims[1]
    gen = np.random.default_rng(seed)
    obs = []
    for _ in times:
        mem = [np.array([s]) for s in gen.choice(n, size=ngroups, replace=False)]
        obs.append((mem, gen.integers(1, 6, size=ngroups).astype(float)))
    return obs


def test_register_chain_clusters_of_many_ctas_carry_rows_across_every_seam():
    # A 40 x 1800 box: 4 CTAs per cluster at 512 threads, 8 at 256 threads.
    # With rho_0 uniform every CTA boundary carries
    # nonzero rows at every jump; both layouts give the same chain, and the
    # oracle's log-likelihood within the FP32 tolerance.
    dims, theta = (40, 1800), (6.0, 1.0, 30.0, 0.5)
    n = dims[0] * dims[1]
    times = np.array([0.02, 0.1, 0.3])
    obs = _spread_obs(dims, times, 40, seed=77)
    rho0 = np.full(n, 1.0 / n)
    thetas = synth.jitter(theta, 2, 0.2, synth.rng(2, 78))
    a = _loglik(dims, theta, thetas, times, obs, rho0, 2)
    b = _loglik(dims, theta, thetas, times, obs, rho0, 2, threads=256)
    np.testing.assert_array_equal(a, b)
    nobs = sum(c.sum() for _, c in obs)
    for i in range(len(thetas)):
        ref = oracle.loglik(oracle.build_model(synth.MRNA_PROT2D, list(dims), thetas[i]), rho0, times, obs)
        assert abs(a[i] - ref) <= PER_OBS_FP32 * nobs


def test_register_chain_handover_wait_that_runs_out_is_reported():
    # A wait limit of zero polls: the first wait for a neighbour CTA's row
    # gives up at once; the status word says so (MJP_ERR_DEVICE_TIMEOUT), and
    # the model and the context stay usable.
    import paper_2312_05647_gb300 as mjp
    from paper_2312_05647_gb300.capi import MJPError
    dims, theta = (200, 200), (20.0, 1.0, 5.0, 0.1)  # 2 CTAs per cluster
    times = np.array([0.05, 0.2])
    obs, rho0 = _case(dims, theta, times, 20, seed=91)
    thetas = synth.jitter(theta, 2, 0.2, synth.rng(2, 92))
    m = mjp.Model(synth.MRNA_PROT2D, dims, theta, mjp.FP32)
    m.set_option(mjp.OPT_CHAIN, 2)
    m.set_option(mjp.OPT_WAIT_LIMIT, 0)
    o = mjp.Obs(dims[0] * dims[1], times, obs, rho0)
    with pytest.raises(MJPError) as ei:
        mjp.loglik(m, o, thetas)
    assert ei.value.code == -5
    m.set_option(mjp.OPT_WAIT_LIMIT, 1 << 24)
    ll = mjp.loglik(m, o, thetas)
    m.check()
    np.testing.assert_array_equal(ll, _loglik(dims, theta, thetas, times, obs, rho0, 2))


def _dense_obs(dims, times, rows, cols, seed):
    # Every state of the given rows and columns is a single-member group at
    # every time, so each thread that holds them has one observation per state
    # (up to all 40 register slots) in every window.
    gen = np.random.default_rng(seed)
    states = [p * dims[0] + m for p in rows for m in cols]
    return [([np.array([s]) for s in states], gen.integers(1, 4, size=len(states)).astype(float)) for _ in times]


@pytest.mark.parametrize("dims,rows,cols,times", [
    ((30, 40), range(0, 40), range(0, 30), [0.05, 0.3, 1.0]),   # one CTA, every state observed
    # Two CTAs, the rows on both sides of their seam, mRNA counts below 100
    # (the higher ones fall below FP32's range by t = 0.3: their log is -inf
    # in FP32 as it is not in FP64).
    ((200, 200), range(93, 107), range(0, 100), [0.3]),
])
def test_register_chain_with_every_state_of_a_band_observed(dims, rows, cols, times):
    theta = (20.0, 1.0, 5.0, 0.1)
    n = dims[0] * dims[1]
    times = np.array(times)
    obs = _dense_obs(dims, times, rows, cols, seed=len(rows))
    rho0 = np.full(n, 1.0 / n)
    thetas = synth.jitter(theta, 2, 0.2, synth.rng(2, 93))
    a = _loglik(dims, theta, thetas, times, obs, rho0, 1)
    b = _loglik(dims, theta, thetas, times, obs, rho0, 2)
    np.testing.assert_array_equal(a, b)
    nobs = sum(c.sum() for _, c in obs)
    ref = oracle.loglik(oracle.build_model(synth.MRNA_PROT2D, list(dims), thetas[0]), rho0, times, obs)
    assert abs(b[0] - ref) <= PER_OBS_FP32 * nobs


@pytest.mark.parametrize("dims,threads", [((200, 200), 0), ((40, 1800), 256)])
def test_register_chain_repeats_bit_for_bit(dims, threads):
    # The same launch ten times (2- and 8-CTA clusters; rows handed over
    # between CTAs by st.async, observations summed after the CTA barrier): a
    # race in the hand-over, the edges or the observation sums would change
    # some result between runs.
    # Snapshots from the empty state reach past the first CTA boundary by
    # t = 3 (p ~ 100 on the 200 x 200 box, ~300 on the 40 x 1800 one).
    theta = (20.0, 1.0, 5.0, 0.1)
    times = np.array([0.3, 1.0, 3.0])
    obs, rho0 = _case(dims, theta, times, 30, seed=13)
    thetas = synth.jitter(theta, 4, 0.2, synth.rng(2, 14))
    runs = [_loglik(dims, theta, thetas, times, obs, rho0, 2, threads=threads) for _ in range(10)]
    assert np.all(np.isfinite(runs[0]))
    for r in runs[1:]:
        np.testing.assert_array_equal(runs[0], r)
