"""The register-resident two-state chain (FP32 promoter log-likelihood, one
CTA per theta): within the FP32 tolerance of the oracle; the same
log-likelihoods for every warp count (the chain and the per-group sums do not
depend on the layout); close to the shared-memory kernel, which runs the same
compensated chain but sums the observations jump by jump; groups of one and two
arbitrary members; windows without a stored copy of their weights."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

LL_PER_OBS = 5e-6      # against the FP64 oracle, per observation (the compensated chain)
# Against the shared-memory kernel: the same chain; the observation sums are
# taken 8 terms at a time with FMA and then Kahan-added, instead of one Kahan
# step per jump, so a group's sum differs by at most ~10 u relative.
LL_VS_SMEM_PER_OBS = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_05647_gb300 import build as lib_build
    lib_build.build()
    torch.cuda.set_device(0)


def _promoter(N_R, times, cells, seed):
    cfg = synth.twostate_promoter(N_R=N_R)
    snaps = synth.gillespie_snapshots(cfg["kind"], cfg["dims"], cfg["theta"], times, cells, synth.rng(9, seed))
    obs = synth.snapshot_obs(cfg["kind"], cfg["dims"], snaps)
    return cfg, obs


def _ll(N_R, thetas, times, obs, rho0, chain=0, threads=0, opts=None):
    import paper_2312_05647_gb300 as mjp
    m = mjp.Model(synth.TWOSTATE, [N_R], thetas[0], mjp.FP32)
    m.set_option(mjp.OPT_CHAIN, chain)
    if threads:
        m.set_option(mjp.OPT_THREADS, threads)
    for k, v in (opts or {}).items():
        m.set_option(k, v)
    o = mjp.Obs(2 * N_R, times, obs, rho0)
    ll = mjp.loglik(m, o, thetas)
    m.check()
    return ll


def _nobs(obs):
    return sum(float(c.sum()) for _, c in obs)


@pytest.mark.parametrize("N_R", [60, 150, 300])
def test_two_state_register_chain_matches_oracle(N_R):
    # N_R = 60: one warp; 150 and 300: two warps (six columns per thread).
    times = np.linspace(0.5, 10.0, 12)
    cfg, obs = _promoter(N_R, times, 60, seed=N_R)
    thetas = synth.jitter(cfg["theta"], 3, 0.2, synth.rng(9, N_R + 1))
    ll = _ll(N_R, thetas, times, obs, cfg["rho0"], chain=2)
    ref = [oracle.loglik(oracle.build_model(synth.TWOSTATE, [N_R], th), cfg["rho0"], times, obs) for th in thetas]
    diffs = np.abs(ll - np.array(ref))
    print(f"N_R {N_R}: |GPU - oracle| per theta", diffs, "over", _nobs(obs), "observations")
    assert np.all(np.isfinite(ll))
    assert diffs.max() <= LL_PER_OBS * _nobs(obs)


def test_two_state_register_chain_is_the_default_and_close_to_shared_memory_kernel():
    cfg = synth.twostate_promoter()
    times = cfg["times"]
    cfg, obs = _promoter(300, times, 100, seed=3)
    thetas = synth.jitter(cfg["theta"], 8, 0.2, synth.rng(9, 4))
    a = _ll(300, thetas, times, obs, cfg["rho0"], chain=0)
    b = _ll(300, thetas, times, obs, cfg["rho0"], chain=2)
    c = _ll(300, thetas, times, obs, cfg["rho0"], chain=1)
    np.testing.assert_array_equal(a, b)
    assert np.abs(b - c).max() <= LL_VS_SMEM_PER_OBS * _nobs(obs)


@pytest.mark.parametrize("threads", [64, 128, 256])
def test_two_state_register_chain_same_result_for_every_warp_count(threads):
    # 2, 4 or 8 warps hold the same chain (bit-identical values); only the
    # final FP64 sum over the groups is taken in a thread-count dependent order.
    times = np.linspace(0.5, 6.0, 10)
    cfg, obs = _promoter(180, times, 40, seed=11)
    thetas = synth.jitter(cfg["theta"], 4, 0.2, synth.rng(9, 12))
    ref = _ll(180, thetas, times, obs, cfg["rho0"], chain=2)  # automatic: one warp (180 <= 192)
    got = _ll(180, thetas, times, obs, cfg["rho0"], chain=2, threads=threads)
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=0)


def test_two_state_register_chain_groups_of_one_and_two_arbitrary_states():
    # Single states (either gene state) and pairs that are not (n, n + N_R),
    # drawn from n_R in [4, 24], where the distribution has its mass at these
    # times (far-tail states would hold FP32 subnormals: no relative accuracy).
    N_R, theta = 90, [40.0, 1.0, 2.0, 1.0]
    n = 2 * N_R
    times = np.array([0.3, 1.0, 2.5, 4.0])
    gen = np.random.default_rng(31)
    bulk = np.concatenate([np.arange(4, 25), N_R + np.arange(4, 25)])
    obs = []
    for _ in times:
        mem, cnt = [], []
        for size in (1, 2, 1, 2, 2, 1):
            mem.append(gen.choice(bulk, size=size, replace=False))
            cnt.append(float(gen.integers(1, 9)))
        obs.append((mem, np.array(cnt)))
    rho0 = synth.delta(n, 0)
    thetas = np.array([theta, [35.0, 1.2, 1.5, 0.8]])
    ll = _ll(N_R, thetas, times, obs, rho0, chain=2)
    ref = [oracle.loglik(oracle.build_model(synth.TWOSTATE, [N_R], th), rho0, times, obs) for th in thetas]
    assert np.abs(ll - np.array(ref)).max() <= LL_PER_OBS * _nobs(obs)


@pytest.mark.parametrize("cap", [1, 3000])
def test_two_state_register_chain_weight_store_fallback(cap):
    # Windows that do not fit the planner's weight store run Algorithm 2's
    # recurrence in the kernel (from P_L instead of outward from the mode:
    # the weights agree to FP64 rounding, so the log-likelihoods to ~1e-7).
    import paper_2312_05647_gb300 as mjp
    times = np.linspace(0.5, 8.0, 9)
    cfg, obs = _promoter(150, times, 50, seed=21)
    thetas = synth.jitter(cfg["theta"], 3, 0.2, synth.rng(9, 22))
    a = _ll(150, thetas, times, obs, cfg["rho0"], chain=2)
    b = _ll(150, thetas, times, obs, cfg["rho0"], chain=2, opts={mjp.OPT_ARENA: cap})
    assert np.abs(a - b).max() <= 1e-7 * _nobs(obs)


def test_two_state_register_chain_edge_cases():
    # K = 0 windows (t = 0), a time whose window starts at jump 0, one theta
    # with every rate zero but one, and a zero-probability observation (-inf).
    N_R = 40
    n = 2 * N_R
    times = np.array([0.0, 0.05, 1.0])
    rho0 = synth.delta(n, 0)
    obs = [([np.array([0, N_R])], np.array([3.0])),
           ([np.array([0, N_R]), np.array([1, 1 + N_R])], np.array([2.0, 1.0])),
           ([np.array([2, 2 + N_R]), np.array([5, 5 + N_R])], np.array([1.0, 2.0]))]
    thetas = np.array([[10.0, 1.0, 2.0, 1.0], [0.0, 1.0, 0.0, 0.0]])
    ll = _ll(N_R, thetas, times, obs, rho0, chain=2)
    ref0 = oracle.loglik(oracle.build_model(synth.TWOSTATE, [N_R], thetas[0]), rho0, times, obs)
    assert abs(ll[0] - ref0) <= LL_PER_OBS * _nobs(obs)
    assert ll[1] == -np.inf  # no births: n_R > 0 has probability zero


def test_two_state_register_chain_handover_wait_that_runs_out_is_reported():
    # A wait limit of zero polls: the first hand-over that is not ready at
    # once gives up; both warp groups stop, the status word says so, and the
    # model (and the context) stay usable.
    import paper_2312_05647_gb300 as mjp
    from paper_2312_05647_gb300.capi import MJPError
    times = np.linspace(0.5, 8.0, 6)
    cfg, obs = _promoter(120, times, 30, seed=41)
    thetas = synth.jitter(cfg["theta"], 4, 0.2, synth.rng(9, 42))
    m = mjp.Model(synth.TWOSTATE, [120], thetas[0], mjp.FP32)
    m.set_option(mjp.OPT_CHAIN, 2)
    m.set_option(mjp.OPT_WAIT_LIMIT, 0)
    o = mjp.Obs(240, times, obs, cfg["rho0"])
    with pytest.raises(MJPError) as ei:
        mjp.loglik(m, o, thetas)  # host call: synchronises and checks the status word
    assert ei.value.code == -5  # MJP_ERR_DEVICE_TIMEOUT
    m.set_option(mjp.OPT_WAIT_LIMIT, 1 << 24)
    ll = mjp.loglik(m, o, thetas)
    m.check()
    ref = _ll(120, thetas, times, obs, cfg["rho0"], chain=2)
    np.testing.assert_array_equal(ll, ref)
