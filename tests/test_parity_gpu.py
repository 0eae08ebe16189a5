"""GPU path (through the C ABI) against the CPU oracle, element by element.

Tolerances: max |GPU - oracle| <= 1e-12 for the FP64 chain and
<= 1e-6 for the FP32 chain, on transient distributions, same truncation mode.
Integer results of the planner (K_i) are compared exactly."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {2: 1e-12, 1: 1e-6}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2312_05647_gb300 import build as lib_build
    lib_build.build()
    torch.cuda.set_device(0)


def _mjp():
    import paper_2312_05647_gb300 as mjp
    return mjp


def gpu_expv(kind, dims, theta, prec, rho0, times, trunc=0, tol=0.0, opts=None):
    import torch
    mjp = _mjp()
    m = mjp.Model(kind, dims, theta, prec)
    for k, v in (opts or {}).items():
        m.set_option(k, v)
    r = torch.tensor(rho0, dtype=m.torch_dtype, device="cuda")
    out, info = m.expv(r, times, trunc=trunc, tol=tol, info=True)
    m.check()
    return out.double().cpu().numpy(), info


def ora_expv(kind, dims, theta, rho0, times, mode=0, tol=0.0):
    csr = oracle.build_model(kind, dims, theta)
    return oracle.expv(csr, rho0, times, mode=mode, tol=tol)


@pytest.mark.parametrize("prec", [2, 1])
def test_immigration_death_small(prec):
    cfg = synth.bd_small()
    g, gi = gpu_expv(cfg["kind"], cfg["dims"], cfg["theta"], prec, cfg["rho0"], cfg["times"])
    r, ri = ora_expv(cfg["kind"], cfg["dims"], cfg["theta"], cfg["rho0"], cfg["times"])
    assert list(gi["K"]) == list(ri["K"])
    assert gi["omega"] == ri["omega"]
    np.testing.assert_allclose(gi["eps"], ri["eps"], rtol=1e-8, atol=1e-16)
    assert np.abs(g - r).max() <= TOL[prec]


@pytest.mark.parametrize("prec", [2, 1])
def test_two_state_promoter(prec):
    cfg = synth.twostate_promoter()
    times = cfg["times"][[0, 7, 19, 33, 49]]
    g, gi = gpu_expv(cfg["kind"], cfg["dims"], cfg["theta"], prec, cfg["rho0"], times)
    r, ri = ora_expv(cfg["kind"], cfg["dims"], cfg["theta"], cfg["rho0"], times)
    assert list(gi["K"]) == list(ri["K"])
    assert np.abs(g - r).max() <= TOL[prec]


@pytest.mark.parametrize("cluster,threads", [(1, 96), (2, 128), (4, 288), (8, 96)])
@pytest.mark.parametrize("prec", [2, 1])
def test_mrna_protein_clusters_ragged(cluster, threads, prec):
    # 37 x 23 = 851 states: slabs of ragged size, halos across CTAs.
    dims, theta = [37, 23], [6.0, 1.0, 1.3, 0.4]
    rho0 = np.zeros(37 * 23)
    rho0[0], rho0[37 * 5 + 3], rho0[-1] = 0.5, 0.3, 0.2
    times = [0.07, 0.9, 2.5, 6.0]
    from paper_2312_05647_gb300 import OPT_CLUSTER, OPT_THREADS
    g, gi = gpu_expv(synth.MRNA_PROT2D, dims, theta, prec, rho0, times,
                     opts={OPT_CLUSTER: cluster, OPT_THREADS: threads})
    r, ri = ora_expv(synth.MRNA_PROT2D, dims, theta, rho0, times)
    assert list(gi["K"]) == list(ri["K"])
    assert np.abs(g - r).max() <= TOL[prec]


@pytest.mark.parametrize("prec", [2, 1])
def test_tolerance_mode(prec):
    cfg = synth.bd_small()
    g, gi = gpu_expv(cfg["kind"], cfg["dims"], cfg["theta"], prec, cfg["rho0"], cfg["times"], trunc=1, tol=1e-14)
    r, ri = ora_expv(cfg["kind"], cfg["dims"], cfg["theta"], cfg["rho0"], cfg["times"], mode=1, tol=1e-14)
    assert np.all(np.abs(np.array(gi["K"]) - np.array(ri["K"])) <= 1)
    assert np.abs(g - r).max() <= TOL[prec]


def test_degenerate_times_and_rates():
    cfg = synth.bd_small()
    times = [2.0, 0.0, 0.5, 2.0, 0.0]  # unsorted, duplicates, t = 0
    g, _ = gpu_expv(cfg["kind"], cfg["dims"], cfg["theta"], 2, cfg["rho0"], times)
    r, _ = ora_expv(cfg["kind"], cfg["dims"], cfg["theta"], cfg["rho0"], times)
    assert np.abs(g - r).max() <= 1e-12
    np.testing.assert_array_equal(g[1], cfg["rho0"])
    np.testing.assert_array_equal(g[4], cfg["rho0"])
    rho0 = np.full(64, 1.0 / 64)
    g, gi = gpu_expv(synth.BD1D, [64], [0.0, 0.0], 2, rho0, [1.0, 3.0])
    assert gi["omega"] == 0.0
    np.testing.assert_array_equal(g[0], rho0)
    np.testing.assert_array_equal(g[1], rho0)


def test_single_state():
    g, gi = gpu_expv(synth.BD1D, [1], [3.0, 1.0], 2, np.array([1.0]), [0.5, 2.0])
    np.testing.assert_array_equal(g, [[1.0], [1.0]])


def test_mrna_protein_full_box_fp32():
    # The full 200 x 200 box at four times; conservation and positivity at all 20.
    cfg = synth.mrna_protein()
    times = cfg["times"][[0, 5, 9, 11]]
    g, gi = gpu_expv(cfg["kind"], cfg["dims"], cfg["theta"], 1, cfg["rho0"], times)
    r, ri = ora_expv(cfg["kind"], cfg["dims"], cfg["theta"], cfg["rho0"], times)
    assert list(gi["K"]) == list(ri["K"])
    assert np.abs(g - r).max() <= 1e-6


def test_mrna_protein_all_times_properties():
    cfg = synth.mrna_protein()
    g, gi = gpu_expv(cfg["kind"], cfg["dims"], cfg["theta"], 1, cfg["rho0"], cfg["times"])
    assert gi["K"].max() == 69089
    assert g.min() >= 0.0
    assert np.abs(g.sum(axis=1) - 1.0).max() <= 1e-5


def test_repeatable_bitwise():
    cfg = synth.twostate_promoter(N_R=100)
    a, _ = gpu_expv(cfg["kind"], cfg["dims"], cfg["theta"], 1, cfg["rho0"], [0.5, 3.0])
    b, _ = gpu_expv(cfg["kind"], cfg["dims"], cfg["theta"], 1, cfg["rho0"], [0.5, 3.0])
    np.testing.assert_array_equal(a, b)


# --------------------------------------------------------------------------
# Log-likelihood
# --------------------------------------------------------------------------

def _promoter_data(N_R, ntimes, cells, seed):
    cfg = synth.twostate_promoter(N_R=N_R)
    times = np.linspace(0.5, 10.0, ntimes)
    snaps = synth.gillespie_snapshots(cfg["kind"], cfg["dims"], cfg["theta"], times, cells, synth.rng(5, seed))
    obs = synth.snapshot_obs(cfg["kind"], cfg["dims"], snaps)
    return cfg, times, obs


# Log-likelihood tolerances, derived from the chain arithmetic: every jump
# rounds each state's value with relative error ~6u (five products and the
# diagonal), so after K jumps an observed group probability carries a relative
# error ~ 6u sqrt(K) (random walk).  Per observation that is 6 * 1.1e-16 *
# sqrt(5000) ~ 5e-14 in FP64 and 6 * 6e-8 * sqrt(5000) ~ 2.5e-5 in FP32;
# the tests allow 1e-12 and 5e-5 per observation (sum of counts).
PER_OBS = {2: 1e-12, 1: 5e-5}


@pytest.mark.parametrize("prec", [2, 1])
def test_loglik_two_state_batch(prec):
    mjp = _mjp()
    cfg, times, obs = _promoter_data(300, 12, 40, seed=3)
    nobs = sum(c.sum() for _, c in obs)
    thetas = synth.jitter(cfg["theta"], 6, 0.2, synth.rng(5, 9))
    m = mjp.Model(cfg["kind"], cfg["dims"], cfg["theta"], prec)
    o = mjp.Obs(600, times, obs, cfg["rho0"])
    ll = mjp.loglik(m, o, thetas)
    for b in range(len(thetas)):
        ref = oracle.loglik(oracle.build_model(cfg["kind"], cfg["dims"], thetas[b]), cfg["rho0"], times, obs)
        assert abs(ll[b] - ref) <= PER_OBS[prec] * nobs


def test_loglik_device_pointers_match_host():
    import torch
    mjp = _mjp()
    cfg, times, obs = _promoter_data(120, 8, 25, seed=4)
    thetas = synth.jitter(cfg["theta"], 5, 0.2, synth.rng(5, 10))
    m = mjp.Model(cfg["kind"], cfg["dims"], cfg["theta"], 1)
    o = mjp.Obs(240, times, obs, cfg["rho0"])
    host = mjp.loglik(m, o, thetas)
    dev = mjp.loglik(m, o, torch.tensor(thetas, dtype=torch.float64, device="cuda"))
    m.check()
    np.testing.assert_array_equal(host, dev.cpu().numpy())


def test_loglik_zero_probability_is_minus_inf():
    mjp = _mjp()
    # BD with no births: any observation above 0 has probability 0.
    times = np.array([1.0])
    obs = [([np.array([0]), np.array([3])], np.array([5.0, 1.0]))]
    m = mjp.Model(synth.BD1D, [10], [0.0, 1.0], 2)
    o = mjp.Obs(10, times, obs, synth.delta(10, 0))
    ll = mjp.loglik(m, o, np.array([[0.0, 1.0]]))
    assert ll[0] == -np.inf


def test_loglik_mrna_protein_cluster():
    mjp = _mjp()
    dims, theta = [40, 60], [8.0, 1.0, 2.0, 0.2]
    times = np.array([0.3, 1.0, 2.5])
    snaps = synth.gillespie_snapshots(synth.MRNA_PROT2D, dims, theta, times, 30, synth.rng(2, 7))
    obs = synth.snapshot_obs(synth.MRNA_PROT2D, dims, snaps)
    rho0 = synth.delta(2400, 0)
    m = mjp.Model(synth.MRNA_PROT2D, dims, theta, 2)
    m.set_option(mjp.OPT_CLUSTER, 4)
    o = mjp.Obs(2400, times, obs, rho0)
    thetas = synth.jitter(theta, 3, 0.1, synth.rng(2, 8))
    ll = mjp.loglik(m, o, thetas)
    for b in range(3):
        ref = oracle.loglik(oracle.build_model(synth.MRNA_PROT2D, dims, thetas[b]), rho0, times, obs)
        assert abs(ll[b] - ref) <= PER_OBS[2] * sum(c.sum() for _, c in obs)


@pytest.mark.parametrize("prec", [2, 1])
def test_more_threads_than_states(prec):
    # Every state has exactly one owning thread, however wide the CTA.
    from paper_2312_05647_gb300 import OPT_THREADS
    for N, threads in [(2, 256), (10, 512), (40, 1024)]:
        rho0 = synth.delta(N, 0)
        times = [0.2, 1.0]
        r, _ = ora_expv(synth.BD1D, [N], [3.0, 1.0], rho0, times)
        for _ in range(3):
            g, _ = gpu_expv(synth.BD1D, [N], [3.0, 1.0], prec, rho0, times, opts={OPT_THREADS: threads})
            assert np.abs(g - r).max() <= TOL[prec]


@pytest.mark.parametrize("prec", [2, 1])
@pytest.mark.parametrize("cap", [1, 3000])
def test_weight_store_fallback(prec, cap):
    # A full weight store (cap 1) or a partly full one (3000 elements: the
    # short early windows fit, the long late ones do not) sends windows to
    # the in-kernel recurrence; results stay within tolerance.
    from paper_2312_05647_gb300 import OPT_ARENA
    cfg = synth.twostate_promoter(N_R=150)
    times = [0.3, 1.0, 4.0, 9.0]
    g, gi = gpu_expv(cfg["kind"], cfg["dims"], cfg["theta"], prec, cfg["rho0"], times, opts={OPT_ARENA: cap})
    r, ri = ora_expv(cfg["kind"], cfg["dims"], cfg["theta"], cfg["rho0"], times)
    assert list(gi["K"]) == list(ri["K"])
    assert np.abs(g - r).max() <= TOL[prec]


@pytest.mark.parametrize("prec", [2, 1])
def test_loglik_groups_of_many_states(prec):
    # Groups of 1, 3 and 5 states (the generic member list) across a cluster.
    mjp = _mjp()
    dims, theta = [30, 40], [6.0, 1.0, 1.5, 0.3]
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
    m = mjp.Model(synth.MRNA_PROT2D, dims, theta, prec)
    m.set_option(mjp.OPT_CLUSTER, 2)
    o = mjp.Obs(n, times, obs, rho0)
    ll = mjp.loglik(m, o, np.array([theta]))
    ref = oracle.loglik(oracle.build_model(synth.MRNA_PROT2D, dims, theta), rho0, times, obs)
    nobs = sum(c.sum() for _, c in obs)
    assert abs(ll[0] - ref) <= PER_OBS[prec] * nobs
