"""General-CSR path (SELL-32 over in-degree-sorted states) against the oracle.

Tolerances as for the stencil chains: 1e-12 (FP64), 1e-6 (FP32) max abs on
transient distributions; K_i compared exactly."""
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


def gpu_csr(rp, col, val, prec, rho0, times, trunc=0, tol=0.0):
    import torch
    import paper_2312_05647_gb300 as mjp
    m = mjp.Model.from_csr(len(rp) - 1, rp, col, val, prec)
    r = torch.tensor(rho0, dtype=m.torch_dtype, device="cuda")
    out, info = m.expv(r, times, trunc=trunc, tol=tol, info=True)
    m.check()
    return out.double().cpu().numpy(), info


@pytest.mark.parametrize("prec", [2, 1])
@pytest.mark.parametrize("n,deg,seed", [(37, 3, 0), (500, 5, 1), (4099, 8, 2)])
def test_random_csr(prec, n, deg, seed):
    gen = np.random.default_rng(seed)
    rp, col, val = synth.random_csr(n, deg, gen, max_exit=50.0)
    rho0 = gen.random(n)
    rho0 /= rho0.sum()
    times = [0.0, 0.05, 0.7, 3.0]
    g, gi = gpu_csr(rp, col, val, prec, rho0, times)
    r, ri = oracle.expv(oracle.CSR(rp, col, val), rho0, times)
    assert gi["omega"] == ri["omega"]
    assert list(gi["K"]) == list(ri["K"])
    assert np.abs(g - r).max() <= TOL[prec]


@pytest.mark.parametrize("prec", [2, 1])
def test_star_graph_and_unsorted_rows(prec):
    # State 0 receives from everybody (in-degree n-1); rows given unsorted.
    n = 300
    rows = []
    for i in range(n):
        tg = [0] if i else list(range(n - 1, 0, -1))
        rows.append(tg)
    rp = np.cumsum([0] + [len(r) for r in rows])
    col = np.concatenate(rows).astype(np.int32)
    gen = np.random.default_rng(5)
    val = gen.lognormal(0.0, 1.0, len(col))
    rho0 = np.full(n, 1.0 / n)
    g, gi = gpu_csr(rp, col, val, prec, rho0, [0.3, 2.0])
    r, ri = oracle.expv(oracle.CSR(rp, col, val), rho0, [0.3, 2.0])
    assert list(gi["K"]) == list(ri["K"])
    assert np.abs(g - r).max() <= TOL[prec]


@pytest.mark.parametrize("prec", [2, 1])
def test_stencil_model_as_csr(prec):
    cfg = synth.twostate_promoter(N_R=150)
    csr = oracle.build_model(cfg["kind"], cfg["dims"], cfg["theta"])
    times = [0.5, 2.0, 6.0]
    g, gi = gpu_csr(csr.row_ptr, csr.col, csr.val, prec, cfg["rho0"], times)
    r, ri = oracle.expv(csr, cfg["rho0"], times)
    assert list(gi["K"]) == list(ri["K"])
    assert np.abs(g - r).max() <= TOL[prec]


def test_zero_rates_csr():
    rp = np.array([0, 1, 2, 2])
    g, gi = gpu_csr(rp, [1, 0], [0.0, 0.0], 2, np.array([0.2, 0.3, 0.5]), [1.0, 4.0])
    assert gi["omega"] == 0.0
    np.testing.assert_array_equal(g, [[0.2, 0.3, 0.5], [0.2, 0.3, 0.5]])


@pytest.mark.parametrize("prec", [1, 2])
def test_large_random_csr_full_size(prec):
    # N = 2^20 states, 8 targets per row, max exit rate 200, t = 1 (K = 309).
    cfg = synth.csr_large()
    g, gi = gpu_csr(cfg["row_ptr"], cfg["col"], cfg["val"], prec, cfg["rho0"], cfg["times"])
    r, ri = oracle.expv(oracle.CSR(cfg["row_ptr"], cfg["col"], cfg["val"]), cfg["rho0"], cfg["times"])
    assert ri["K"][0] == 309 and list(gi["K"]) == [309]
    assert np.abs(g - r).max() <= TOL[prec]
    assert abs(g.sum() - 1.0) <= (1e-12 if prec == 2 else 1e-5)


def test_csr_loglik():
    import paper_2312_05647_gb300 as mjp
    cfg = synth.twostate_promoter(N_R=80)
    theta = [30.0, 1.0, 2.0, 1.0]
    times = np.linspace(0.5, 4.0, 5)
    snaps = synth.gillespie_snapshots(cfg["kind"], cfg["dims"], theta, times, 30, synth.rng(5, 77))
    obs = synth.snapshot_obs(cfg["kind"], cfg["dims"], snaps)
    csr = oracle.build_model(cfg["kind"], cfg["dims"], theta)
    m = mjp.Model.from_csr(csr.n, csr.row_ptr, csr.col, csr.val, 2)
    o = mjp.Obs(csr.n, times, obs, cfg["rho0"])
    ll = mjp.loglik(m, o, np.zeros((1, 0)))
    ref = oracle.loglik(csr, cfg["rho0"], times, obs)
    assert abs(ll[0] - ref) <= 1e-12 * 150


def _csr_run(rp, col, val, prec, rho0, times, opts):
    import torch
    import paper_2312_05647_gb300 as mjp
    m = mjp.Model.from_csr(len(rp) - 1, rp, col, val, prec)
    for k, v in opts.items():
        m.set_option(k, v)
    r = torch.tensor(rho0, dtype=m.torch_dtype, device="cuda")
    out = m.expv(r, times)
    return m, out


@pytest.mark.parametrize("prec", [2, 1])
def test_one_launch_chain_equals_per_jump_launches(prec):
    # The cooperative one-launch chain and one launch per jump run the same
    # per-jump code: identical results (several CTAs, many grid barriers).
    import paper_2312_05647_gb300 as mjp
    gen = np.random.default_rng(8)
    n = 70000
    rp, col, val = synth.random_csr(n, 6, gen, max_exit=80.0)
    rho0 = gen.random(n)
    rho0 /= rho0.sum()
    times = [0.1, 0.8, 2.0]
    m1, a = _csr_run(rp, col, val, prec, rho0, times, {mjp.OPT_CHAIN: 2})
    m1.check()
    m2, b = _csr_run(rp, col, val, prec, rho0, times, {})
    m2.check()
    np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())


def test_grid_barrier_wait_that_runs_out_is_reported():
    # A wait limit of zero polls: every CTA but the last to arrive gives up at
    # the first barrier; the chain stops, the status word says so, and the
    # model (and the context) stay usable.
    import paper_2312_05647_gb300 as mjp
    from paper_2312_05647_gb300.capi import MJPError
    gen = np.random.default_rng(9)
    n = 1 << 15
    rp, col, val = synth.random_csr(n, 4, gen, max_exit=40.0)
    rho0 = np.full(n, 1.0 / n)
    m, _ = _csr_run(rp, col, val, 2, rho0, [1.0], {mjp.OPT_CHAIN: 2, mjp.OPT_WAIT_LIMIT: 0})
    with pytest.raises(MJPError) as ei:
        m.check()
    assert ei.value.code == -5  # MJP_ERR_DEVICE_TIMEOUT
    m.set_option(mjp.OPT_WAIT_LIMIT, 1 << 24)
    import torch
    out = m.expv(torch.tensor(rho0, dtype=torch.float64, device="cuda"), [1.0])
    m.check()
    r, _ = oracle.expv(oracle.CSR(rp, col, val), rho0, [1.0])
    assert np.abs(out.cpu().numpy() - r).max() <= 1e-12
