"""The autoregulatory gene network (Sec. 3.1.3, Eq. STS_chem; MJP_AUTOREG) on
the GPU against the oracle: transient distributions (1e-12 FP64, 1e-6 FP32,
one CTA and clusters of 2 and 4, ragged boxes) and log-likelihoods of
(n_R, n_P) snapshots with the gene state summed out (groups of two states,
Sec. 3.1.3), per observation within the tolerances of the other models."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
TOL = {2: 1e-12, 1: 1e-6}
PER_OBS = {2: 1e-12, 1: 5e-5}
THETA = [10.0, 0.5, 1.0, 0.1, 0.1, 0.05]  # Sec. 3.1.3: (beta_R, beta_P) = (10, .5), gamma_R 1, gamma_P .1, lambdas .1 / .05


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2312_05647_gb300 import build as lib_build
    lib_build.build()
    torch.cuda.set_device(0)


def _model(dims, theta, prec, opts=None):
    import paper_2312_05647_gb300 as mjp
    m = mjp.Model(mjp.AUTOREG, dims, theta, prec)
    for k, v in (opts or {}).items():
        m.set_option(k, v)
    return m


@pytest.mark.parametrize("prec", [2, 1])
@pytest.mark.parametrize("dims,cluster", [([12, 10], 0), ([23, 17], 0), ([30, 41], 2), ([9, 25], 4)])
def test_autoreg_expv_matches_oracle(prec, dims, cluster):
    import torch
    import paper_2312_05647_gb300 as mjp
    N = 2 * dims[0] * dims[1]
    gen = np.random.default_rng(N + cluster)
    rho0 = gen.random(N)
    rho0 /= rho0.sum()
    times = [2.0, 0.1, 0.0, 5.0]
    m = _model(dims, THETA, prec, {mjp.OPT_CLUSTER: cluster} if cluster else None)
    r = torch.tensor(rho0, dtype=m.torch_dtype, device="cuda")
    out, info = m.expv(r, times, info=True)
    m.check()
    ref, rinfo = oracle.expv(oracle.build_model(oracle.AUTOREG, dims, THETA), rho0, times)
    assert list(info["K"]) == list(rinfo["K"]) and info["omega"] == rinfo["omega"]
    assert np.abs(out.double().cpu().numpy() - ref).max() <= TOL[prec]


@pytest.mark.parametrize("prec", [2, 1])
def test_autoreg_loglik_matches_oracle(prec):
    import paper_2312_05647_gb300 as mjp
    dims = [25, 30]
    NR, NP = dims
    N = 2 * NR * NP
    rho0 = synth.delta(N, 0)
    times = np.linspace(0.5, 10.0, 8)
    # (n_R, n_P) snapshots drawn from the oracle's distribution at each time;
    # the group of an observation holds both gene states.
    csr = oracle.build_model(oracle.AUTOREG, dims, THETA)
    rho_t, _ = oracle.expv(csr, rho0, times)
    gen = np.random.default_rng(17)
    obs = []
    for i in range(len(times)):
        p = np.clip(rho_t[i], 0, None)
        s = gen.choice(N, size=60, p=p / p.sum())
        key = s % (NR * NP)
        vals, counts = np.unique(key, return_counts=True)
        obs.append(([np.array([v, v + NR * NP]) for v in vals], counts.astype(np.float64)))
    nobs = sum(c.sum() for _, c in obs)
    thetas = synth.jitter(THETA, 5, 0.2, synth.rng(5, 11))
    m = _model(dims, THETA, prec)
    o = mjp.Obs(N, times, obs, rho0)
    ll = mjp.loglik(m, o, thetas)
    m.check()
    for b in range(len(thetas)):
        ref = oracle.loglik(oracle.build_model(oracle.AUTOREG, dims, thetas[b]), rho0, times, obs)
        assert abs(ll[b] - ref) <= PER_OBS[prec] * nobs


def test_autoreg_refusals():
    import paper_2312_05647_gb300 as mjp
    from paper_2312_05647_gb300.capi import MJPError
    with pytest.raises(MJPError):
        mjp.Model(mjp.AUTOREG, [10, 1], THETA, 2)       # N_P >= 2
    with pytest.raises(MJPError):
        mjp.Model(mjp.AUTOREG, [10, 10], THETA[:4], 2)  # six rates
