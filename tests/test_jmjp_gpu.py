"""J-MJP state probabilities on the GPU (Method #2, Algorithm 1;
jmjp_state_probs) against the oracle's chain: phi_i = sum over observation
i's group of rho0 B^{k_i}, birth-death and two-state models, FP64 within
1e-12 and FP32 within 1e-6; unsorted and repeated jump counts, k = 0, groups
of both gene states, one observation, a chain of one state, and the refusals."""
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


def _gpu(kind, dims, theta, rho0, ks, groups, prec):
    import torch
    import paper_2312_05647_gb300 as mjp
    m = mjp.Model(kind, dims, theta, prec)
    r = torch.tensor(rho0, dtype=m.torch_dtype, device="cuda")
    phi = m.jmjp_probs(r, ks, groups)
    m.check()
    return phi


@pytest.mark.parametrize("prec", [2, 1])
@pytest.mark.parametrize("kind,dims,theta,kmax,nobs", [
    (synth.BD1D, [64], [10.0, 1.0], 400, 300),
    (synth.BD1D, [1], [3.0, 1.0], 10, 5),
    (synth.BD1D, [1500], [300.0, 1.0], 900, 700),
    (synth.TWOSTATE, [300], [100.0, 1.0, 2.0, 1.0], 2500, 1000),    # the promoter of Sec. 3.1.2
    (synth.TWOSTATE, [37], [20.0, 0.5, 0.3, 1.5], 800, 1),
])
def test_jmjp_matches_oracle(prec, kind, dims, theta, kmax, nobs):
    N = synth.n_states(kind, dims)
    gen = np.random.default_rng(N + nobs)
    rho0 = gen.random(N)
    rho0 /= rho0.sum()
    ks = gen.integers(0, kmax + 1, size=nobs)
    ks[: min(3, nobs)] = [0, kmax, 0][: min(3, nobs)]
    if kind == synth.TWOSTATE:
        NR = dims[0]
        groups = [np.array([r, r + NR]) for r in gen.integers(0, NR, size=nobs)]
    else:
        groups = [gen.choice(N, size=gen.integers(1, min(N, 3) + 1), replace=False) for _ in range(nobs)]
    got = _gpu(kind, dims, theta, rho0, ks, groups, prec)
    ref = oracle.jmjp_probs(oracle.build_model(kind, dims, theta), rho0, ks, groups)
    assert np.abs(got - ref).max() <= TOL[prec]


@pytest.mark.parametrize("prec", [2, 1])
@pytest.mark.parametrize("kind,dims,theta,kmax,nobs", [
    (synth.TWOSTATE, [300], [100.0, 1.0, 2.0, 1.0], 1500, 30000),   # several chunks of observations
    (synth.BD1D, [14000], [3000.0, 1.0], 150, 1200),                # a chain filling shared memory
])
def test_jmjp_chunked_observations(prec, kind, dims, theta, kmax, nobs):
    # More observations than one shared-memory chunk holds: equal jump counts
    # straddle the chunk boundaries.
    N = synth.n_states(kind, dims)
    gen = np.random.default_rng(nobs)
    rho0 = gen.random(N)
    rho0 /= rho0.sum()
    ks = np.sort(gen.integers(0, kmax + 1, size=nobs))[gen.permutation(nobs)]
    groups = [gen.choice(N, size=gen.integers(1, 4), replace=False) for _ in range(nobs)]
    got = _gpu(kind, dims, theta, rho0, ks, groups, prec)
    ref = oracle.jmjp_probs(oracle.build_model(kind, dims, theta), rho0, ks, groups)
    assert np.abs(got - ref).max() <= TOL[prec]


def test_jmjp_promoter_snapshots():
    # Jump counts drawn as in Sec. 2.2.2: k_i ~ Poisson(Omega T_i) at the
    # promoter's collection times, one observed n_R per cell (both gene states).
    cfg = synth.twostate_promoter(300)
    NR = cfg["dims"][0]
    csr = oracle.build_model(cfg["kind"], cfg["dims"], cfg["theta"])
    omega = 1.1 * oracle.max_exit(csr)
    gen = np.random.default_rng(5)
    T = np.repeat(cfg["times"][::5], 20)
    ks = gen.poisson(omega * T)
    groups = [np.array([r, r + NR]) for r in gen.integers(0, 150, size=len(ks))]
    got = _gpu(cfg["kind"], cfg["dims"], cfg["theta"], cfg["rho0"], ks, groups, 2)
    ref = oracle.jmjp_probs(csr, cfg["rho0"], ks, groups)
    assert np.abs(got - ref).max() <= 1e-12
    # The same groups passed flat as (group_ptr, members).
    flat = (np.arange(0, 2 * len(ks) + 1, 2), np.concatenate(groups))
    np.testing.assert_array_equal(_gpu(cfg["kind"], cfg["dims"], cfg["theta"], cfg["rho0"], ks, flat, 2), got)


def test_jmjp_refusals():
    import torch
    import paper_2312_05647_gb300 as mjp
    from paper_2312_05647_gb300.capi import MJPError
    m = mjp.Model(synth.BD1D, [10], [2.0, 1.0], mjp.FP64)
    r = torch.tensor(synth.delta(10, 0), device="cuda")
    with pytest.raises(MJPError):
        m.jmjp_probs(r, [-1], [np.array([0])])         # negative jump count
    with pytest.raises(MJPError):
        m.jmjp_probs(r, [3], [np.array([10])])         # member out of range
    with pytest.raises(MJPError):
        m.jmjp_probs(r, [3, 4], [np.array([1]), np.array([], dtype=np.int32)])  # empty group
    big = mjp.Model(synth.BD1D, [40000], [2.0, 1.0], mjp.FP64)
    with pytest.raises(MJPError):
        big.jmjp_probs(torch.tensor(synth.delta(40000, 0), device="cuda"), [3], [np.array([0])])
    with pytest.raises(MJPError):
        m.jmjp_probs(r, [2 ** 31], [np.array([0])])    # jump counts below 2^31 - 1
    two_d = mjp.Model(synth.MRNA_PROT2D, [10, 10], [5.0, 1.0, 1.0, 0.2], mjp.FP64)
    with pytest.raises(MJPError):
        two_d.jmjp_probs(torch.tensor(synth.delta(100, 0), device="cuda"), [3], [np.array([0])])
