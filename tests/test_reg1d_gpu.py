"""The register-resident birth-death chain (expv: batches and single models):
bit-identical to the shared-memory chain kernel (same operation order per
state, same weights) for every cluster size and halo width, and within the
tolerance of the oracle.  Edge cases of the segment layout: one state, fewer
states than one thread's run, instances split so finely that the last CTA owns
fewer states than the halo, instances that need several CTAs to fit at all,
windows without a stored copy of their weights."""
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


def _small_batch(n, seed):
    gen = np.random.default_rng(seed)
    N = np.concatenate([[1, 2, 3], np.floor(np.exp(gen.uniform(np.log(5), np.log(3000), n - 3)))]).astype(np.int64)
    lam = gen.uniform(1.0, np.maximum(N / 4.0, 1.5))
    mu = gen.uniform(0.5, 2.0, n)
    t = np.exp(gen.uniform(np.log(0.01), np.log(0.6), n))
    t[0] = 0.0
    s0 = (gen.random(n) * N * 0.3).astype(np.int64)
    return N, np.stack([lam, mu], 1), t, s0


def _run_batch(N, th, t, s0, prec, chain, cluster=0, halo=0, graph=False):
    import paper_2312_05647_gb300 as mjp
    b = mjp.Batch(N, th, t, s0=s0, precision=prec)
    b.set_option(mjp.OPT_CHAIN, chain)
    if cluster:
        b.set_option(mjp.OPT_CLUSTER, cluster)
    if halo:
        b.set_option(mjp.OPT_HALO, halo)
    out = b.run(b.empty_out(), use_graph=graph)
    b.check()
    return out.cpu().numpy(), b


def _oracle_bd(N, th, t, s0):
    csr = oracle.build_model(oracle.BD1D, [int(N)], th)
    r0 = np.zeros(int(N))
    r0[int(s0)] = 1.0
    out, _ = oracle.expv(csr, r0, [t])
    return out[0]


@pytest.mark.parametrize("prec", [1, 2])
def test_batch_bitwise_over_clusters_and_halos(prec):
    N, th, t, s0 = _small_batch(96, 11)
    ref, _ = _run_batch(N, th, t, s0, prec, chain=1)
    # Forced clusters split instances as far as the last CTA still owns one
    # round of states (down to a few dozen states per CTA); halos below one
    # round are raised to it.
    for cluster, halo in [(0, 0), (2, 1), (3, 7), (8, 32), (5, 100)]:
        got, _ = _run_batch(N, th, t, s0, prec, chain=2, cluster=cluster, halo=halo)
        np.testing.assert_array_equal(got, ref, err_msg=f"cluster {cluster} halo {halo}")
    got, b = _run_batch(N, th, t, s0, prec, chain=2, graph=True)
    np.testing.assert_array_equal(got, ref)
    res = b.split(got.astype(np.float64))
    for j in range(len(N)):
        assert np.abs(res[j] - _oracle_bd(N[j], th[j], t[j], s0[j])).max() <= TOL[prec], j


@pytest.mark.parametrize("prec", [1, 2])
def test_batch_instances_that_need_a_cluster(prec):
    # FP32 CTAs hold 5,040 states, FP64 CTAs 3,360: these need up to 4 and 6 CTAs.
    N = np.array([20000, 12000, 9000, 8193, 4097, 300], dtype=np.int64)
    th = np.stack([N / 5.0, np.full(len(N), 1.0)], 1)
    t = np.array([0.02, 0.03, 0.01, 0.02, 0.05, 0.5])
    s0 = (N * 0.4).astype(np.int64)
    ref, _ = _run_batch(N, th, t, s0, prec, chain=1)
    got, b = _run_batch(N, th, t, s0, prec, chain=2)
    np.testing.assert_array_equal(got, ref)
    res = b.split(got.astype(np.float64))
    for j in range(len(N)):
        assert np.abs(res[j] - _oracle_bd(N[j], th[j], t[j], s0[j])).max() <= TOL[prec], j


@pytest.mark.parametrize("period", [0, 8, 64])
def test_defect_period_bitwise_across_kernels(period):
    # The exit-defect correction is local to a state, so every kernel and
    # cluster shape applies it identically, at any period or switched off.
    import paper_2312_05647_gb300 as mjp
    N, th, t, s0 = _small_batch(48, 17)
    outs = []
    for chain, cluster in ((1, 0), (2, 0), (2, 3)):
        b = mjp.Batch(N, th, t, s0=s0, precision=1)
        b.set_option(mjp.OPT_RENORM_PERIOD, period)
        b.set_option(mjp.OPT_CHAIN, chain)
        if cluster:
            b.set_option(mjp.OPT_CLUSTER, cluster)
        out = b.run(b.empty_out())
        b.check()
        outs.append(out.cpu().numpy())
    np.testing.assert_array_equal(outs[1], outs[0])
    np.testing.assert_array_equal(outs[2], outs[0])


def test_batch_tune_keeps_results():
    N, th, t, s0 = _small_batch(120, 13)
    ref, _ = _run_batch(N, th, t, s0, 1, chain=1)
    import paper_2312_05647_gb300 as mjp
    b = mjp.Batch(N, th, t, s0=s0, precision=1)
    out = b.empty_out()
    cfg = b.tune(out)
    assert '"chain"' in cfg
    got = b.run(out, use_graph=True).cpu().numpy()
    b.check()
    np.testing.assert_array_equal(got, ref)


def _model_expv(N, theta, prec, rho0, times, chain, opts=None):
    import torch
    import paper_2312_05647_gb300 as mjp
    m = mjp.Model(synth.BD1D, [N], theta, prec)
    m.set_option(mjp.OPT_CHAIN, chain)
    for k, v in (opts or {}).items():
        m.set_option(k, v)
    r = torch.tensor(rho0, dtype=m.torch_dtype, device="cuda")
    out, info = m.expv(r, times, info=True)
    m.check()
    return out.cpu().numpy(), info


@pytest.mark.parametrize("prec", [1, 2])
def test_model_expv_bitwise_and_oracle(prec):
    cfg = synth.bd_small()
    times = [5.0, 0.1, 2.0, 0.0, 0.5, 1.0]  # unsorted, with t = 0
    ref, ri = _model_expv(64, cfg["theta"], prec, cfg["rho0"], times, chain=1)
    got, gi = _model_expv(64, cfg["theta"], prec, cfg["rho0"], times, chain=2)
    np.testing.assert_array_equal(got, ref)
    assert list(gi["K"]) == list(ri["K"])
    r, _ = oracle.expv(oracle.build_model(synth.BD1D, [64], cfg["theta"]), cfg["rho0"], times)
    assert np.abs(got - r).max() <= TOL[prec]


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("N", [1, 2, 15, 16, 17, 1000, 9000])
def test_model_expv_sizes(prec, N):
    gen = np.random.default_rng(N)
    rho0 = gen.random(N)
    rho0 /= rho0.sum()
    theta = [N / 3.0 + 1.0, 1.3]
    times = [0.01, 0.05] if N > 100 else [0.3, 1.5]
    got, _ = _model_expv(N, theta, prec, rho0, times, chain=2)
    ref, _ = _model_expv(N, theta, prec, rho0, times, chain=1)
    np.testing.assert_array_equal(got, ref)
    r, _ = oracle.expv(oracle.build_model(synth.BD1D, [N], theta), rho0, times)
    assert np.abs(got - r).max() <= TOL[prec]


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("cap", [1, 300])
def test_model_expv_weight_store_fallback(prec, cap):
    # Windows without a stored copy run Algorithm 2's recurrence in the chain.
    from paper_2312_05647_gb300 import OPT_ARENA
    cfg = synth.bd_small()
    times = [0.1, 1.0, 5.0]
    got, _ = _model_expv(64, cfg["theta"], prec, cfg["rho0"], times, chain=2, opts={OPT_ARENA: cap})
    ref, _ = _model_expv(64, cfg["theta"], prec, cfg["rho0"], times, chain=1, opts={OPT_ARENA: cap})
    np.testing.assert_array_equal(got, ref)
    r, _ = oracle.expv(oracle.build_model(synth.BD1D, [64], cfg["theta"]), cfg["rho0"], times)
    assert np.abs(got - r).max() <= TOL[prec]


def test_register_chain_refusals():
    import paper_2312_05647_gb300 as mjp
    from paper_2312_05647_gb300.capi import MJPError
    cfg = synth.bd_small()
    with pytest.raises(MJPError):
        _model_expv(64, cfg["theta"], 1, cfg["rho0"], [1.0], chain=2, opts={mjp.OPT_THREADS: 128})
    with pytest.raises(MJPError):  # the defect-correction period is a multiple of 8
        _model_expv(64, cfg["theta"], 1, cfg["rho0"], [1.0], chain=2, opts={mjp.OPT_RENORM_PERIOD: 12})
    b = mjp.Batch(np.array([10]), np.array([[1.0, 1.0]]), np.array([0.5]))
    with pytest.raises(MJPError):
        b.set_option(mjp.OPT_HALO, 0)
    with pytest.raises(MJPError):
        b.set_option(mjp.OPT_CHAIN, 3)


def test_shared_memory_attribute_never_lowered():
    # A large shared-memory batch, then a small single model (whose launch
    # configuration query sizes the same kernel's shared memory), then a
    # medium batch: the kernel attribute must still admit the medium launch.
    import paper_2312_05647_gb300 as mjp
    big = np.array([20000], dtype=np.int64)
    _run_batch(big, np.array([[400.0, 1.0]]), np.array([0.01]), np.array([0]), 1, chain=1)
    cfg = synth.bd_small()
    _model_expv(64, cfg["theta"], 1, cfg["rho0"], [0.5], chain=1)
    mid = np.array([6000], dtype=np.int64)
    got, b = _run_batch(mid, np.array([[300.0, 1.0]]), np.array([0.02]), np.array([0]), 1, chain=1)
    assert np.abs(got.astype(np.float64) - _oracle_bd(6000, [300.0, 1.0], 0.02, 0)).max() <= TOL[1]
