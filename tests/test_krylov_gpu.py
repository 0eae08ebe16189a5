"""Krylov subspace steps on the GPU (Method #5, Sec. 2.3; MJP_OPT_METHOD = 2)
against the oracle's Krylov steps: the same step rule (ceil(interval x
max_n |a_nn| / (2 kappa)) equal steps between ascending times), the same
Arnoldi process (modified Gram-Schmidt, full projection) and Pade-13 exponential
of the small projection, within 1e-12 (the inner products are summed in a
different order); subspace sizes 1, 5, 20, 32 and spaces smaller than kappa."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2312_05647_gb300 import build as lib_build
    lib_build.build()
    torch.cuda.set_device(0)


def _krylov_gpu(N, theta, rho0, times, kappa=20, prec=2, kind=synth.BD1D):
    import torch
    import paper_2312_05647_gb300 as mjp
    m = mjp.Model(kind, [N], theta, prec)
    m.set_option(mjp.OPT_METHOD, mjp.METHOD_KRYLOV)
    m.set_option(mjp.OPT_KAPPA, kappa)
    r = torch.tensor(rho0, dtype=m.torch_dtype, device="cuda")
    out, info = m.expv(r, times, info=True)
    m.check()
    return out.cpu().numpy(), info


@pytest.mark.parametrize("N,theta,times,kappa", [
    (64, [10.0, 1.0], [0.1, 0.5, 1.0, 2.0, 5.0], 20),      # immigration-death
    (1, [3.0, 1.0], [0.5], 20),
    (2, [2.0, 3.0], [0.9, 0.0, 3.3], 20),                  # invariant space after 2 vectors
    (12, [3.0, 1.0], [2.0, 0.7], 20),
    (300, [60.0, 1.0], [0.3], 5),
    (700, [150.0, 1.0], [0.05, 0.01], 32),
    (513, [100.0, 0.8], [0.02], 1),
    (4096, [1000.0, 1.0], [0.003], 20),
])
def test_krylov_matches_oracle(N, theta, times, kappa):
    gen = np.random.default_rng(N + kappa)
    rho0 = gen.random(N)
    rho0 /= rho0.sum()
    got, info = _krylov_gpu(N, theta, rho0, times, kappa)
    ref, rinfo = oracle.krylov(oracle.build_model(oracle.BD1D, [N], theta), rho0, times, kappa=kappa)
    assert info["omega"] == rinfo["max_exit"]
    assert list(info["K"]) == list(rinfo["steps"])
    assert np.abs(got - ref).max() <= 1e-12


@pytest.mark.parametrize("NR,theta,times,kappa", [
    (300, [100.0, 1.0, 2.0, 1.0], [0.5, 0.05], 20),          # the promoter of Sec. 3.1.2
    (2, [3.0, 0.5, 1.5, 2.0], [1.0, 0.3], 20),               # 4 states: the space is whole
    (37, [20.0, 0.5, 0.3, 1.5], [0.7], 8),
    (2048, [900.0, 1.0, 2.0, 1.0], [0.002], 20),
])
def test_krylov_two_state_matches_oracle(NR, theta, times, kappa):
    gen = np.random.default_rng(NR + kappa)
    rho0 = gen.random(2 * NR)
    rho0 /= rho0.sum()
    got, info = _krylov_gpu(NR, theta, rho0, times, kappa, kind=synth.TWOSTATE)
    ref, rinfo = oracle.krylov(oracle.build_model(oracle.TWOSTATE, [NR], theta), rho0, times, kappa=kappa)
    assert info["omega"] == rinfo["max_exit"]
    assert list(info["K"]) == list(rinfo["steps"])
    assert np.abs(got - ref).max() <= 1e-12


def test_krylov_accuracy_and_refusals():
    import torch
    import paper_2312_05647_gb300 as mjp
    from paper_2312_05647_gb300.capi import MJPError
    cfg = synth.bd_small()
    got, _ = _krylov_gpu(64, cfg["theta"], cfg["rho0"], cfg["times"])
    ref, _ = oracle.expv(oracle.build_model(oracle.BD1D, [64], cfg["theta"]), cfg["rho0"], cfg["times"],
                         mode=oracle.TOL, tol=1e-16)
    assert np.abs(got - ref).max() <= 1e-9
    with pytest.raises(MJPError):
        _krylov_gpu(64, cfg["theta"], cfg["rho0"], [1.0], prec=1)  # FP32
    m = mjp.Model(synth.BD1D, [64], cfg["theta"], mjp.FP64)
    for bad in (0, 33):
        with pytest.raises(MJPError):
            m.set_option(mjp.OPT_KAPPA, bad)
    m.set_option(mjp.OPT_METHOD, mjp.METHOD_KRYLOV)
    with pytest.raises(MJPError):
        mjp.Model(synth.BD1D, [5000], cfg["theta"], mjp.FP64).set_option(mjp.OPT_METHOD, 3)
    big = mjp.Model(synth.BD1D, [5000], cfg["theta"], mjp.FP64)
    big.set_option(mjp.OPT_METHOD, mjp.METHOD_KRYLOV)
    with pytest.raises(MJPError):
        big.expv(torch.tensor(synth.delta(5000, 0), device="cuda"), [0.01])
