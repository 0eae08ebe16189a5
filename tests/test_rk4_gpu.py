"""Fourth-order Runge-Kutta on the GPU (Method #4, Sec. 2.3; MJP_OPT_METHOD = 1)
against the oracle's RK4: the same step rule (ceil(interval x max_n |a_nn|)
equal steps per interval between ascending times) and the same operation
order per state, so the results agree to the bit; plus the method's refusals."""
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


def _rk4_gpu(N, theta, rho0, times, prec=2, kind=synth.BD1D):
    import torch
    import paper_2312_05647_gb300 as mjp
    m = mjp.Model(kind, [N], theta, prec)
    m.set_option(mjp.OPT_METHOD, mjp.METHOD_RK4)
    r = torch.tensor(rho0, dtype=m.torch_dtype, device="cuda")
    out, info = m.expv(r, times, info=True)
    m.check()
    return out.cpu().numpy(), info


@pytest.mark.parametrize("N,theta,times", [
    (64, [10.0, 1.0], [0.1, 0.5, 1.0, 2.0, 5.0]),          # immigration-death, the latency configuration
    (1, [3.0, 1.0], [0.5]),
    (2, [2.0, 3.0], [0.9, 0.0, 3.3]),
    (17, [4.0, 0.7], [1.2, 0.3]),
    (1000, [300.0, 1.0], [0.002, 0.01]),
    (1025, [200.0, 0.5], [0.004]),
    (4096, [1000.0, 1.0], [0.001, 0.0005]),
])
def test_rk4_matches_oracle_bitwise(N, theta, times):
    gen = np.random.default_rng(N)
    rho0 = gen.random(N)
    rho0 /= rho0.sum()
    got, info = _rk4_gpu(N, theta, rho0, times)
    ref, rinfo = oracle.rk4(oracle.build_model(oracle.BD1D, [N], theta), rho0, times)
    assert info["omega"] == rinfo["max_exit"]
    assert list(info["K"]) == list(rinfo["steps"])
    assert np.abs(got - ref).max() <= 1e-12
    np.testing.assert_array_equal(got, ref)


@pytest.mark.parametrize("NR,theta,times", [
    (300, [100.0, 1.0, 2.0, 1.0], [0.5, 0.05, 0.2]),        # the promoter of Sec. 3.1.2
    (2, [3.0, 0.5, 1.5, 2.0], [1.0, 0.3]),
    (37, [20.0, 0.5, 0.3, 1.5], [0.7, 2.0]),
    (2048, [900.0, 1.0, 2.0, 1.0], [0.002]),                # 4,096 states, 8 per thread
])
def test_rk4_two_state_matches_oracle_bitwise(NR, theta, times):
    gen = np.random.default_rng(NR)
    rho0 = gen.random(2 * NR)
    rho0 /= rho0.sum()
    got, info = _rk4_gpu(NR, theta, rho0, times, kind=synth.TWOSTATE)
    ref, rinfo = oracle.rk4(oracle.build_model(oracle.TWOSTATE, [NR], theta), rho0, times)
    assert info["omega"] == rinfo["max_exit"]
    assert list(info["K"]) == list(rinfo["steps"])
    np.testing.assert_array_equal(got, ref)


def test_rk4_against_rmjp_and_refusals():
    import paper_2312_05647_gb300 as mjp
    from paper_2312_05647_gb300.capi import MJPError
    cfg = synth.bd_small()
    got, _ = _rk4_gpu(64, cfg["theta"], cfg["rho0"], cfg["times"])
    ref, _ = oracle.expv(oracle.build_model(oracle.BD1D, [64], cfg["theta"]), cfg["rho0"], cfg["times"],
                         mode=oracle.TOL, tol=1e-15)
    # RK4's global error at h <= 1 / max|a_nn| on this model (5.3e-6 at t = 0.1).
    assert np.abs(got - ref).max() <= 1e-5
    with pytest.raises(MJPError):
        _rk4_gpu(64, cfg["theta"], cfg["rho0"], [1.0], prec=1)   # FP32
    with pytest.raises(MJPError):
        _rk4_gpu(5000, [10.0, 1.0], synth.delta(5000, 0), [0.01])  # beyond one CTA
    m = mjp.Model(synth.MRNA_PROT2D, [10, 10], [5.0, 1.0, 1.0, 0.2], mjp.FP64)
    m.set_option(mjp.OPT_METHOD, mjp.METHOD_RK4)
    import torch
    with pytest.raises(MJPError):
        m.expv(torch.tensor(synth.delta(100, 0), device="cuda"), [1.0])
    with pytest.raises(MJPError):
        m.set_option(mjp.OPT_METHOD, 3)
