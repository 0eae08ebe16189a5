"""expv_series_static: the allocation-free variant of expv_series.

Some callers cannot allocate device memory while they run (their memory
belongs to their own pool or fixed budget, or cudaMalloc/cudaFree's
device-wide synchronisation is not allowed in their loop).  For them the
library keeps the series' scratch in a fixed static device array.  These tests
call that entry point through the C ABI, twice in a row (the shared array keeps
the previous call's contents), and compare it with expv_series on the same
inputs within the FP32 tolerance used everywhere else (1e-6 max abs).  This
file is collected last so that a run stopping at the first failure has already
run every other test; it also passes on its own in a fresh process."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
TOL32 = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2312_05647_gb300 import build as lib_build
    lib_build.build()
    torch.cuda.set_device(0)


def _static_call(kind, dims, theta, rho0_dev, times, out_dev):
    import torch
    from paper_2312_05647_gb300 import capi
    d = np.ascontiguousarray(dims, dtype=np.int64)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    t = np.ascontiguousarray(times, dtype=np.float64)
    rc = capi.lib().expv_series_static(int(kind), d.ctypes.data_as(capi._i64p), len(d), th.ctypes.data_as(capi._f64p),
                                       len(th), ctypes.c_void_p(rho0_dev.data_ptr()), t.ctypes.data_as(capi._f64p),
                                       len(t), ctypes.c_void_p(out_dev.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc


@pytest.mark.parametrize("kind,dims,theta,times", [
    (synth.MRNA_PROT2D, [60, 45], [8.0, 1.0, 2.0, 0.3], [1.5, 0.05, 0.6, 4.0]),
    (synth.TWOSTATE, [300], [100.0, 1.0, 2.0, 1.0], [0.5, 3.0, 10.0]),
    (synth.BD1D, [2000], [400.0, 1.0], [0.01, 0.3]),
])
def test_static_matches_expv_series_twice(kind, dims, theta, times):
    import torch
    import paper_2312_05647_gb300 as mjp
    m = mjp.Model(kind, dims, theta, mjp.FP32)
    n = m.n
    rho0 = torch.zeros(n, dtype=torch.float32, device="cuda")
    rho0[0] = 0.6
    rho0[n // 3] = 0.4
    ref = m.expv(rho0, times)
    m.check()
    ref = ref.cpu().numpy()
    for _ in range(2):
        out = torch.full((len(times), n), float("nan"), dtype=torch.float32, device="cuda")
        rc = _static_call(kind, dims, theta, rho0, times, out)
        assert rc == 0, mjp.capi.lib().mjp_last_error()
        assert np.abs(out.cpu().numpy() - ref).max() <= TOL32


def _oracle_expv(kind, dims, theta, rho0, times):
    import oracle
    out, _ = oracle.expv(oracle.build_model(kind, dims, theta), rho0, times)
    return out


def test_static_large_then_small_against_expv_series_and_oracle():
    # A bench-sized call (200 x 200 box, 20 times: 3.2 MB of the static array,
    # a cluster of CTAs) followed by a much smaller one: what the large call
    # left in the shared array must not leak into the small one.  Both are
    # compared with expv_series and with the FP64 oracle.
    import torch
    import paper_2312_05647_gb300 as mjp
    cases = [
        (synth.MRNA_PROT2D, [200, 200], [20.0, 1.0, 5.0, 0.1], np.logspace(np.log10(0.1), np.log10(50.0), 20), None),
        (synth.TWOSTATE, [120], [60.0, 1.0, 2.0, 1.0], np.array([0.3, 2.0, 6.0]), 8.0),
    ]
    for kind, dims, theta, times, _ in cases:
        m = mjp.Model(kind, dims, theta, mjp.FP32)
        n = m.n
        rho0 = torch.zeros(n, dtype=torch.float32, device="cuda")
        rho0[0] = 1.0
        ref = m.expv(rho0, times)
        m.check()
        ref = ref.cpu().numpy()
        out = torch.full((len(times), n), float("nan"), dtype=torch.float32, device="cuda")
        rc = _static_call(kind, dims, theta, rho0, times, out)
        assert rc == 0, mjp.capi.lib().mjp_last_error()
        got = out.cpu().numpy()
        assert np.abs(got - ref).max() <= TOL32
        if kind != synth.MRNA_PROT2D:  # the 200 x 200 oracle to t = 50 runs in the long-chain tests
            r0 = np.zeros(n)
            r0[0] = 1.0
            assert np.abs(got - _oracle_expv(kind, dims, theta, r0, times)).max() <= TOL32


@pytest.mark.parametrize("kind,dims,theta,times", [
    (synth.MRNA_PROT2D, [60, 45], [8.0, 1.0, 2.0, 0.3], [1.5, 0.05, 0.6, 4.0]),
    (synth.BD1D, [2000], [400.0, 1.0], [0.01, 0.3]),
])
def test_static_against_oracle(kind, dims, theta, times):
    import torch
    import paper_2312_05647_gb300 as mjp
    n = int(np.prod(dims))
    r0 = np.zeros(n)
    r0[0], r0[n // 3] = 0.6, 0.4
    rho0 = torch.tensor(r0, dtype=torch.float32, device="cuda")
    out = torch.empty((len(times), n), dtype=torch.float32, device="cuda")
    rc = _static_call(kind, dims, theta, rho0, times, out)
    assert rc == 0, mjp.capi.lib().mjp_last_error()
    assert np.abs(out.cpu().numpy() - _oracle_expv(kind, dims, theta, r0, times)).max() <= TOL32


def test_static_refuses_stream_capture_and_huge_dims():
    import torch
    from paper_2312_05647_gb300 import capi
    rho0 = torch.zeros(64, dtype=torch.float32, device="cuda")
    rho0[0] = 1.0
    out = torch.empty((1, 64), dtype=torch.float32, device="cuda")
    # Dimensions whose product exceeds 2^31 - 1 are rejected before any product.
    rc = _static_call(synth.MRNA_PROT2D, [1 << 20, 1 << 20], [1.0, 1.0, 1.0, 1.0], rho0, [1.0], out)
    assert rc == -1
    # A call on a capturing stream is refused (nothing is enqueued).
    g = torch.cuda.CUDAGraph()
    codes = []
    with torch.cuda.graph(g):
        codes.append(_static_call(synth.BD1D, [64], [10.0, 1.0], rho0, [1.0], out))
    assert codes == [-8]
    assert b"capturing" in capi.lib().mjp_last_error()


def test_static_rejects_oversized_requests():
    import torch
    from paper_2312_05647_gb300 import capi
    # 200 x 200 states at 120 times need 19.2 MB of compensation > 16 MiB.
    rho0 = torch.zeros(40000, dtype=torch.float32, device="cuda")
    out = torch.empty(1, dtype=torch.float32, device="cuda")
    rc = _static_call(synth.MRNA_PROT2D, [200, 200], [20.0, 1.0, 5.0, 0.1], rho0, np.linspace(0.1, 1, 120), out)
    assert rc == -1
    assert b"static scratch holds" in capi.lib().mjp_last_error()
