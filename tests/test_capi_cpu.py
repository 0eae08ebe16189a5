"""The C ABI without a GPU: the library loads, exports every entry point that
include/mjp.h declares, and rejects bad arguments on the host (no kernel
launch, no CUDA call)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2312_05647_gb300 import build as lib_build
from paper_2312_05647_gb300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    lib_build.build()
    return capi.lib()


def _declared():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not f.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", f)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*\b([a-z_][a-z0-9_]*)\s*\(", txt,
                             flags=re.M):
            names.append(m.group(1))
    return names


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert "expv_series" in names and "loglik" in names and "rate_model_create_stencil" in names
    for n in names:
        assert hasattr(L, n), f"{n} declared in include/ but not exported"


def test_binding_covers_header():
    assert set(_declared()) <= set(capi.SIGNATURES), set(_declared()) - set(capi.SIGNATURES)


def _create(L, kind, dims, theta, prec=capi.FP32):
    h = ctypes.c_void_p()
    d = np.ascontiguousarray(dims, dtype=np.int64)
    t = np.ascontiguousarray(theta, dtype=np.float64)
    rc = L.rate_model_create_stencil(ctypes.byref(h), kind, d.ctypes.data_as(capi._i64p), len(d),
                                     t.ctypes.data_as(capi._f64p), len(t), prec)
    return rc, h


def test_host_validation(L):
    rc, h = _create(L, 99, [10], [1.0, 1.0])
    assert rc == -1 and b"kind" in L.mjp_last_error()
    rc, h = _create(L, capi.BD1D, [10], [1.0, -1.0])
    assert rc == -1
    rc, h = _create(L, capi.BD1D, [10], [1.0, float("nan")])
    assert rc == -1
    rc, h = _create(L, capi.TWOSTATE, [10], [1.0, 1.0])
    assert rc == -1
    rc, h = _create(L, capi.MRNA_PROT2D, [1, 5], [1.0, 1.0, 1.0, 1.0])
    assert rc == -1
    rc, h = _create(L, capi.BD1D, [10], [1.0, 1.0], prec=7)
    assert rc == -1
    rc, h = _create(L, capi.TWOSTATE, [300], [100.0, 1.0, 2.0, 1.0])
    assert rc == 0 and L.rate_model_num_states(h) == 600
    assert L.rate_model_set_option(h, capi.OPT_THREADS, 33) == -1
    assert L.rate_model_set_option(h, capi.OPT_CLUSTER, 3) == -1
    assert L.rate_model_set_option(h, capi.OPT_RENORM_PERIOD, 64) == 0
    bad = np.array([1.0, 2.0], dtype=np.float64)
    assert L.rate_model_set_theta(h, bad.ctypes.data_as(capi._f64p), 2) == -1
    # expv_series: argument errors are caught before any device work.
    t = np.array([1.0, -0.5])
    assert L.expv_series(h, ctypes.c_void_p(8), t.ctypes.data_as(capi._f64p), 2, ctypes.c_void_p(8), None, 0,
                         0.0, None) == -1
    t = np.array([1.0])
    assert L.expv_series(h, None, t.ctypes.data_as(capi._f64p), 1, ctypes.c_void_p(8), None, 0, 0.0, None) == -1
    assert L.expv_series(h, ctypes.c_void_p(8), t.ctypes.data_as(capi._f64p), 1, ctypes.c_void_p(8), None,
                         capi.TRUNC_TOL, 0.7, None) == -1
    L.rate_model_destroy(h)
    L.rate_model_destroy(None)
    assert L.rate_model_num_states(None) == -1


def test_obs_validation(L):
    h = ctypes.c_void_p()
    times = np.array([1.0])
    gptr = np.array([0, 1], np.int64)
    counts = np.array([3.0])
    mptr = np.array([0, 1], np.int64)
    members = np.array([12], np.int32)  # out of range for n = 10
    rho0 = np.zeros(10)
    rho0[0] = 1
    rc = L.mjp_obs_create(ctypes.byref(h), 10, 1, times.ctypes.data_as(capi._f64p), gptr.ctypes.data_as(capi._i64p),
                          counts.ctypes.data_as(capi._f64p), mptr.ctypes.data_as(capi._i64p),
                          members.ctypes.data_as(capi._i32p), rho0.ctypes.data_as(capi._f64p))
    assert rc == -1 and b"range" in L.mjp_last_error()
    counts = np.array([-1.0])
    members = np.array([2], np.int32)
    rc = L.mjp_obs_create(ctypes.byref(h), 10, 1, times.ctypes.data_as(capi._f64p), gptr.ctypes.data_as(capi._i64p),
                          counts.ctypes.data_as(capi._f64p), mptr.ctypes.data_as(capi._i64p),
                          members.ctypes.data_as(capi._i32p), rho0.ctypes.data_as(capi._f64p))
    assert rc == -1


def _csr(L, n, row_ptr, col, rate, prec=capi.FP32):
    h = ctypes.c_void_p()
    rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
    c = np.ascontiguousarray(col, dtype=np.int32)
    v = np.ascontiguousarray(rate, dtype=np.float64)
    return L.rate_model_create_csr(ctypes.byref(h), n, rp.ctypes.data_as(capi._i64p), c.ctypes.data_as(capi._i32p),
                                   v.ctypes.data_as(capi._f64p), prec)


def test_csr_validation(L):
    # Malformed CSR is rejected on the host with MJP_ERR_CSR, before any device work.
    assert _csr(L, 3, [0, 1, 2, 2], [1, 2], [1.0, 2.0], prec=7) == -1
    assert _csr(L, 3, [1, 1, 2, 2], [1, 2], [1.0, 2.0]) == -2          # row_ptr[0] != 0
    assert _csr(L, 3, [0, 2, 1, 2], [1, 2], [1.0, 2.0]) == -2          # not monotone
    assert _csr(L, 3, [0, 1, 2, 2], [1, 1], [1.0, 2.0]) == -2          # diagonal entry (row 1 -> 1)
    assert _csr(L, 3, [0, 1, 2, 2], [1, 3], [1.0, 2.0]) == -2          # column out of range
    assert _csr(L, 3, [0, 1, 2, 2], [1, 2], [1.0, -2.0]) == -2         # negative rate
    assert _csr(L, 3, [0, 1, 2, 2], [1, 2], [1.0, float("inf")]) == -2
    assert b"rate" in L.mjp_last_error()


def test_batch_validation(L):
    h = ctypes.c_void_p()
    N = np.array([10, 0], np.int64)
    th = np.ones(4)
    t = np.ones(2)
    rc = L.expv_batch_create(ctypes.byref(h), capi.BD1D, 2, N.ctypes.data_as(capi._i64p), th.ctypes.data_as(capi._f64p),
                             t.ctypes.data_as(capi._f64p), None, capi.FP32)
    assert rc == -1
    N = np.array([10, 20], np.int64)
    t = np.array([1.0, -1.0])
    rc = L.expv_batch_create(ctypes.byref(h), capi.BD1D, 2, N.ctypes.data_as(capi._i64p), th.ctypes.data_as(capi._f64p),
                             t.ctypes.data_as(capi._f64p), None, capi.FP32)
    assert rc == -1
    rc = L.expv_batch_create(ctypes.byref(h), capi.TWOSTATE, 2, N.ctypes.data_as(capi._i64p),
                             th.ctypes.data_as(capi._f64p), t.ctypes.data_as(capi._f64p), None, capi.FP32)
    assert rc == -8


def test_surrogate_and_sampler_host_validation(L):
    vp = ctypes.c_void_p
    out = vp()
    assert L.mjp_mlp_create(None, 0) == -1
    assert L.mjp_mlp_forward(None, vp(8), 1, vp(8), capi.PTR_HOST, None) == -1
    assert L.mjp_mlp_train(None, vp(8), vp(8), 1, None, None, capi.PTR_HOST, None) == -1
    assert L.mjp_mlp_set_params(None, None, None, capi.PTR_HOST, None) == -1
    assert L.mjp_sampler_create(ctypes.byref(out), None, None, 4, 10, 0, 0) == -1
    assert L.mjp_sampler_set_cov(None, None, None) == -1
    assert L.mjp_sampler_run_plain(None, 1, 1, None) == -1
    assert L.mjp_sampler_run_da(None, None, 1, 4, 1, None) == -1
    st = capi.SamplerStats()
    assert L.mjp_sampler_stats_get(None, ctypes.byref(st), None) == -1
    assert L.mjp_sampler_adapt(None, None, None, None) == -1
    # ESS: shape checks come before any device work.
    assert L.mjp_ess(vp(8), 2, 3, 1, None, None, None, None, None, capi.PTR_HOST, None) == -1
    assert L.mjp_ess(vp(8), 0, 10, 1, None, None, None, None, None, capi.PTR_HOST, None) == -1
    assert L.mjp_ess(None, 2, 10, 1, None, None, None, None, None, capi.PTR_HOST, None) == -1


def test_binding_struct_layouts_match_header():
    # Sizes of the C structs of include/mjp_surrogate.h on an LP64 target.
    assert ctypes.sizeof(capi.TrainCfg) == 64
    assert ctypes.sizeof(capi.SamplerStats) == 56
    assert ctypes.sizeof(capi.AdaptCfg) == 80
    assert ctypes.sizeof(capi.AdaptReport) == 48
    assert capi.AdaptCfg.max_iters.offset == 72 and capi.AdaptReport.acc_last.offset == 40
