"""GB300 (sm_103a) implementation of the R-MJP jump-truncated uniformisation
series of Pessoa, Schweiger & Presse (arXiv 2312.05647).

Thin Python layer over the C ABI in ``include/mjp.h``: handles, argument
marshalling and torch tensors for device memory and streams.  Importing the
package does not load the CUDA library; the first call does, and fails
loudly if it is missing.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import capi
from .capi import (AUTOREG, BD1D, CSR, FP32, FP64, METHOD_KRYLOV, METHOD_RK4, METHOD_RMJP, MRNA_PROT2D, OPT_ARENA,
                   OPT_CHAIN, OPT_CLUSTER, OPT_HALO, OPT_K_CAP, OPT_KAPPA, OPT_METHOD, OPT_PROFILE, OPT_WAIT_LIMIT, OPT_RENORM_PERIOD, OPT_THREADS, PEAK_FP32_FMA, PEAK_L2_GATHER, PEAK_SMEM, PTR_DEVICE, PTR_HOST, TRUNC_PAPER, TRUNC_TOL, TWOSTATE,
                   MJPError)

__all__ = ["Model", "Obs", "Batch", "loglik", "BD1D", "TWOSTATE", "MRNA_PROT2D", "AUTOREG", "CSR", "FP32", "FP64",
           "TRUNC_PAPER", "TRUNC_TOL", "MJPError"]

_NTHETA = {BD1D: 2, TWOSTATE: 4, MRNA_PROT2D: 4, AUTOREG: 6}


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Model:
    """A rate model (stencil or CSR) living on the current CUDA device."""

    def __init__(self, kind: int, dims, theta, precision: int = FP32):
        L = capi.lib()
        self._h = ctypes.c_void_p()
        d = np.ascontiguousarray(dims, dtype=np.int64)
        th = _f64(theta)
        capi.check(L.rate_model_create_stencil(ctypes.byref(self._h), int(kind), d.ctypes.data_as(capi._i64p),
                                               len(d), th.ctypes.data_as(capi._f64p), len(th), int(precision)))
        self.kind, self.dims, self.precision = kind, list(d), precision

    @classmethod
    def from_csr(cls, n, row_ptr, col, rate, precision: int = FP32):
        self = cls.__new__(cls)
        L = capi.lib()
        self._h = ctypes.c_void_p()
        rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
        c = np.ascontiguousarray(col, dtype=np.int32)
        v = _f64(rate)
        capi.check(L.rate_model_create_csr(ctypes.byref(self._h), int(n), rp.ctypes.data_as(capi._i64p),
                                           c.ctypes.data_as(capi._i32p), v.ctypes.data_as(capi._f64p),
                                           int(precision)))
        self.kind, self.dims, self.precision = CSR, [int(n)], precision
        return self

    @property
    def n(self) -> int:
        return int(capi.lib().rate_model_num_states(self._h))

    @property
    def torch_dtype(self):
        import torch
        return torch.float64 if self.precision == FP64 else torch.float32

    def set_theta(self, theta):
        th = _f64(theta)
        capi.check(capi.lib().rate_model_set_theta(self._h, th.ctypes.data_as(capi._f64p), len(th)))

    def set_option(self, option: int, value: int):
        capi.check(capi.lib().rate_model_set_option(self._h, int(option), int(value)))

    def expv(self, rho0, times, trunc: int = TRUNC_PAPER, tol: float = 0.0, info: bool = False,
             out=None, stream=None):
        """rho*(t_i) for each time; rho0 is a CUDA tensor of length N in the
        model's precision.  Returns (ntimes, N) [and the truncation info]."""
        import torch
        if not (isinstance(rho0, torch.Tensor) and rho0.is_cuda and rho0.dtype == self.torch_dtype
                and rho0.is_contiguous() and rho0.numel() == self.n):
            raise ValueError("rho0 must be a contiguous CUDA tensor of N values in the model precision")
        t = _f64(np.atleast_1d(times))
        if out is None:
            out = torch.empty((len(t), self.n), dtype=self.torch_dtype, device=rho0.device)
        inf = None
        if info:
            K = np.zeros(len(t), np.int64)
            eps = np.zeros(len(t))
            inf = capi.SeriesInfo(0.0, K.ctypes.data_as(capi._i64p), eps.ctypes.data_as(capi._f64p))
        capi.check(capi.lib().expv_series(self._h, ctypes.c_void_p(rho0.data_ptr()), t.ctypes.data_as(capi._f64p),
                                          len(t), ctypes.c_void_p(out.data_ptr()),
                                          ctypes.byref(inf) if info else None, int(trunc), float(tol),
                                          _stream_ptr(stream)))
        if info:
            return out, {"omega": inf.omega, "K": K, "eps": eps}
        return out

    def check(self, stream=None):
        capi.check(capi.lib().rate_model_check(self._h, _stream_ptr(stream)))

    def jmjp_probs(self, rho0, k, groups, stream=None):
        """J-MJP state probabilities (Algorithm 1): phi_i = sum over groups[i]
        of (rho0 B^{k_i}) for the model's theta; rho0 a device tensor.  groups:
        a list of member arrays, or the flat pair (group_ptr, members) with
        group_ptr[0] = 0 and len(group_ptr) = len(k) + 1."""
        kk = np.ascontiguousarray(k, dtype=np.int64)
        if isinstance(groups, tuple) and len(groups) == 2 and np.ndim(groups[0]) == 1 and len(groups[0]) == len(kk) + 1:
            gp = np.ascontiguousarray(groups[0], dtype=np.int64)
            mem = np.ascontiguousarray(groups[1], dtype=np.int32)
        else:
            gp = np.zeros(len(groups) + 1, np.int64)
            gp[1:] = np.cumsum([len(g) for g in groups])
            mem = np.ascontiguousarray(np.concatenate(groups), dtype=np.int32)
        phi = np.zeros(len(kk))
        capi.check(capi.lib().jmjp_state_probs(self._h, ctypes.c_void_p(rho0.data_ptr()), len(kk),
                                               kk.ctypes.data_as(capi._i64p), gp.ctypes.data_as(capi._i64p),
                                               mem.ctypes.data_as(capi._i32p), phi.ctypes.data_as(capi._f64p),
                                               _stream_ptr(stream)))
        return phi

    def last_timing(self):
        """(planner ms, chain ms) of the last call (needs OPT_PROFILE = 1)."""
        a, b = ctypes.c_double(), ctypes.c_double()
        capi.check(capi.lib().rate_model_last_timing(self._h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            capi.lib().rate_model_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Obs:
    """Snapshot observations (times, groups of states with counts, rho0)."""

    def __init__(self, n: int, times, obs_groups, rho0):
        """obs_groups: list over times of (members_list, counts)."""
        gptr, counts, mptr, members = [0], [], [0], []
        for mem_list, cnt in obs_groups:
            for mem, c in zip(mem_list, cnt):
                members.extend(int(v) for v in np.atleast_1d(mem))
                mptr.append(len(members))
                counts.append(float(c))
            gptr.append(len(counts))
        t = _f64(times)
        g = np.array(gptr, np.int64)
        c = np.array(counts if counts else [0.0], np.float64)
        mp = np.array(mptr, np.int64)
        mem = np.array(members if members else [0], np.int32)
        r0 = _f64(rho0)
        self._h = ctypes.c_void_p()
        capi.check(capi.lib().mjp_obs_create(ctypes.byref(self._h), int(n), len(t), t.ctypes.data_as(capi._f64p),
                                             g.ctypes.data_as(capi._i64p), c.ctypes.data_as(capi._f64p),
                                             mp.ctypes.data_as(capi._i64p), mem.ctypes.data_as(capi._i32p),
                                             r0.ctypes.data_as(capi._f64p)))
        self.n, self.ntimes, self.ngroups = n, len(t), len(counts)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            capi.lib().mjp_obs_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def loglik(model: Model, obs: Obs, theta, trunc: int = TRUNC_PAPER, tol: float = 0.0, out=None, stream=None):
    """Log-likelihood for each row of theta (B x ntheta).

    theta as a NumPy array -> host call, returns a NumPy array (synchronous).
    theta as a CUDA float64 tensor -> device call, returns a CUDA tensor
    (asynchronous on the current stream)."""
    L = capi.lib()
    try:
        import torch
        is_tensor = isinstance(theta, torch.Tensor)
    except ImportError:
        is_tensor = False
    if is_tensor:
        if not (theta.is_cuda and theta.dtype == torch.float64 and theta.is_contiguous()):
            raise ValueError("device theta must be a contiguous CUDA float64 tensor")
        B = theta.shape[0] if theta.dim() == 2 else 1
        if out is None:
            out = torch.empty(B, dtype=torch.float64, device=theta.device)
        capi.check(L.loglik(model._h, obs._h, ctypes.c_void_p(theta.data_ptr()), B,
                            ctypes.c_void_p(out.data_ptr()), PTR_DEVICE, int(trunc), float(tol),
                            _stream_ptr(stream)))
        return out
    th = _f64(np.atleast_2d(theta))
    B = th.shape[0]
    res = np.zeros(B)
    capi.check(L.loglik(model._h, obs._h, ctypes.c_void_p(th.ctypes.data), B, ctypes.c_void_p(res.ctypes.data),
                        PTR_HOST, int(trunc), float(tol), _stream_ptr(stream)))
    return res


def measure_peak(which: int, iters: int = 200000, stream=None) -> float:
    """Measured on-chip peak of the current device: PEAK_FP32_FMA (TFLOP/s)
    or PEAK_SMEM (GB/s, read + write); see mjp_measure_peak."""
    v = ctypes.c_double()
    capi.check(capi.lib().mjp_measure_peak(int(which), int(iters), ctypes.byref(v), _stream_ptr(stream)))
    return v.value


class Batch:
    """Uneven birth-death instances evaluated in one call (expv_batch_*)."""

    def __init__(self, N, theta, t, s0=None, precision: int = FP32, kind: int = BD1D):
        L = capi.lib()
        n = np.ascontiguousarray(N, dtype=np.int64)
        th = _f64(theta).reshape(len(n), 2)
        tt = _f64(t)
        s = None if s0 is None else np.ascontiguousarray(s0, dtype=np.int64)
        self._h = ctypes.c_void_p()
        capi.check(L.expv_batch_create(ctypes.byref(self._h), int(kind), len(n), n.ctypes.data_as(capi._i64p),
                                       th.ctypes.data_as(capi._f64p), tt.ctypes.data_as(capi._f64p),
                                       None if s is None else s.ctypes.data_as(capi._i64p), int(precision)))
        self.n, self.precision = len(n), precision
        self.offsets = np.zeros(len(n) + 1, np.int64)
        capi.check(L.expv_batch_offsets(self._h, self.offsets.ctypes.data_as(capi._i64p)))

    @property
    def torch_dtype(self):
        import torch
        return torch.float64 if self.precision == FP64 else torch.float32

    def empty_out(self, device="cuda"):
        import torch
        return torch.empty(int(self.offsets[-1]), dtype=self.torch_dtype, device=device)

    def run(self, out, use_graph: bool = False, stream=None):
        capi.check(capi.lib().expv_batch_run(self._h, ctypes.c_void_p(out.data_ptr()), int(use_graph),
                                             _stream_ptr(stream)))
        return out

    def tune(self, out, stream=None) -> str:
        buf = ctypes.create_string_buffer(512)
        capi.check(capi.lib().expv_batch_tune(self._h, ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream), buf,
                                              512))
        return buf.value.decode()

    def check(self, stream=None):
        capi.check(capi.lib().expv_batch_check(self._h, _stream_ptr(stream)))

    def set_option(self, option: int, value: int):
        capi.check(capi.lib().expv_batch_set_option(self._h, int(option), int(value)))

    def split(self, out):
        """Per-instance views of a run's output."""
        return [out[self.offsets[j]:self.offsets[j + 1]] for j in range(self.n)]

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            capi.lib().expv_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
