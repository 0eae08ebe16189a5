"""ctypes binding of libmjp.so (include/mjp.h, include/mjp_surrogate.h): argument
marshalling only.

Every numerical step runs in the library's CUDA kernels.  PyTorch supplies
device memory and the current stream; there is no CPU fallback, and loading
fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_lib", "libmjp.so")

MJP_OK = 0
ERRORS = {-1: "MJP_ERR_ARG", -2: "MJP_ERR_CSR", -3: "MJP_ERR_ALLOC", -4: "MJP_ERR_CUDA",
          -5: "MJP_ERR_DEVICE_TIMEOUT", -6: "MJP_ERR_KCAP", -7: "MJP_ERR_NUMERIC",
          -8: "MJP_ERR_UNSUPPORTED"}
BD1D, TWOSTATE, MRNA_PROT2D, CSR, AUTOREG = 1, 2, 3, 4, 5
FP32, FP64 = 1, 2
TRUNC_PAPER, TRUNC_TOL = 0, 1
PTR_HOST, PTR_DEVICE = 0, 1
OPT_RENORM_PERIOD, OPT_K_CAP, OPT_THREADS, OPT_CLUSTER, OPT_PROFILE, OPT_ARENA, OPT_CHAIN, OPT_HALO = 1, 2, 3, 4, 5, 6, 7, 8
OPT_METHOD, OPT_KAPPA, OPT_WAIT_LIMIT = 9, 10, 11
METHOD_RMJP, METHOD_RK4, METHOD_KRYLOV = 0, 1, 2
PEAK_FP32_FMA, PEAK_SMEM, PEAK_L2_GATHER = 1, 2, 3

# Every entry point of include/mjp.h: name -> (restype, argtypes).
_vp = ctypes.c_void_p
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)
_f32p = ctypes.POINTER(ctypes.c_float)


class SeriesInfo(ctypes.Structure):
    _fields_ = [("omega", ctypes.c_double), ("K", _i64p), ("eps", _f64p)]


class TrainCfg(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("batch", ctypes.c_int64), ("lr", ctypes.c_double),
                ("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("eps", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("fit_norm", ctypes.c_int)]


class SamplerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("iterations", "accepted", "stage1", "exact_evals", "rounds", "kept",
                                              "evals_kept")]


class AdaptCfg(ctypes.Structure):
    _fields_ = [("every", ctypes.c_int64), ("window", ctypes.c_int64), ("cycle", ctypes.c_int64),
                ("good_cycles", ctypes.c_int64), ("z0", ctypes.c_double), ("eps", ctypes.c_double),
                ("acc_lo", ctypes.c_double), ("acc_hi", ctypes.c_double), ("restart_at_best", ctypes.c_int),
                ("max_iters", ctypes.c_int64)]


class AdaptReport(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int64 * 2), ("good", ctypes.c_int64 * 2), ("converged", ctypes.c_int),
                ("acc_last", ctypes.c_double)]


MLP_NPAR, MLP_NNORM = 17281, 10

SIGNATURES = {
    "mjp_last_error": (ctypes.c_char_p, []),
    "mjp_version": (ctypes.c_char_p, []),
    "rate_model_create_stencil": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, _i64p, ctypes.c_int,
                                                 _f64p, ctypes.c_int, ctypes.c_int]),
    "rate_model_create_csr": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int64, _i64p, _i32p, _f64p,
                                             ctypes.c_int]),
    "rate_model_set_theta": (ctypes.c_int, [_vp, _f64p, ctypes.c_int]),
    "rate_model_set_option": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int64]),
    "rate_model_num_states": (ctypes.c_int64, [_vp]),
    "rate_model_destroy": (None, [_vp]),
    "rate_model_check": (ctypes.c_int, [_vp, _vp]),
    "rate_model_last_timing": (ctypes.c_int, [_vp, _f64p, _f64p]),
    "expv_series": (ctypes.c_int, [_vp, _vp, _f64p, ctypes.c_int, _vp, ctypes.POINTER(SeriesInfo),
                                   ctypes.c_int, ctypes.c_double, _vp]),
    "mjp_obs_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int64, ctypes.c_int, _f64p, _i64p, _f64p,
                                      _i64p, _i32p, _f64p]),
    "mjp_obs_destroy": (None, [_vp]),
    "loglik": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                              _vp]),
    "expv_batch_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, _i64p, _f64p, _f64p,
                                         _i64p, ctypes.c_int]),
    "expv_batch_offsets": (ctypes.c_int, [_vp, _i64p]),
    "expv_batch_run": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp]),
    "expv_batch_tune": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_char_p, ctypes.c_int]),
    "expv_batch_check": (ctypes.c_int, [_vp, _vp]),
    "expv_batch_set_option": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int64]),
    "jmjp_state_probs": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, _i64p, _i64p, _i32p, _f64p, _vp]),
    "expv_batch_destroy": (None, [_vp]),
    "mjp_measure_peak": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _f64p, _vp]),
    "expv_series_static": (ctypes.c_int, [ctypes.c_int, _i64p, ctypes.c_int, _f64p, ctypes.c_int, _vp, _f64p,
                                          ctypes.c_int, _vp, _vp]),
    # include/mjp_surrogate.h
    "mjp_mlp_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_uint64]),
    "mjp_mlp_destroy": (None, [_vp]),
    "mjp_mlp_set_params": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp]),
    "mjp_mlp_get_params": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp]),
    "mjp_mlp_fit_norm": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64, ctypes.c_int, _vp]),
    "mjp_mlp_forward": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, _vp, ctypes.c_int, _vp]),
    "mjp_mlp_loss_grad": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64, _vp, _vp, ctypes.c_int, _vp]),
    "mjp_mlp_train": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64, ctypes.POINTER(TrainCfg), _vp, ctypes.c_int,
                                     _vp]),
    "mjp_sampler_create": (ctypes.c_int, [ctypes.POINTER(_vp), _vp, _vp, ctypes.c_int, ctypes.c_int64,
                                          ctypes.c_int64, ctypes.c_uint64]),
    "mjp_sampler_destroy": (None, [_vp]),
    "mjp_sampler_set_state": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp]),
    "mjp_sampler_get_state": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp]),
    "mjp_sampler_set_cov": (ctypes.c_int, [_vp, _f64p, _vp]),
    "mjp_sampler_get_cov": (ctypes.c_int, [_vp, _f64p, _vp]),
    "mjp_sampler_adapt_cov": (ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_double, _vp]),
    "mjp_sampler_run_plain": (ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_int, _vp]),
    "mjp_sampler_run_da": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _vp]),
    "mjp_sampler_clear": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
    "mjp_sampler_stats_get": (ctypes.c_int, [_vp, ctypes.POINTER(SamplerStats), _vp]),
    "mjp_sampler_trace": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _vp]),
    "mjp_sampler_evals": (ctypes.c_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i64p]),
    "mjp_sampler_checkpoint_size": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "mjp_sampler_save": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t, _vp]),
    "mjp_sampler_load": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t, _vp]),
    "mjp_sampler_adapt": (ctypes.c_int, [_vp, ctypes.POINTER(AdaptCfg), ctypes.POINTER(AdaptReport), _vp]),
    "mjp_ess": (ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, _vp, _vp, _vp, _vp, _vp,
                               ctypes.c_int, _vp]),
}

_LIB = None


class MJPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def lib():
    """Load libmjp.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_2312_05647_gb300.build.build() "
                              "(or __graft_entry__.build()) first; there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _LIB = L
    return _LIB


def check(rc: int):
    if rc != MJP_OK:
        raise MJPError(rc, lib().mjp_last_error().decode())
    return rc
