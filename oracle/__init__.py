"""CPU oracle for the R-MJP transient distribution -- TEST INFRASTRUCTURE ONLY.

Plain, slow, FP64 reference code written from the paper (Pessoa, Schweiger &
Presse, arXiv 2312.05647).  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package; the product path
(the CUDA library and its binding) never does, and this package imports
nothing from it.  The compiled part lives in ``mjp_oracle.c``; this module is
argument marshalling plus the few steps that are plain NumPy:

* ``loglik`` -- the snapshot log-likelihood of Sec. 2.1.2 (``p(s^i|theta) =
  rho(T^i)_{s^i}``, product over observations, hidden states summed out as in
  Sec. 3.1.2), evaluated from ``expv`` output;
* ``log_prior`` -- the normal prior on Psi = log(theta), Eq. prior (SI A.4.1).

Parity status: every function is pinned by ``tests/test_oracle_pins.py``
(closed forms, an independent library routine, brute force or a statistical
test); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mjp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_LOCK = threading.Lock()
_LIB = None

BD1D, TWOSTATE, MRNA_PROT2D, AUTOREG = 1, 2, 3, 5
PAPER, TOL = 0, 1

_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add, no -ffast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            lib.orc_build_model.restype = ctypes.c_int64
            lib.orc_build_model.argtypes = [ctypes.c_int, _i64p, ctypes.c_int, _f64p, ctypes.c_int,
                                            _i64p, _i32p, _f64p, ctypes.c_int64]
            lib.orc_max_exit.restype = ctypes.c_double
            lib.orc_max_exit.argtypes = [ctypes.c_int64, _i64p, _f64p]
            lib.orc_K_paper.restype = ctypes.c_int64
            lib.orc_K_paper.argtypes = [ctypes.c_double]
            lib.orc_K_tol.restype = ctypes.c_int64
            lib.orc_K_tol.argtypes = [ctypes.c_double, ctypes.c_double]
            lib.orc_poisson_weights.restype = ctypes.c_int
            lib.orc_poisson_weights.argtypes = [ctypes.c_double, ctypes.c_int64, _f64p, _f64p]
            lib.orc_expv.restype = ctypes.c_int
            lib.orc_expv.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, _f64p, _f64p, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_double, ctypes.c_double, _f64p, _f64p,
                                     _i64p, _f64p]
            lib.orc_jmjp.restype = ctypes.c_int
            lib.orc_jmjp.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, _f64p, ctypes.c_int64, _i64p, _i64p,
                                     _i32p, ctypes.c_double, _f64p]
            lib.orc_rk4.restype = ctypes.c_int
            lib.orc_rk4.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, _f64p, _f64p, ctypes.c_int, _f64p,
                                    _i64p, _f64p]
            lib.orc_krylov.restype = ctypes.c_int
            lib.orc_krylov.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, _f64p, _f64p, ctypes.c_int,
                                       ctypes.c_int, _f64p, _i64p, _f64p]
            lib.orc_expm_pade13.restype = ctypes.c_int
            lib.orc_expm_pade13.argtypes = [ctypes.c_int, _f64p, _f64p]
            lib.orc_gillespie.restype = ctypes.c_int
            lib.orc_gillespie.argtypes = [ctypes.c_int64, _i64p, _i32p, _f64p, ctypes.c_int64, _f64p,
                                          ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, _i64p]
            _LIB = lib
    return _LIB


def _p(a, t):
    return a.ctypes.data_as(t)


class CSR:
    """Rate matrix Lambda, rows = source state, off-diagonal rates only."""

    def __init__(self, row_ptr, col, val):
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.val = np.ascontiguousarray(val, dtype=np.float64)
        self.n = len(self.row_ptr) - 1

    def dense_generator(self) -> np.ndarray:
        """A of Eq. A_def as a dense matrix (tiny N only)."""
        A = np.zeros((self.n, self.n))
        for s in range(self.n):
            for j in range(self.row_ptr[s], self.row_ptr[s + 1]):
                A[s, self.col[j]] += self.val[j]
        A[np.diag_indices(self.n)] = -A.sum(axis=1)
        return A


def build_model(kind: int, dims, theta) -> CSR:
    """Lambda for a stencil model (Eqs. BD_def, Gene_def; Sec. 3.1.3 indexing)."""
    lib = _lib()
    d = np.ascontiguousarray(dims, dtype=np.int64)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    nnz = lib.orc_build_model(kind, _p(d, _i64p), len(d), _p(th, _f64p), len(th), None, None, None, 0)
    if nnz < 0:
        raise ValueError("bad model arguments")
    n = int(np.prod(d)) * (2 if kind in (TWOSTATE, AUTOREG) else 1)
    row_ptr = np.zeros(n + 1, np.int64)
    col = np.zeros(max(nnz, 1), np.int32)
    val = np.zeros(max(nnz, 1), np.float64)
    rc = lib.orc_build_model(kind, _p(d, _i64p), len(d), _p(th, _f64p), len(th), _p(row_ptr, _i64p),
                             _p(col, _i32p), _p(val, _f64p), nnz)
    if rc != nnz:
        raise RuntimeError("model build failed")
    return CSR(row_ptr, col[:nnz], val[:nnz])


def max_exit(csr: CSR) -> float:
    return _lib().orc_max_exit(csr.n, _p(csr.row_ptr, _i64p), _p(csr.val, _f64p))


def K_paper(x: float) -> int:
    """K = floor(x + 6 sqrt(x)) + 1 (Algorithm 2)."""
    return int(_lib().orc_K_paper(float(x)))


def K_tol(x: float, tol: float) -> int:
    return int(_lib().orc_K_tol(float(x), float(tol)))


def poisson_weights(x: float, K: int):
    """(P_0..P_K, eps) with eps = 1 - sum P (Eq. R-MJP_expansion)."""
    P = np.zeros(K + 1)
    eps = ctypes.c_double()
    rc = _lib().orc_poisson_weights(float(x), int(K), _p(P, _f64p), ctypes.byref(eps))
    if rc != 0:
        raise ValueError("bad weight arguments")
    return P, eps.value


def expv(csr: CSR, rho0, times, mode: int = PAPER, tol: float = 0.0, omega_factor: float = 1.1):
    """rho*(t_i) for all times (Algorithm 2 per time, one shared chain).

    Returns (out[ntimes, n], info) with info = {"omega", "K", "eps"}."""
    rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
    times = np.ascontiguousarray(np.atleast_1d(times), dtype=np.float64)
    nt = len(times)
    out = np.zeros((nt, csr.n))
    om = ctypes.c_double()
    K = np.zeros(max(nt, 1), np.int64)
    eps = np.zeros(max(nt, 1))
    rc = _lib().orc_expv(csr.n, _p(csr.row_ptr, _i64p), _p(csr.col, _i32p), _p(csr.val, _f64p),
                         _p(rho0, _f64p), _p(times, _f64p), nt, int(mode), float(tol),
                         float(omega_factor), _p(out, _f64p), ctypes.byref(om), _p(K, _i64p),
                         _p(eps, _f64p))
    if rc != 0:
        raise ValueError(f"orc_expv failed ({rc})")
    return out, {"omega": om.value, "K": K[:nt].copy(), "eps": eps[:nt].copy()}


def jmjp_probs(csr: CSR, rho0, k, groups, omega_factor: float = 1.1):
    """phi_i = sum over group i of (rho0 B^{k_i}) (Algorithm 1, J-MJP): one
    chain read at each observation's jump count.  groups: list of member
    arrays (one per observation)."""
    rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
    k = np.ascontiguousarray(k, dtype=np.int64)
    gp = np.zeros(len(groups) + 1, np.int64)
    gp[1:] = np.cumsum([len(g) for g in groups])
    mem = np.ascontiguousarray(np.concatenate(groups) if len(groups) else np.zeros(0), dtype=np.int32)
    phi = np.zeros(max(len(k), 1))
    rc = _lib().orc_jmjp(csr.n, _p(csr.row_ptr, _i64p), _p(csr.col, _i32p), _p(csr.val, _f64p), _p(rho0, _f64p),
                         len(k), _p(k, _i64p), _p(gp, _i64p), _p(mem, _i32p), float(omega_factor), _p(phi, _f64p))
    if rc != 0:
        raise ValueError(f"oracle jmjp failed ({rc})")
    return phi[: len(k)]


def rk4(csr: CSR, rho0, times):
    """rho(t_i) by fourth-order Runge-Kutta (Method #4, Eqs. RKstep and
    RKintermediate): ascending times, each interval split into
    ceil(interval x max_n |a_nn|) equal steps (h <= 1 / max_n |a_nn|).

    Returns (out[ntimes, n], info) with info = {"max_exit", "steps"} (steps:
    cumulative step counts per time, in the caller's order)."""
    rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
    times = np.ascontiguousarray(np.atleast_1d(times), dtype=np.float64)
    nt = len(times)
    out = np.zeros((nt, csr.n))
    steps = np.zeros(max(nt, 1), np.int64)
    maxe = ctypes.c_double()
    rc = _lib().orc_rk4(csr.n, _p(csr.row_ptr, _i64p), _p(csr.col, _i32p), _p(csr.val, _f64p),
                        _p(rho0, _f64p), _p(times, _f64p), nt, _p(out, _f64p), _p(steps, _i64p),
                        ctypes.byref(maxe))
    if rc != 0:
        raise ValueError(f"oracle rk4 failed ({rc})")
    return out, {"max_exit": maxe.value, "steps": steps[:nt].copy()}


def krylov(csr: CSR, rho0, times, kappa: int = 20):
    """rho(t_i) by Krylov steps (Method #5: Algorithm 3 with the full
    projection of Eq. Krylov_projection, Eq. Krylov_expansion): ascending
    times, each interval split into ceil(interval x max_n |a_nn| / (2 kappa))
    equal steps.  Returns (out[ntimes, n], {"max_exit", "steps"})."""
    rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
    times = np.ascontiguousarray(np.atleast_1d(times), dtype=np.float64)
    nt = len(times)
    out = np.zeros((nt, csr.n))
    steps = np.zeros(max(nt, 1), np.int64)
    maxe = ctypes.c_double()
    rc = _lib().orc_krylov(csr.n, _p(csr.row_ptr, _i64p), _p(csr.col, _i32p), _p(csr.val, _f64p),
                           _p(rho0, _f64p), _p(times, _f64p), nt, int(kappa), _p(out, _f64p), _p(steps, _i64p),
                           ctypes.byref(maxe))
    if rc != 0:
        raise ValueError(f"oracle krylov failed ({rc})")
    return out, {"max_exit": maxe.value, "steps": steps[:nt].copy()}


def expm(A) -> np.ndarray:
    """Dense exp(A): degree-13 Pade with scaling and squaring (Higham 2005)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    E = np.zeros_like(A)
    rc = _lib().orc_expm_pade13(A.shape[0], _p(A, _f64p), _p(E, _f64p))
    if rc != 0:
        raise ValueError("expm failed")
    return E


def gillespie(csr: CSR, s0: int, times, nruns: int, seed: int) -> np.ndarray:
    """State histogram at each time from nruns Gillespie trajectories."""
    times = np.ascontiguousarray(times, dtype=np.float64)
    counts = np.zeros((len(times), csr.n), np.int64)
    rc = _lib().orc_gillespie(csr.n, _p(csr.row_ptr, _i64p), _p(csr.col, _i32p), _p(csr.val, _f64p),
                              int(s0), _p(times, _f64p), len(times), int(nruns),
                              ctypes.c_uint64(seed & (2**64 - 1)), _p(counts, _i64p))
    if rc != 0:
        raise ValueError("gillespie failed")
    return counts


def loglik_from_rho(rho_t: np.ndarray, obs) -> float:
    """Snapshot log-likelihood sum_i sum_g c_{i,g} log(sum_{s in g} rho(T^i)_s).

    ``obs`` is a list over times of (members_list, counts): members_list[g] is
    the array of state indices whose probabilities are summed (the hidden gene
    state of Sec. 3.1.2 is marginalised this way), counts[g] how many
    observations fell in group g.  An observed group of probability zero gives
    -inf (the sampler then rejects)."""
    total = 0.0
    for i, (members, counts) in enumerate(obs):
        for mem, c in zip(members, counts):
            a = float(np.sum(rho_t[i, np.asarray(mem, dtype=np.int64)]))
            if c == 0:
                continue
            total += float(c) * (np.log(a) if a > 0 else -np.inf)
    return total


def loglik(csr: CSR, rho0, times, obs, mode: int = PAPER) -> float:
    rho_t, _ = expv(csr, rho0, times, mode=mode)
    return loglik_from_rho(rho_t, obs)


def log_prior(psi, mu: float = 1.0, sigma: float = 1e5) -> float:
    """log p(Psi), Eq. prior: independent Normal(mu, sigma) on each log-rate."""
    psi = np.asarray(psi, dtype=np.float64)
    return float(np.sum(-0.5 * ((psi - mu) / sigma) ** 2 - np.log(sigma * np.sqrt(2.0 * np.pi))))
