// api.cu -- the C ABI declared in include/mjp.h: handles, argument checks,
// workspace and the launch sequence planner -> chain.  Every numerical step
// runs in the library's kernels; this file only marshals.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "host_util.h"
#include "internal.cuh"

using namespace mjp;

namespace mjp {
std::string& last_error() {
  static thread_local std::string msg;
  return msg;
}
}  // namespace mjp

namespace {

bool finite_nonneg(const double* v, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (!(v[i] >= 0.0) || !std::isfinite(v[i])) return false;
  return true;
}

int ntheta_of(int kind) {
  switch (kind) {
    case MJP_BD1D: return 2;
    case MJP_TWOSTATE: return 4;
    case MJP_MRNA_PROT2D: return 4;
    case MJP_AUTOREG: return 6;
    default: return 0;
  }
}

}  // namespace

struct mjp_model {
  int kind = 0;
  int precision = MJP_FP32;
  int64_t N = 0, M = 0, P = 1;
  std::vector<double> theta;
  // options
  int renorm = kDefectPeriod;  // MJP_OPT_RENORM_PERIOD
  int64_t kcap = (int64_t)1 << 26;
  int threads = 0;
  int chain = 0;  // MJP_OPT_CHAIN
  int method = 0;  // MJP_OPT_METHOD
  int kappa = 20;  // MJP_OPT_KAPPA
  DevBuf d_kq;     // Krylov basis scratch
  DevBuf d_jk, d_jorder, d_jgp, d_jmem, d_jphi, d_jchunk;  // J-MJP observations
  DevBuf d_jmap;                                  // loglik: cluster -> theta, longest chain first
  int cluster = 0;
  int profile = 0;
  bool timed = false;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  // general CSR: B^T in SELL-32 form over states renumbered by in-degree
  double csr_omega = 0.0;
  int64_t nslices = 0;
  DevBuf d_slice_ptr, d_slice_len, d_col, d_val, d_diag, d_perm;
  DevBuf d_bar;                            // grid barrier of the one-launch CSR chain
  long long wait_limit = (long long)1 << 24;  // MJP_OPT_WAIT_LIMIT
  // workspace (scratch owned by the handle)
  DevBuf d_times, d_orig, d_win, d_info, d_theta, d_comp, d_status, d_ll;
  DevBuf d_rho2, d_outp, d_wtab, d_woff, d_L, d_K;
  // Poisson-weight arena filled by the planner (elements of the model precision)
  DevBuf d_arena, d_arena_ctl;
  int64_t arena_cap = 0;
  bool arena_grow = false;
  bool arena_fixed = false;  // capacity set by MJP_OPT_ARENA (never grown)
  ~mjp_model() {
    d_arena.release(); d_arena_ctl.release();
    d_slice_ptr.release(); d_slice_len.release(); d_col.release(); d_val.release(); d_diag.release();
    d_perm.release(); d_rho2.release(); d_outp.release(); d_wtab.release(); d_woff.release(); d_bar.release();
    d_L.release(); d_K.release();
    d_kq.release(); d_jk.release(); d_jorder.release(); d_jgp.release(); d_jmem.release(); d_jphi.release(); d_jchunk.release();
    d_jmap.release();
    d_times.release(); d_orig.release(); d_win.release(); d_info.release();
    d_theta.release(); d_comp.release(); d_status.release(); d_ll.release();
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
  }
};

struct mjp_obs {
  int64_t n = 0;
  int ntimes = 0;
  int G = 0;
  int nmem = 0;
  int maxmem = 0;  // most members in one group
  std::vector<double> times;  // ascending (host copy)
  std::vector<int32_t> members;  // host copy (groups in ascending time order)
  DevBuf d_times, d_gptr, d_counts, d_mptr, d_members, d_rho64, d_rho32;
  ~mjp_obs() {
    d_times.release(); d_gptr.release(); d_counts.release(); d_mptr.release();
    d_members.release(); d_rho64.release(); d_rho32.release();
  }
};

namespace {

int ensure_status(mjp_model* m) {
  if (m->d_status.p) return MJP_OK;
  int rc = m->d_status.ensure(sizeof(int));
  if (rc) return rc;
  MJP_CUDA(cudaMemset(m->d_status.p, 0, sizeof(int)));
  return MJP_OK;
}

// Pick cluster size and threads for a stencil chain of this model.
int stencil_config(mjp_model* m, int loglik_mode, int nt, int G, int nmem, int* cluster, int* threads,
                   int64_t* slab) {
  const size_t kSmemMax = 227 * 1024;
  int C = m->cluster;
  auto smem_of = [&](int c) {
    return chain_stencil_smem(m->kind, m->precision, loglik_mode, m->M, m->P,
                              chain_stencil_slab(m->kind, m->M, m->P, c), nt, G, nmem);
  };
  if (C <= 0) {
    C = 0;
    for (int c = 1; c <= 16; c *= 2) {
      if (smem_of(c) <= kSmemMax) {
        C = c;
        break;
      }
    }
    if (C == 0) return fail(MJP_ERR_UNSUPPORTED, "state space too large for an on-chip stencil chain");
  }
  if (C != 1 && C != 2 && C != 4 && C != 8 && C != 16) return fail(MJP_ERR_ARG, "cluster must be 1, 2, 4, 8 or 16");
  int64_t s = chain_stencil_slab(m->kind, m->M, m->P, C);
  size_t smem = smem_of(C);
  if (smem > kSmemMax) return fail(MJP_ERR_UNSUPPORTED, "slab does not fit shared memory; raise the cluster size");
  int t = m->threads;
  if (t <= 0) {
    // One thread per column when a row fits the CTA, ~8+ states per thread,
    // plus one warp that forms the Poisson weights.
    // Two-dimensional models: runs of about 20 pair-rows per thread measured
    // best on GB300 (fewer threads hide less latency, more add overhead).
    int64_t W = (m->kind == MJP_BD1D) ? s : m->M;
    int64_t rows = (m->kind == MJP_BD1D) ? 1 : s / m->M;
    int64_t want;
    if (W >= 992) want = 992;
    else {
      int64_t pair_rows = (rows + 1) / 2;
      int64_t groups = std::max<int64_t>(1, std::min<int64_t>((pair_rows + 19) / 20, 992 / W));
      want = W * groups;
    }
    want = (want + 31) / 32 * 32 + 32;
    t = (int)std::min<int64_t>(1024, std::max<int64_t>(64, want));
  }
  if (t % 32 != 0 || t < 64 || t > 1024) return fail(MJP_ERR_ARG, "threads must be a multiple of 32 in [64, 1024]");
  // Two-dimensional models give each stencil thread one column.
  if (m->kind != MJP_BD1D && m->M > t - 32) {
    if (m->M > 992) return fail(MJP_ERR_UNSUPPORTED, "rows longer than 992 states are not supported");
    return fail(MJP_ERR_ARG, "threads - 32 must be >= the row length M");
  }
  int nclusters = chain_stencil_max_cluster_blocks(m->kind, m->precision, loglik_mode, C, t, smem);
  if (nclusters <= 0) return fail(MJP_ERR_UNSUPPORTED, "stencil chain configuration cannot be made resident");
  *cluster = C;
  *threads = t;
  *slab = s;
  return MJP_OK;
}

// Record profiling event i (0: before the planner, 1: before the chain,
// 2: after the chain) when MJP_OPT_PROFILE is on.
int mark(mjp_model* m, int i, cudaStream_t s) {
  if (!m->profile) return MJP_OK;
  if (!m->ev[i]) MJP_CUDA(cudaEventCreate(&m->ev[i]));
  MJP_CUDA(cudaEventRecord(m->ev[i], s));
  if (i == 2) m->timed = true;
  return MJP_OK;
}

int map_status(int st);

// Closed-form upper bound of max_n e_n for a stencil model (sizes the arena).
double omega_bound(const mjp_model* m, const double* th) {
  switch (m->kind) {
    case MJP_BD1D: return 1.1 * (th[0] + th[1] * (double)(m->M - 1));
    case MJP_TWOSTATE: return 1.1 * (th[0] + th[1] * (double)(m->M - 1) + th[2] + th[3]);
    case MJP_MRNA_PROT2D:
      return 1.1 * (th[0] + (th[1] + th[2]) * (double)(m->M - 1) + th[3] * (double)(m->P - 1));
    case MJP_AUTOREG:  // Sec. 3.1.3's bound with each decay rate in its place (P = 2 N_P tile rows)
      return 1.1 * (th[0] + (th[1] + th[2]) * (double)(m->M - 1) + (th[3] + th[5]) * (double)(m->P / 2 - 1) + th[4]);
    default: return 0.0;
  }
}

// Make room in the weight arena for B instances at the given times: windows
// hold at most 16 sqrt(x) + 3 weights (x = Omega t).  The thetas are the
// call's when they are on the host, else the model's (the arena then grows
// after a call that reported overflow).  Fills the arena fields of pp.
int arena_prepare(mjp_model* m, const double* host_theta, int B, const double* times, int nt, cudaStream_t s,
                  PlanParams& pp) {
  const int ntheta = (int)m->theta.size();
  double need = 0.0;
  for (int b = 0; b < B; ++b) {
    const double* th = host_theta ? host_theta + (int64_t)b * ntheta : m->theta.data();
    const double om = omega_bound(m, th) * (host_theta ? 1.0 : 1.5);
    for (int i = 0; i < nt; ++i) need += 16.0 * std::sqrt(om * times[i]) + 3.0;
  }
  int64_t want = (int64_t)std::min(need, 2.0e9);
  if (m->arena_grow) want = std::max<int64_t>(want, 2 * m->arena_cap);
  m->arena_grow = false;
  if (want > m->arena_cap && !m->arena_fixed) {
    const size_t elt = m->precision == MJP_FP64 ? 8 : 4;
    int rc = m->d_arena.ensure(elt * (size_t)want);
    if (rc) return rc;
    m->arena_cap = want;
  }
  int rc = m->d_arena_ctl.ensure(16);
  if (rc) return rc;
  MJP_CUDA(cudaMemsetAsync(m->d_arena_ctl.p, 0, 16, s));
  pp.arena = m->d_arena.p;
  pp.arena_cap = m->arena_cap;
  pp.arena_used = m->d_arena_ctl.as<unsigned long long>();
  pp.arena_over = reinterpret_cast<int*>(m->d_arena_ctl.as<char>() + 8);
  pp.arena_fp64 = m->precision == MJP_FP64 ? 1 : 0;
  pp.fp64_weights = pp.arena_fp64;
  return MJP_OK;
}

// The general-CSR chain: planner, windows back to the host (the number of
// launches is the largest K), weight table, rho0 into the in-degree order,
// then one launch per jump.  Leaves the outputs (times in ascending order,
// states in the internal order) in m->d_outp.
int csr_run(mjp_model* m, const void* rho0, const double* sorted_times, int nt, int trunc_mode, double tol,
            cudaStream_t s, std::vector<Win>* wins) {
  const size_t elt = m->precision == MJP_FP64 ? 8 : 4;
  const int64_t n = m->N;
  int rc = 0;
  if ((rc = ensure_status(m)) || (rc = m->d_times.ensure(sizeof(double) * nt)) ||
      (rc = m->d_win.ensure(sizeof(Win) * nt)) || (rc = m->d_info.ensure(sizeof(JobInfo))) ||
      (rc = m->d_rho2.ensure(2 * elt * n)) || (rc = m->d_outp.ensure(elt * (size_t)nt * n)) ||
      (rc = m->d_woff.ensure(sizeof(int64_t) * nt)) || (rc = m->d_L.ensure(sizeof(int64_t) * nt)) ||
      (rc = m->d_K.ensure(sizeof(int64_t) * nt)))
    return rc;
  if (m->precision == MJP_FP32 && (rc = m->d_comp.ensure(sizeof(float) * (size_t)nt * n))) return rc;
  MJP_CUDA(cudaMemcpyAsync(m->d_times.p, sorted_times, sizeof(double) * nt, cudaMemcpyHostToDevice, s));
  PlanParams pp = {};
  pp.kind = MJP_CSR; pp.M = 1; pp.P = 1; pp.N = n; pp.ntheta = 0; pp.theta = nullptr; pp.B = 1;
  pp.ntimes = nt; pp.times = m->d_times.as<double>();
  pp.trunc_mode = trunc_mode; pp.tol = tol; pp.omega_factor = 1.1; pp.omega_fixed = m->csr_omega;
  pp.fp64_weights = m->precision == MJP_FP64 ? 1 : 0;
  pp.kcap = m->kcap; pp.win = m->d_win.as<Win>(); pp.info = m->d_info.as<JobInfo>();
  pp.status = m->d_status.as<int>();
  if ((rc = mark(m, 0, s))) return rc;
  MJP_CUDA(launch_plan(pp, s));
  wins->resize(nt);
  MJP_CUDA(cudaMemcpyAsync(wins->data(), m->d_win.p, sizeof(Win) * nt, cudaMemcpyDeviceToHost, s));
  MJP_CUDA(cudaStreamSynchronize(s));
  int st = 0;
  MJP_CUDA(cudaMemcpy(&st, m->d_status.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (st) {
    MJP_CUDA(cudaMemset(m->d_status.p, 0, sizeof(int)));
    return map_status(st);
  }
  std::vector<int64_t> woff(nt), L(nt), K(nt);
  int64_t tot = 0, kmax = 0;
  for (int i = 0; i < nt; ++i) {
    woff[i] = tot;
    L[i] = (*wins)[i].L;
    K[i] = (*wins)[i].K;
    tot += K[i] - L[i] + 1;
    kmax = std::max(kmax, K[i]);
  }
  if ((rc = m->d_wtab.ensure(sizeof(double) * std::max<int64_t>(tot, 1)))) return rc;
  MJP_CUDA(cudaMemcpyAsync(m->d_woff.p, woff.data(), sizeof(int64_t) * nt, cudaMemcpyHostToDevice, s));
  MJP_CUDA(cudaMemcpyAsync(m->d_L.p, L.data(), sizeof(int64_t) * nt, cudaMemcpyHostToDevice, s));
  MJP_CUDA(cudaMemcpyAsync(m->d_K.p, K.data(), sizeof(int64_t) * nt, cudaMemcpyHostToDevice, s));
  MJP_CUDA(launch_fill_weights(m->d_win.as<Win>(), nt, m->d_woff.as<int64_t>(), m->d_wtab.as<double>(), s));
  char* rho = m->d_rho2.as<char>();
  MJP_CUDA(launch_permute_in(m->precision, rho0, m->d_perm.as<int32_t>(), rho, n, s));
  if ((rc = mark(m, 1, s))) return rc;
  CsrJumpParams jp = {};
  jp.n = n; jp.nslices = m->nslices;
  jp.slice_ptr = m->d_slice_ptr.as<int64_t>(); jp.slice_len = m->d_slice_len.as<int32_t>();
  jp.col = m->d_col.as<int32_t>(); jp.val = m->d_val.p; jp.diag = m->d_diag.p;
  jp.wtab = m->d_wtab.as<double>(); jp.woff = m->d_woff.as<int64_t>();
  jp.L = m->d_L.as<int64_t>(); jp.K = m->d_K.as<int64_t>();
  jp.out = m->d_outp.p; jp.comp = m->d_comp.as<float>();
  if (m->chain == 2) {
    // The whole chain in one cooperative launch, jumps separated by a
    // bounded grid barrier (a wait that runs out is reported by
    // rate_model_check as MJP_ERR_DEVICE_TIMEOUT).  Measured slower than
    // one launch per jump at N = 2^20 (12.6 against 11.4 ms for 309 jumps,
    // FP32): the barrier costs more than the gap between launches.
    if ((rc = m->d_bar.ensure(2 * sizeof(unsigned)))) return rc;
    MJP_CUDA(cudaMemsetAsync(m->d_bar.p, 0, 2 * sizeof(unsigned), s));
    CsrChainParams cp = {};
    cp.j = jp;
    cp.ntimes = nt;
    cp.kmax = kmax;
    cp.rho = rho;
    cp.bar = m->d_bar.as<unsigned>();
    cp.wait_limit = m->wait_limit;
    cp.status = m->d_status.as<int>();
    MJP_CUDA(launch_csr_chain(m->precision, cp, s));
  } else {
    int lo = 0, hi = -1;  // times whose window holds jump k-1 (ascending times)
    for (int64_t k = 1; k <= kmax + 1; ++k) {
      const int64_t kp = k - 1;
      while (lo < nt && K[lo] < kp) ++lo;
      while (hi + 1 < nt && L[hi + 1] <= kp) ++hi;
      jp.k = k;
      jp.jump = k <= kmax;
      jp.tlo = lo;
      jp.thi = hi;
      jp.rho_prev = rho + ((kp & 1) ? elt * n : 0);
      jp.rho_next = rho + ((kp & 1) ? 0 : elt * n);
      MJP_CUDA(launch_csr_jump(m->precision, jp, s));
    }
  }
  if ((rc = mark(m, 2, s))) return rc;
  return MJP_OK;
}

int map_status(int st) {
  switch (st) {
    case kStatusOk: return MJP_OK;
    case kStatusKcap: return fail(MJP_ERR_KCAP, "truncation index K above the cap");
    case kStatusNumeric: return fail(MJP_ERR_NUMERIC, "non-finite or negative probability");
    case kStatusTimeout: return fail(MJP_ERR_DEVICE_TIMEOUT, "a bounded device wait ran out");
    default: return fail(MJP_ERR_ARG, "device rejected an argument");
  }
}

}  // namespace

extern "C" {

const char* mjp_last_error(void) { return mjp::last_error().c_str(); }

const char* mjp_version(void) { return "mjp-gb300 0.1 (sm_103a)"; }

int rate_model_create_stencil(mjp_model** out, int kind, const int64_t* dims, int ndims,
                              const double* theta, int ntheta, int precision) try {
  if (!out) return fail(MJP_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (kind != MJP_BD1D && kind != MJP_TWOSTATE && kind != MJP_MRNA_PROT2D && kind != MJP_AUTOREG)
    return fail(MJP_ERR_ARG, "unknown stencil kind");
  if (precision != MJP_FP32 && precision != MJP_FP64) return fail(MJP_ERR_ARG, "precision must be MJP_FP32 or MJP_FP64");
  if (!dims || !theta) return fail(MJP_ERR_ARG, "dims/theta is NULL");
  if (ntheta != ntheta_of(kind)) return fail(MJP_ERR_ARG, "wrong number of parameters for this kind");
  if (!finite_nonneg(theta, ntheta)) return fail(MJP_ERR_ARG, "rates must be finite and >= 0");
  auto* m = new mjp_model();
  m->kind = kind;
  m->precision = precision;
  m->theta.assign(theta, theta + ntheta);
  if (kind == MJP_BD1D) {
    if (ndims != 1 || dims[0] < 1) { delete m; return fail(MJP_ERR_ARG, "BD1D needs dims = {N}, N >= 1"); }
    m->M = dims[0]; m->P = 1; m->N = dims[0];
  } else if (kind == MJP_TWOSTATE) {
    if (ndims != 1 || dims[0] < 2) { delete m; return fail(MJP_ERR_ARG, "TWOSTATE needs dims = {N_R}, N_R >= 2"); }
    m->M = dims[0]; m->P = 2; m->N = 2 * dims[0];
  } else if (kind == MJP_AUTOREG) {
    if (ndims != 2 || dims[0] < 2 || dims[1] < 2) { delete m; return fail(MJP_ERR_ARG, "AUTOREG needs dims = {N_R >= 2, N_P >= 2}"); }
    m->M = dims[0]; m->P = 2 * dims[1]; m->N = 2 * dims[0] * dims[1];
  } else {
    if (ndims != 2 || dims[0] < 2 || dims[1] < 1) { delete m; return fail(MJP_ERR_ARG, "MRNA_PROT2D needs dims = {M >= 2, P >= 1}"); }
    m->M = dims[0]; m->P = dims[1]; m->N = dims[0] * dims[1];
  }
  if (m->N > ((int64_t)1 << 31) - 1) { delete m; return fail(MJP_ERR_ARG, "too many states"); }
  *out = m;
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

int rate_model_create_csr(mjp_model** out, int64_t n, const int64_t* row_ptr, const int32_t* col,
                          const double* rate, int precision) try {
  if (!out) return fail(MJP_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || n > ((int64_t)1 << 31) - 1) return fail(MJP_ERR_ARG, "n out of range");
  if (!row_ptr || !col || !rate) return fail(MJP_ERR_ARG, "NULL CSR array");
  if (precision != MJP_FP32 && precision != MJP_FP64) return fail(MJP_ERR_ARG, "precision must be MJP_FP32 or MJP_FP64");
  if (row_ptr[0] != 0) return fail(MJP_ERR_CSR, "row_ptr[0] must be 0");
  for (int64_t i = 0; i < n; ++i)
    if (row_ptr[i + 1] < row_ptr[i]) return fail(MJP_ERR_CSR, "row_ptr is not monotone");
  const int64_t nnz = row_ptr[n];
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j) {
      if (col[j] < 0 || col[j] >= n) return fail(MJP_ERR_CSR, "column index out of range");
      if (col[j] == i) return fail(MJP_ERR_CSR, "diagonal entries are not rates (lambda_nn = 0)");
      if (!(rate[j] >= 0.0) || !std::isfinite(rate[j])) return fail(MJP_ERR_CSR, "rates must be finite and >= 0");
    }
  // Exit rates e_n = sum_m lambda_nm, each row summed in ascending column order.
  std::vector<int64_t> ord(nnz);
  std::vector<double> e(n, 0.0);
  std::vector<int64_t> indeg(n, 0);
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j) ord[j] = j;
    std::stable_sort(ord.begin() + row_ptr[i], ord.begin() + row_ptr[i + 1],
                     [&](int64_t a, int64_t b) { return col[a] < col[b]; });
    double acc = 0.0;
    for (int64_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j) {
      acc = acc + rate[ord[j]];
      indeg[col[ord[j]]] += 1;
    }
    e[i] = acc;
  }
  double maxe = 0.0;
  for (int64_t i = 0; i < n; ++i) maxe = e[i] > maxe ? e[i] : maxe;
  volatile double factor = 1.1;  // Omega = 1.1 max_n |a_nn| with one rounding
  const double omega = maxe > 0.0 ? factor * maxe : 0.0;
  // Renumber states by decreasing in-degree; slices of 32 states.
  std::vector<int32_t> iperm(n), perm(n);
  for (int64_t i = 0; i < n; ++i) iperm[i] = (int32_t)i;
  std::stable_sort(iperm.begin(), iperm.end(), [&](int32_t a, int32_t b) { return indeg[a] > indeg[b]; });
  for (int64_t q = 0; q < n; ++q) perm[iperm[q]] = (int32_t)q;
  const int64_t nslices = (n + 31) / 32;
  std::vector<int32_t> slen(nslices, 0);
  std::vector<int64_t> sptr(nslices + 1, 0);
  for (int64_t s0 = 0; s0 < nslices; ++s0) {
    int64_t w = 0;
    for (int64_t l = 0; l < 32 && s0 * 32 + l < n; ++l) w = std::max(w, indeg[iperm[s0 * 32 + l]]);
    slen[s0] = (int32_t)w;
    sptr[s0 + 1] = sptr[s0] + w * 32;
  }
  const int64_t npad = sptr[nslices];
  std::vector<int32_t> ecol(npad);
  std::vector<double> eval(npad, 0.0);
  for (int64_t q = 0; q < n; ++q) {  // padding: self index, weight 0
    int64_t s0 = q / 32, l = q % 32;
    for (int64_t j = 0; j < slen[s0]; ++j) ecol[sptr[s0] + j * 32 + l] = (int32_t)q;
  }
  std::vector<int32_t> fill(n, 0);
  for (int64_t i = 0; i < n; ++i)  // incoming entries in ascending source order
    for (int64_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j) {
      const int64_t t = col[ord[j]];
      const int64_t q = perm[t], s0 = q / 32, l = q % 32;
      const int64_t slot = sptr[s0] + (int64_t)fill[t]++ * 32 + l;
      ecol[slot] = perm[i];
      eval[slot] = omega > 0.0 ? rate[ord[j]] / omega : 0.0;
    }
  std::vector<double> diag(n);
  for (int64_t q = 0; q < n; ++q) diag[q] = omega > 0.0 ? 1.0 - e[iperm[q]] / omega : 1.0;

  auto* m = new mjp_model();
  m->kind = MJP_CSR;
  m->precision = precision;
  m->N = n; m->M = n; m->P = 1;
  m->csr_omega = omega;
  m->nslices = nslices;
  const size_t elt = precision == MJP_FP64 ? 8 : 4;
  int rc = 0;
  if ((rc = m->d_slice_ptr.ensure(sizeof(int64_t) * nslices)) || (rc = m->d_slice_len.ensure(sizeof(int32_t) * nslices)) ||
      (rc = m->d_col.ensure(sizeof(int32_t) * std::max<int64_t>(npad, 1))) ||
      (rc = m->d_val.ensure(elt * std::max<int64_t>(npad, 1))) || (rc = m->d_diag.ensure(elt * n)) ||
      (rc = m->d_perm.ensure(sizeof(int32_t) * n))) {
    delete m;
    return rc;
  }
  auto up = [](DevBuf& b, const void* src, size_t bytes) { return cudaMemcpy(b.p, src, bytes, cudaMemcpyHostToDevice); };
  cudaError_t ce = cudaSuccess;
  if (precision == MJP_FP64) {
    ce = up(m->d_val, eval.data(), 8 * npad);
    if (ce == cudaSuccess) ce = up(m->d_diag, diag.data(), 8 * n);
  } else {
    std::vector<float> v32(eval.begin(), eval.end()), d32(diag.begin(), diag.end());
    ce = up(m->d_val, v32.data(), 4 * npad);
    if (ce == cudaSuccess) ce = up(m->d_diag, d32.data(), 4 * n);
  }
  if (ce == cudaSuccess) ce = up(m->d_slice_ptr, sptr.data(), sizeof(int64_t) * nslices);
  if (ce == cudaSuccess) ce = up(m->d_slice_len, slen.data(), sizeof(int32_t) * nslices);
  if (ce == cudaSuccess && npad > 0) ce = up(m->d_col, ecol.data(), sizeof(int32_t) * npad);
  if (ce == cudaSuccess) ce = up(m->d_perm, perm.data(), sizeof(int32_t) * n);
  if (ce != cudaSuccess) {
    cudaGetLastError();
    delete m;
    return fail(MJP_ERR_CUDA, std::string("uploading the CSR model failed: ") + cudaGetErrorString(ce));
  }
  *out = m;
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

int rate_model_set_theta(mjp_model* m, const double* theta, int ntheta) try {
  if (!m || !theta) return fail(MJP_ERR_ARG, "NULL argument");
  if (m->kind == MJP_CSR) return fail(MJP_ERR_ARG, "CSR models have no theta");
  if (ntheta != ntheta_of(m->kind)) return fail(MJP_ERR_ARG, "wrong number of parameters");
  if (!finite_nonneg(theta, ntheta)) return fail(MJP_ERR_ARG, "rates must be finite and >= 0");
  m->theta.assign(theta, theta + ntheta);
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

int rate_model_set_option(mjp_model* m, int option, int64_t value) try {
  if (!m) return fail(MJP_ERR_ARG, "NULL model");
  switch (option) {
    case MJP_OPT_RENORM_PERIOD:
      if (value < 0 || value > (1 << 20) || value % 8 != 0)
        return fail(MJP_ERR_ARG, "renorm period must be 0 or a multiple of 8 in [8, 2^20]");
      m->renorm = (int)value;
      return MJP_OK;
    case MJP_OPT_K_CAP:
      if (value < 1 || value > ((int64_t)1 << 40)) return fail(MJP_ERR_ARG, "K cap must be in [1, 2^40]");
      m->kcap = value;
      return MJP_OK;
    case MJP_OPT_THREADS:
      if (value != 0 && (value % 32 != 0 || value < 64 || value > 1024)) return fail(MJP_ERR_ARG, "threads must be 0 or a multiple of 32 in [64, 1024]");
      m->threads = (int)value;
      return MJP_OK;
    case MJP_OPT_CHAIN:
      if (value < 0 || value > 2) return fail(MJP_ERR_ARG, "chain must be 0, 1 or 2");
      m->chain = (int)value;
      return MJP_OK;
    case MJP_OPT_METHOD:
      if (value < 0 || value > 2) return fail(MJP_ERR_ARG, "method must be 0 (R-MJP), 1 (RK4) or 2 (Krylov)");
      m->method = (int)value;
      return MJP_OK;
    case MJP_OPT_KAPPA:
      if (value < 1 || value > krylov_max_kappa()) return fail(MJP_ERR_ARG, "kappa must be in [1, 32]");
      m->kappa = (int)value;
      return MJP_OK;
    case MJP_OPT_ARENA:
      if (value < 0) return fail(MJP_ERR_ARG, "arena capacity must be >= 0");
      m->d_arena.release();
      m->arena_cap = 0;
      if (value > 0) {
        int rc = m->d_arena.ensure((m->precision == MJP_FP64 ? 8 : 4) * (size_t)value);
        if (rc) return rc;
        m->arena_cap = value;
        m->arena_fixed = true;
      } else {
        m->arena_fixed = false;
      }
      return MJP_OK;
    case MJP_OPT_PROFILE:
      if (value != 0 && value != 1) return fail(MJP_ERR_ARG, "profile must be 0 or 1");
      m->profile = (int)value;
      m->timed = false;
      return MJP_OK;
    case MJP_OPT_CLUSTER:
      if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8 && value != 16) return fail(MJP_ERR_ARG, "cluster must be 0, 1, 2, 4, 8 or 16");
      m->cluster = (int)value;
      return MJP_OK;
    case MJP_OPT_WAIT_LIMIT:
      if (value < 0) return fail(MJP_ERR_ARG, "wait limit must be >= 0");
      m->wait_limit = (long long)value;
      return MJP_OK;
    default:
      return fail(MJP_ERR_ARG, "unknown option");
  }
} catch (...) {
  return ::mjp::exception_status();
}

int64_t rate_model_num_states(const mjp_model* m) { return m ? m->N : -1; }

void rate_model_destroy(mjp_model* m) { delete m; }

int rate_model_last_timing(mjp_model* m, double* ms_plan, double* ms_chain) try {
  if (!m) return fail(MJP_ERR_ARG, "NULL model");
  if (!m->profile || !m->timed) return fail(MJP_ERR_ARG, "no profiled call (set MJP_OPT_PROFILE first)");
  MJP_CUDA(cudaEventSynchronize(m->ev[2]));
  float a = 0.f, b = 0.f;
  MJP_CUDA(cudaEventElapsedTime(&a, m->ev[0], m->ev[1]));
  MJP_CUDA(cudaEventElapsedTime(&b, m->ev[1], m->ev[2]));
  if (ms_plan) *ms_plan = a;
  if (ms_chain) *ms_chain = b;
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

int rate_model_check(mjp_model* m, void* stream) try {
  if (!m) return fail(MJP_ERR_ARG, "NULL model");
  MJP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  if (m->d_arena_ctl.p) {  // windows that did not fit ran the in-kernel recurrence: grow
    int over = 0;
    MJP_CUDA(cudaMemcpy(&over, m->d_arena_ctl.as<char>() + 8, sizeof(int), cudaMemcpyDeviceToHost));
    if (over) m->arena_grow = true;
  }
  if (!m->d_status.p) return MJP_OK;
  int st = 0;
  MJP_CUDA(cudaMemcpy(&st, m->d_status.p, sizeof(int), cudaMemcpyDeviceToHost));
  MJP_CUDA(cudaMemset(m->d_status.p, 0, sizeof(int)));
  return map_status(st);
} catch (...) {
  return ::mjp::exception_status();
}

// expv_series by fourth-order Runge-Kutta (Method #4) or Krylov steps
// (Method #5), Sec. 2.3: ascending times, each interval split into
// ceil(interval x max_n |a_nn| / D) equal steps, D = 1 (RK4) or 2 kappa
// (Krylov); max_n |a_nn| summed per row in the rate matrix's order (death,
// then birth).
int expv_ode(mjp_model* m, const void* rho0, const std::vector<double>& st, const std::vector<int32_t>& order,
             void* out, mjp_series_info* info, cudaStream_t s) {
  const bool kry = m->method == 2;
  if ((m->kind != MJP_BD1D && m->kind != MJP_TWOSTATE) || m->precision != MJP_FP64)
    return fail(MJP_ERR_UNSUPPORTED, "RK4 and Krylov steps are available for FP64 birth-death and two-state models");
  if (m->N > (kry ? (int64_t)krylov_max_states() : rk4_max_states()))
    return fail(MJP_ERR_UNSUPPORTED, "RK4 and Krylov steps hold at most 4096 states");
  const int nt = (int)st.size();
  const double* th = m->theta.data();
  // max_n |a_nn|, each row summed in ascending target order.
  double maxe = 0.0;
  for (int64_t n = 0; n < m->N; ++n) {
    double e = 0.0;
    if (m->kind == MJP_BD1D) {
      if (n >= 1) e = e + th[1] * (double)n;
      if (n + 1 < m->N) e = e + th[0];
    } else {
      const int64_t sg = n / m->M, r = n - sg * m->M;
      if (sg == 0) {
        if (r >= 1) e = e + th[1] * (double)r;
        if (r + 1 < m->M) e = e + th[0];
        e = e + th[3];
      } else {
        e = e + th[2];
        if (r >= 1) e = e + th[1] * (double)r;
      }
    }
    if (e > maxe) maxe = e;
  }
  const double div = kry ? 2.0 * m->kappa : 1.0;
  std::vector<int64_t> steps(nt);
  std::vector<double> h(nt);
  double tprev = 0.0;
  for (int q = 0; q < nt; ++q) {
    const double tau = st[q] - tprev;
    steps[q] = (maxe > 0.0 && tau > 0.0) ? (int64_t)std::ceil(kry ? tau * maxe / div : tau * maxe) : 0;
    h[q] = steps[q] > 0 ? tau / (double)steps[q] : 0.0;
    tprev = st[q];
  }
  int rc = 0;
  if ((rc = m->d_orig.ensure(sizeof(int32_t) * nt)) || (rc = m->d_K.ensure(sizeof(int64_t) * nt)) ||
      (rc = m->d_wtab.ensure(sizeof(double) * nt)) || (rc = m->d_theta.ensure(sizeof(double) * m->theta.size())) ||
      (rc = ensure_status(m)))
    return rc;
  if (kry && (rc = m->d_kq.ensure(sizeof(double) * (size_t)m->kappa * m->N))) return rc;
  MJP_CUDA(cudaMemcpyAsync(m->d_orig.p, order.data(), sizeof(int32_t) * nt, cudaMemcpyHostToDevice, s));
  MJP_CUDA(cudaMemcpyAsync(m->d_K.p, steps.data(), sizeof(int64_t) * nt, cudaMemcpyHostToDevice, s));
  MJP_CUDA(cudaMemcpyAsync(m->d_wtab.p, h.data(), sizeof(double) * nt, cudaMemcpyHostToDevice, s));
  MJP_CUDA(cudaMemcpyAsync(m->d_theta.p, m->theta.data(), sizeof(double) * m->theta.size(), cudaMemcpyHostToDevice, s));
  if ((rc = mark(m, 0, s)) || (rc = mark(m, 1, s))) return rc;
  if (kry) {
    KrylovParams kp = {};
    kp.theta = m->d_theta.as<double>();
    kp.kind = m->kind;
    kp.N = (int)m->N;
    kp.M = (int)m->M;
    kp.rho0 = reinterpret_cast<const double*>(rho0);
    kp.out = reinterpret_cast<double*>(out);
    kp.orig = m->d_orig.as<int32_t>();
    kp.steps = m->d_K.as<int64_t>();
    kp.hstep = m->d_wtab.as<double>();
    kp.ntimes = nt;
    kp.kappa = m->kappa;
    kp.maxe = maxe;
    kp.Q = m->d_kq.as<double>();
    kp.status = m->d_status.as<int>();
    MJP_CUDA(launch_krylov(kp, s));
  } else {
    Rk4Params rp = {};
    rp.theta = m->d_theta.as<double>();
    rp.kind = m->kind;
    rp.N = (int)m->N;
    rp.M = (int)m->M;
    rp.rho0 = reinterpret_cast<const double*>(rho0);
    rp.out = reinterpret_cast<double*>(out);
    rp.orig = m->d_orig.as<int32_t>();
    rp.steps = m->d_K.as<int64_t>();
    rp.hstep = m->d_wtab.as<double>();
    rp.ntimes = nt;
    MJP_CUDA(launch_rk4(rp, s));
  }
  if ((rc = mark(m, 2, s))) return rc;
  // The host arrays above are pageable: the copies have been staged before
  // cudaMemcpyAsync returned, so they may go out of scope now.
  if (info) {
    MJP_CUDA(cudaStreamSynchronize(s));
    info->omega = maxe;
    int64_t total = 0;
    for (int q = 0; q < nt; ++q) {
      total += steps[q];
      if (info->K) info->K[order[q]] = total;
      if (info->eps) info->eps[order[q]] = 0.0;
    }
    return rate_model_check(m, (void*)s);
  }
  return MJP_OK;
}

int expv_series(mjp_model* m, const void* rho0, const double* times, int ntimes, void* out,
                mjp_series_info* info, int trunc_mode, double tol, void* stream) try {
  if (!m || !rho0 || !times || !out) return fail(MJP_ERR_ARG, "NULL argument");
  if (ntimes < 1 || ntimes > kMaxTimes) return fail(MJP_ERR_ARG, "ntimes must be in [1, 256]");
  if (trunc_mode != MJP_TRUNC_PAPER && trunc_mode != MJP_TRUNC_TOL) return fail(MJP_ERR_ARG, "unknown truncation mode");
  if (trunc_mode == MJP_TRUNC_TOL && !(tol >= 1e-20 && tol < 0.5)) return fail(MJP_ERR_ARG, "tol must be in [1e-20, 0.5)");
  for (int i = 0; i < ntimes; ++i)
    if (!(times[i] >= 0.0) || !std::isfinite(times[i])) return fail(MJP_ERR_ARG, "times must be finite and >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  const int nt = ntimes;
  std::vector<int32_t> order(nt);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return times[a] < times[b]; });
  std::vector<double> st(nt);
  for (int i = 0; i < nt; ++i) st[i] = times[order[i]];
  if (m->method != 0) return expv_ode(m, rho0, st, order, out, info, s);
  if (m->kind == MJP_CSR) {
    std::vector<Win> w;
    int rc = csr_run(m, rho0, st.data(), nt, trunc_mode, tol, s, &w);
    if (rc) return rc;
    if ((rc = m->d_orig.ensure(sizeof(int32_t) * nt))) return rc;
    MJP_CUDA(cudaMemcpyAsync(m->d_orig.p, order.data(), sizeof(int32_t) * nt, cudaMemcpyHostToDevice, s));
    MJP_CUDA(launch_permute_out(m->precision, m->d_outp.p, m->d_perm.as<int32_t>(), out, m->N, nt,
                                m->d_orig.as<int32_t>(), s));
    if (info) {
      info->omega = m->csr_omega;
      for (int i = 0; i < nt; ++i) {
        if (info->K) info->K[order[i]] = w[i].K;
        if (info->eps) info->eps[order[i]] = w[i].tail;
      }
      return rate_model_check(m, stream);
    }
    return MJP_OK;
  }

  // Birth-death chains: the register-resident kernel (one CTA, or the fewest
  // CTAs of a cluster that hold the chain, halo 32) unless a thread count is
  // asked for.
  Reg1dPlan rp1 = {};
  bool use_reg1 = false;
  if (m->kind == MJP_BD1D && m->chain != 1 && m->threads == 0) {
    const int c0 = m->cluster > 0 ? m->cluster : 1, c1 = m->cluster > 0 ? m->cluster : 8;
    for (int c = c0; c <= c1 && !use_reg1; ++c) use_reg1 = chain_reg1d_plan(m->precision, m->N, nt, c, 32, &rp1, true);
  }
  if (m->chain == 2 && m->kind == MJP_BD1D && !use_reg1)
    return fail(MJP_ERR_UNSUPPORTED, "the register-resident expv chain needs a birth-death model without "
                                     "a forced thread count that fits 8 CTAs");
  int C = 0, T = 0;
  int64_t slab = 0;
  int rc = 0;
  if (!use_reg1 && (rc = stencil_config(m, 0, nt, 0, 0, &C, &T, &slab))) return rc;
  if ((rc = ensure_status(m))) return rc;
  if ((rc = m->d_times.ensure(sizeof(double) * nt))) return rc;
  if ((rc = m->d_orig.ensure(sizeof(int32_t) * nt))) return rc;
  if ((rc = m->d_win.ensure(sizeof(Win) * nt))) return rc;
  if ((rc = m->d_info.ensure(sizeof(JobInfo)))) return rc;
  if ((rc = m->d_theta.ensure(sizeof(double) * m->theta.size()))) return rc;
  if (!use_reg1 && m->precision == MJP_FP32 && (rc = m->d_comp.ensure(sizeof(float) * (size_t)nt * m->N))) return rc;
  MJP_CUDA(cudaMemcpyAsync(m->d_times.p, st.data(), sizeof(double) * nt, cudaMemcpyHostToDevice, s));
  MJP_CUDA(cudaMemcpyAsync(m->d_orig.p, order.data(), sizeof(int32_t) * nt, cudaMemcpyHostToDevice, s));
  MJP_CUDA(cudaMemcpyAsync(m->d_theta.p, m->theta.data(), sizeof(double) * m->theta.size(), cudaMemcpyHostToDevice, s));

  PlanParams pp = {};
  pp.kind = m->kind; pp.M = (int32_t)m->M; pp.P = (int32_t)m->P; pp.N = m->N;
  pp.ntheta = (int)m->theta.size(); pp.theta = m->d_theta.as<double>(); pp.B = 1;
  pp.ntimes = nt; pp.times = m->d_times.as<double>();
  pp.trunc_mode = trunc_mode; pp.tol = tol; pp.omega_factor = 1.1; pp.omega_fixed = -1.0;
  pp.kcap = m->kcap; pp.win = m->d_win.as<Win>(); pp.info = m->d_info.as<JobInfo>();
  pp.status = m->d_status.as<int>();
  if ((rc = arena_prepare(m, m->theta.data(), 1, st.data(), nt, s, pp))) return rc;
  if ((rc = mark(m, 0, s))) return rc;
  MJP_CUDA(launch_plan(pp, s));
  if ((rc = mark(m, 1, s))) return rc;

  ChainParams cp = {};
  cp.arena = pp.arena;
  cp.M = (int32_t)m->M; cp.P = (int32_t)m->P; cp.N = m->N;
  cp.ntheta = pp.ntheta; cp.theta = pp.theta; cp.B = 1; cp.ntimes = nt;
  cp.orig = m->d_orig.as<int32_t>(); cp.win = pp.win; cp.info = pp.info; cp.rho0 = rho0;
  cp.out = out; cp.out_stride = 0; cp.comp = m->d_comp.as<float>(); cp.comp_stride = 0;
  cp.renorm = (m->precision == MJP_FP32) ? m->renorm : 0;
  cp.slab = slab; cp.status = pp.status;
  if (use_reg1) MJP_CUDA(launch_chain_reg1d(m->precision, cp, rp1, s));
  else MJP_CUDA(launch_chain_stencil(m->kind, m->precision, 0, cp, C, T, s));
  if ((rc = mark(m, 2, s))) return rc;

  if (info) {
    std::vector<Win> w(nt);
    JobInfo ji;
    MJP_CUDA(cudaMemcpyAsync(w.data(), m->d_win.p, sizeof(Win) * nt, cudaMemcpyDeviceToHost, s));
    MJP_CUDA(cudaMemcpyAsync(&ji, m->d_info.p, sizeof(JobInfo), cudaMemcpyDeviceToHost, s));
    MJP_CUDA(cudaStreamSynchronize(s));
    info->omega = ji.omega;
    for (int i = 0; i < nt; ++i) {
      if (info->K) info->K[order[i]] = w[i].K;
      if (info->eps) info->eps[order[i]] = w[i].tail;
    }
    return rate_model_check(m, stream);
  }
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

int jmjp_state_probs(mjp_model* m, const void* rho0, int64_t nobs, const int64_t* k, const int64_t* group_ptr,
                     const int32_t* members, double* phi, void* stream) try {
  if (!m || !rho0 || !k || !group_ptr || !members || !phi) return fail(MJP_ERR_ARG, "NULL argument");
  if (m->kind != MJP_BD1D && m->kind != MJP_TWOSTATE)
    return fail(MJP_ERR_UNSUPPORTED, "J-MJP probabilities are available for birth-death and two-state models");
  if (m->N > jmjp_max_states(m->precision)) return fail(MJP_ERR_UNSUPPORTED, "state space too large for one CTA");
  if (nobs < 1 || nobs > ((int64_t)1 << 31) - 1) return fail(MJP_ERR_ARG, "nobs out of range");
  if (group_ptr[0] != 0) return fail(MJP_ERR_ARG, "group_ptr[0] must be 0");
  for (int64_t i = 0; i < nobs; ++i) {
    if (k[i] < 0) return fail(MJP_ERR_ARG, "jump counts must be >= 0");
    if (group_ptr[i + 1] <= group_ptr[i]) return fail(MJP_ERR_ARG, "every group needs a member");
  }
  const int64_t nmem = group_ptr[nobs];
  for (int64_t q = 0; q < nmem; ++q)
    if (members[q] < 0 || members[q] >= m->N) return fail(MJP_ERR_ARG, "member state out of range");
  cudaStream_t s = (cudaStream_t)stream;
  // Omega = 1.1 max_n |a_nn| (Eq. B_def), each row summed in target order.
  const double* th = m->theta.data();
  double maxe = 0.0;
  for (int64_t n = 0; n < m->N; ++n) {
    double e = 0.0;
    if (m->kind == MJP_BD1D) {
      if (n >= 1) e = e + th[1] * (double)n;
      if (n + 1 < m->N) e = e + th[0];
    } else {
      const int64_t sg = n / m->M, r = n - sg * m->M;
      if (sg == 0) {
        if (r >= 1) e = e + th[1] * (double)r;
        if (r + 1 < m->M) e = e + th[0];
        e = e + th[3];
      } else {
        e = e + th[2];
        if (r >= 1) e = e + th[1] * (double)r;
      }
    }
    if (e > maxe) maxe = e;
  }
  // Observations sorted by jump count (stable), groups in that order.
  for (int64_t i = 0; i < nobs; ++i)
    if (k[i] > INT32_MAX - 1) return fail(MJP_ERR_UNSUPPORTED, "jump counts must be below 2^31 - 1");
  if (nmem > INT32_MAX) return fail(MJP_ERR_ARG, "too many members");
  std::vector<int32_t> order(nobs);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return k[a] < k[b]; });
  std::vector<int32_t> ks(nobs), gp(nobs + 1, 0);
  std::vector<int32_t> mem((size_t)nmem);
  for (int64_t o = 0; o < nobs; ++o) {
    const int32_t i = order[o];
    ks[o] = (int32_t)k[i];
    const int64_t c = group_ptr[i + 1] - group_ptr[i];
    std::copy(members + group_ptr[i], members + group_ptr[i + 1], mem.begin() + gp[o]);
    gp[o + 1] = gp[o] + (int32_t)c;
  }
  // Chunks of sorted observations that fit the shared memory beside the chain:
  // 12 bytes per observation (k, position, group offset) + 4 per member, the
  // space split by the mean group size.
  const size_t avail = jmjp_chunk_bytes(m->precision, (int)m->N);
  const double mbar = (double)nmem / (double)nobs;
  int64_t cap_obs = (int64_t)((double)(avail - 4) / (12.0 + 4.0 * mbar));
  cap_obs = std::max<int64_t>(1, std::min<int64_t>(cap_obs, nobs));
  const int64_t cap_mem = ((int64_t)avail - 4 - 12 * cap_obs) / 4;
  std::vector<int32_t> chunk(1, 0);
  for (int64_t o = 0; o < nobs;) {
    const int64_t s0 = o;
    int64_t used = 0;
    while (o < nobs && o - s0 < cap_obs && used + (gp[o + 1] - gp[o]) <= cap_mem) used += gp[o + 1] - gp[o], ++o;
    if (o == s0) return fail(MJP_ERR_UNSUPPORTED, "an observation group does not fit shared memory");
    chunk.push_back((int32_t)o);
  }
  const int nchunks = (int)chunk.size() - 1;
  int rc = 0;
  if ((rc = m->d_jk.ensure(sizeof(int32_t) * nobs)) || (rc = m->d_jorder.ensure(sizeof(int32_t) * nobs)) ||
      (rc = m->d_jgp.ensure(sizeof(int32_t) * (nobs + 1))) || (rc = m->d_jmem.ensure(sizeof(int32_t) * nmem)) ||
      (rc = m->d_jphi.ensure(sizeof(double) * nobs)) || (rc = m->d_jchunk.ensure(sizeof(int32_t) * chunk.size())) ||
      (rc = m->d_theta.ensure(sizeof(double) * m->theta.size())))
    return rc;
  MJP_CUDA(cudaMemcpyAsync(m->d_jk.p, ks.data(), sizeof(int32_t) * nobs, cudaMemcpyHostToDevice, s));
  MJP_CUDA(cudaMemcpyAsync(m->d_jorder.p, order.data(), sizeof(int32_t) * nobs, cudaMemcpyHostToDevice, s));
  MJP_CUDA(cudaMemcpyAsync(m->d_jgp.p, gp.data(), sizeof(int32_t) * (nobs + 1), cudaMemcpyHostToDevice, s));
  MJP_CUDA(cudaMemcpyAsync(m->d_jmem.p, mem.data(), sizeof(int32_t) * nmem, cudaMemcpyHostToDevice, s));
  MJP_CUDA(cudaMemcpyAsync(m->d_jchunk.p, chunk.data(), sizeof(int32_t) * chunk.size(), cudaMemcpyHostToDevice, s));
  MJP_CUDA(cudaMemcpyAsync(m->d_theta.p, m->theta.data(), sizeof(double) * m->theta.size(), cudaMemcpyHostToDevice, s));
  JmjpParams jp = {};
  jp.theta = m->d_theta.as<double>();
  jp.N = (int)m->N;
  jp.M = (int)m->M;
  jp.rho0 = rho0;
  jp.nobs = (int)nobs;
  jp.ksorted = m->d_jk.as<int32_t>();
  jp.order = m->d_jorder.as<int32_t>();
  jp.group_ptr = m->d_jgp.as<int32_t>();
  jp.members = m->d_jmem.as<int32_t>();
  jp.phi = m->d_jphi.as<double>();
  jp.omega = 1.1 * maxe;
  jp.nchunks = nchunks;
  jp.chunk = m->d_jchunk.as<int32_t>();
  jp.cap_obs = (int)cap_obs;
  jp.cap_mem = (int)cap_mem;
  jp.kmax = ks[nobs - 1];
  if ((rc = mark(m, 0, s)) || (rc = mark(m, 1, s))) return rc;
  MJP_CUDA(launch_jmjp(m->kind, m->precision, jp, s));
  if ((rc = mark(m, 2, s))) return rc;
  MJP_CUDA(cudaMemcpyAsync(phi, jp.phi, sizeof(double) * nobs, cudaMemcpyDeviceToHost, s));
  MJP_CUDA(cudaStreamSynchronize(s));
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

int mjp_obs_create(mjp_obs** out, int64_t n, int ntimes, const double* times,
                   const int64_t* group_ptr, const double* counts, const int64_t* member_ptr,
                   const int32_t* members, const double* rho0) try {
  if (!out) return fail(MJP_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || ntimes < 1 || ntimes > kMaxTimes) return fail(MJP_ERR_ARG, "bad n or ntimes");
  if (!times || !group_ptr || !counts || !member_ptr || !members || !rho0) return fail(MJP_ERR_ARG, "NULL argument");
  if (group_ptr[0] != 0) return fail(MJP_ERR_ARG, "group_ptr[0] must be 0");
  for (int i = 0; i < ntimes; ++i) {
    if (group_ptr[i + 1] < group_ptr[i]) return fail(MJP_ERR_ARG, "group_ptr not monotone");
    if (!(times[i] >= 0.0) || !std::isfinite(times[i])) return fail(MJP_ERR_ARG, "times must be finite and >= 0");
  }
  const int64_t G = group_ptr[ntimes];
  if (G > kMaxGroups) return fail(MJP_ERR_ARG, "too many observation groups (limit 8192)");
  if (member_ptr[0] != 0) return fail(MJP_ERR_ARG, "member_ptr[0] must be 0");
  for (int64_t g = 0; g < G; ++g) {
    if (member_ptr[g + 1] < member_ptr[g]) return fail(MJP_ERR_ARG, "member_ptr not monotone");
    if (!(counts[g] >= 0.0) || !std::isfinite(counts[g])) return fail(MJP_ERR_ARG, "counts must be finite and >= 0");
  }
  const int64_t nm = member_ptr[G];
  for (int64_t q = 0; q < nm; ++q)
    if (members[q] < 0 || members[q] >= n) return fail(MJP_ERR_ARG, "member state out of range");
  if (!finite_nonneg(rho0, n)) return fail(MJP_ERR_ARG, "rho0 must be finite and >= 0");

  // Reorder times ascending (groups follow their time).
  std::vector<int> order(ntimes);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return times[a] < times[b]; });
  std::vector<double> st(ntimes), cnt;
  std::vector<int64_t> gp(ntimes + 1, 0), mp(1, 0);
  std::vector<int32_t> mem;
  for (int ii = 0; ii < ntimes; ++ii) {
    int i = order[ii];
    st[ii] = times[i];
    for (int64_t g = group_ptr[i]; g < group_ptr[i + 1]; ++g) {
      cnt.push_back(counts[g]);
      for (int64_t q = member_ptr[g]; q < member_ptr[g + 1]; ++q) mem.push_back(members[q]);
      mp.push_back((int64_t)mem.size());
    }
    gp[ii + 1] = (int64_t)cnt.size();
  }
  if (mem.empty()) mem.push_back(0);
  if (cnt.empty()) cnt.push_back(0.0);
  std::vector<float> r32(n);
  for (int64_t i = 0; i < n; ++i) r32[i] = (float)rho0[i];

  auto* o = new mjp_obs();
  o->n = n;
  o->ntimes = ntimes;
  o->G = (int)G;
  o->nmem = (int)(mp.back());
  for (size_t g = 0; g + 1 < mp.size(); ++g) o->maxmem = std::max<int>(o->maxmem, (int)(mp[g + 1] - mp[g]));
  o->times = st;
  o->members = mem;
  int rc = 0;
  if ((rc = o->d_times.ensure(sizeof(double) * ntimes)) || (rc = o->d_gptr.ensure(sizeof(int64_t) * gp.size())) ||
      (rc = o->d_counts.ensure(sizeof(double) * cnt.size())) || (rc = o->d_mptr.ensure(sizeof(int64_t) * mp.size())) ||
      (rc = o->d_members.ensure(sizeof(int32_t) * mem.size())) || (rc = o->d_rho64.ensure(sizeof(double) * n)) ||
      (rc = o->d_rho32.ensure(sizeof(float) * n))) {
    delete o;
    return rc;
  }
  auto up = [](DevBuf& b, const void* src, size_t bytes) { return cudaMemcpy(b.p, src, bytes, cudaMemcpyHostToDevice); };
  if (up(o->d_times, st.data(), sizeof(double) * ntimes) != cudaSuccess ||
      up(o->d_gptr, gp.data(), sizeof(int64_t) * gp.size()) != cudaSuccess ||
      up(o->d_counts, cnt.data(), sizeof(double) * cnt.size()) != cudaSuccess ||
      up(o->d_mptr, mp.data(), sizeof(int64_t) * mp.size()) != cudaSuccess ||
      up(o->d_members, mem.data(), sizeof(int32_t) * mem.size()) != cudaSuccess ||
      up(o->d_rho64, rho0, sizeof(double) * n) != cudaSuccess ||
      up(o->d_rho32, r32.data(), sizeof(float) * n) != cudaSuccess) {
    cudaGetLastError();
    delete o;
    return fail(MJP_ERR_CUDA, "copying observations to the device failed");
  }
  *out = o;
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

void mjp_obs_destroy(mjp_obs* obs) { delete obs; }

int loglik(mjp_model* m, const mjp_obs* obs, const double* theta, int B, double* out, int where,
           int trunc_mode, double tol, void* stream) try {
  if (!m || !obs || !out) return fail(MJP_ERR_ARG, "NULL argument");
  if (B < 1) return fail(MJP_ERR_ARG, "B must be >= 1");
  if (where != MJP_PTR_HOST && where != MJP_PTR_DEVICE) return fail(MJP_ERR_ARG, "where must be MJP_PTR_HOST or MJP_PTR_DEVICE");
  if (obs->n != m->N) return fail(MJP_ERR_ARG, "observations were built for a different state space");
  if (trunc_mode != MJP_TRUNC_PAPER && trunc_mode != MJP_TRUNC_TOL) return fail(MJP_ERR_ARG, "unknown truncation mode");
  if (trunc_mode == MJP_TRUNC_TOL && !(tol >= 1e-20 && tol < 0.5)) return fail(MJP_ERR_ARG, "tol must be in [1e-20, 0.5)");
  if (m->kind == MJP_CSR) {
    // A CSR model has fixed rates: one instance, theta ignored.
    if (B != 1) return fail(MJP_ERR_ARG, "CSR models evaluate one instance (B = 1)");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<Win> w;
    const void* r0 = (m->precision == MJP_FP64) ? obs->d_rho64.p : obs->d_rho32.p;
    int rc = csr_run(m, r0, obs->times.data(), obs->ntimes, trunc_mode, tol, s, &w);
    if (rc) return rc;
    double* d_out = out;
    if (where == MJP_PTR_HOST) {
      if ((rc = m->d_ll.ensure(sizeof(double)))) return rc;
      d_out = m->d_ll.as<double>();
    }
    MJP_CUDA(launch_csr_loglik(m->d_outp.p, m->precision, m->N, obs->d_gptr.as<int64_t>(), obs->ntimes,
                               obs->d_counts.as<double>(), obs->d_mptr.as<int64_t>(), obs->d_members.as<int32_t>(),
                               m->d_perm.as<int32_t>(), d_out, m->d_status.as<int>(), s));
    if (where == MJP_PTR_HOST) {
      MJP_CUDA(cudaMemcpyAsync(out, d_out, sizeof(double), cudaMemcpyDeviceToHost, s));
      return rate_model_check(m, stream);
    }
    return MJP_OK;
  }
  if (!theta) return fail(MJP_ERR_ARG, "theta is NULL");
  const int ntheta = ntheta_of(m->kind);
  if (where == MJP_PTR_HOST)
    for (int b = 0; b < B; ++b)
      if (!finite_nonneg(theta + (int64_t)b * ntheta, ntheta)) return fail(MJP_ERR_ARG, "rates must be finite and >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  const int nt = obs->ntimes;
  int C = 0, T = 0;
  int64_t slab = 0;
  // The chain keeps a generic member list only for groups of > 2 members.
  const int nmem_list = obs->maxmem > 2 ? obs->nmem : 0;
  // Register-resident chain: FP32 mRNA/protein boxes, no forced launch shape.
  RegPlan rp = {};
  bool use_reg = false;
  if (m->chain != 1 && m->kind == MJP_MRNA_PROT2D && m->precision == MJP_FP32 &&
      (m->chain == 2 || (m->cluster == 0 && m->threads == 0)))
    use_reg = chain_reg2d_plan(m->M, m->P, nt, obs->nmem, 8, m->threads, &rp);
  // Register-resident two-state chain: FP32, groups of at most two members,
  // no forced cluster size (a thread count picks its warps).
  RegTsPlan tp = {};
  bool use_ts = false;
  if (m->chain != 1 && m->kind == MJP_TWOSTATE && m->precision == MJP_FP32 && m->cluster == 0) {
    int col_lo = -1, col_hi = -1;  // columns (n_R) of the observed states
    if (obs->G > 0)
      for (int32_t sidx : obs->members) {
        const int c = (int)(sidx % m->M);
        col_lo = col_lo < 0 ? c : std::min(col_lo, c);
        col_hi = std::max(col_hi, c);
      }
    use_ts = chain_regts_plan(m->M, nt, obs->G, obs->maxmem, col_lo, col_hi, m->threads, &tp);
  }
  if (m->chain == 2 && !use_reg && !use_ts)
    return fail(MJP_ERR_UNSUPPORTED, "the register-resident chain needs an FP32 mRNA/protein box that fits 8 "
                                     "CTAs, at the automatic thread count or 256, or an FP32 two-state model whose "
                                     "groups have at most two members and that fits one CTA");
  int rc = 0;
  if (!use_reg && !use_ts && (rc = stencil_config(m, 1, nt, obs->G, nmem_list, &C, &T, &slab))) return rc;
  if ((rc = ensure_status(m))) return rc;
  if ((rc = m->d_win.ensure(sizeof(Win) * (size_t)nt * B))) return rc;
  if ((rc = m->d_info.ensure(sizeof(JobInfo) * (size_t)B))) return rc;
  if ((rc = m->d_jmap.ensure(sizeof(int32_t) * (size_t)B))) return rc;
  const double* d_theta = theta;
  double* d_out = out;
  if (where == MJP_PTR_HOST) {
    if ((rc = m->d_theta.ensure(sizeof(double) * (size_t)B * ntheta))) return rc;
    if ((rc = m->d_ll.ensure(sizeof(double) * (size_t)B))) return rc;
    MJP_CUDA(cudaMemcpyAsync(m->d_theta.p, theta, sizeof(double) * (size_t)B * ntheta, cudaMemcpyHostToDevice, s));
    d_theta = m->d_theta.as<double>();
    d_out = m->d_ll.as<double>();
  }
  PlanParams pp = {};
  pp.kind = m->kind; pp.M = (int32_t)m->M; pp.P = (int32_t)m->P; pp.N = m->N;
  pp.ntheta = ntheta; pp.theta = d_theta; pp.B = B;
  pp.ntimes = nt; pp.times = obs->d_times.as<double>();
  pp.trunc_mode = trunc_mode; pp.tol = tol; pp.omega_factor = 1.1; pp.omega_fixed = -1.0;
  pp.kcap = m->kcap; pp.win = m->d_win.as<Win>(); pp.info = m->d_info.as<JobInfo>();
  pp.status = m->d_status.as<int>();
  if ((rc = arena_prepare(m, where == MJP_PTR_HOST ? theta : nullptr, B, obs->times.data(), nt, s, pp))) return rc;
  if ((rc = mark(m, 0, s))) return rc;
  MJP_CUDA(launch_plan(pp, s));
  // Chains of different theta differ in length (K grows with Omega): start
  // the longest first so the last wave of clusters holds the short ones.  The
  // ranking compares all pairs, so batches above kOrderMax keep launch order.
  constexpr int kOrderMax = 8192;
  const bool ordered = B > 1 && B <= kOrderMax;
  if (ordered) MJP_CUDA(launch_order_jobs(pp.info, B, m->d_jmap.as<int32_t>(), s));
  if ((rc = mark(m, 1, s))) return rc;

  ChainParams cp = {};
  cp.arena = pp.arena;
  cp.M = (int32_t)m->M; cp.P = (int32_t)m->P; cp.N = m->N;
  cp.ntheta = ntheta; cp.theta = d_theta; cp.B = B; cp.ntimes = nt;
  cp.orig = nullptr; cp.win = pp.win; cp.info = pp.info;
  cp.rho0 = (m->precision == MJP_FP64) ? obs->d_rho64.p : obs->d_rho32.p;
  cp.gptr = obs->d_gptr.as<int64_t>(); cp.counts = obs->d_counts.as<double>();
  cp.mptr = obs->d_mptr.as<int64_t>(); cp.members = obs->d_members.as<int32_t>();
  cp.G = obs->G; cp.nmem = nmem_list; cp.ll = d_out; cp.wait_limit = m->wait_limit;
  cp.renorm = (m->precision == MJP_FP32) ? m->renorm : 0;
  cp.slab = slab; cp.status = pp.status;
  cp.job_map = ordered ? m->d_jmap.as<int32_t>() : nullptr;
  if (use_reg) MJP_CUDA(launch_chain_reg2d(cp, rp, s));
  else if (use_ts) MJP_CUDA(launch_chain_regts(cp, tp, s));
  else MJP_CUDA(launch_chain_stencil(m->kind, m->precision, 1, cp, C, T, s));
  if ((rc = mark(m, 2, s))) return rc;
  if (where == MJP_PTR_HOST) {
    MJP_CUDA(cudaMemcpyAsync(out, d_out, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
    return rate_model_check(m, stream);
  }
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

}  // extern "C"

// ---- internal accessors for the sampler (not part of the C ABI) -----------
namespace mjp {

int model_kind(const mjp_model* m) { return m->kind; }

// Wait for `s`, grow the weight arena if a window overflowed it, then return
// and clear the device status word (MJP_OK when nothing was flagged).  A
// sampler keeps going after a flagged evaluation: its result is NaN and the
// proposal is rejected.
int model_take_status(mjp_model* m, cudaStream_t s, int* status) {
  *status = 0;
  MJP_CUDA(cudaStreamSynchronize(s));
  if (m->d_arena_ctl.p) {
    int over = 0;
    MJP_CUDA(cudaMemcpy(&over, m->d_arena_ctl.as<char>() + 8, sizeof(int), cudaMemcpyDeviceToHost));
    if (over) m->arena_grow = true;
  }
  if (!m->d_status.p) return MJP_OK;
  MJP_CUDA(cudaMemcpy(status, m->d_status.p, sizeof(int), cudaMemcpyDeviceToHost));
  MJP_CUDA(cudaMemset(m->d_status.p, 0, sizeof(int)));
  return MJP_OK;
}

}  // namespace mjp
