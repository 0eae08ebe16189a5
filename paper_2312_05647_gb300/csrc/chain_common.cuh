// chain_common.cuh -- device helpers shared by the jump-chain kernels
// (stencil.cu, stencil_reg.cu): status word, split cluster barrier, cp.async
// copies, scaled rate coefficients and fixed-order (uncontracted) arithmetic.
#pragma once

#include "internal.cuh"

namespace mjp {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ void set_status(int* st, int code) {
  if (st) atomicCAS(st, 0, code);
}

__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Arrive without ordering; callers order their writes first with a fence of
// the scope their readers need (fence_cta / fence_cluster).
__device__ __forceinline__ void cluster_arrive_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void fence_cta() { asm volatile("fence.acq_rel.cta;" ::: "memory"); }
__device__ __forceinline__ void fence_cluster() { asm volatile("fence.acq_rel.cluster;" ::: "memory"); }

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Row n of y = x A (Eq. A_def) for the FP64 comparison methods, matrix-free:
// y_n = (inflows in ascending source order) - x_n e_n, with e_n summed over
// row n in ascending target order.  Birth-death: inflow beta from n-1 and
// gamma (n+1) from n+1.  Two-state (n = n_R + sigma N_R, sigma 0 active):
// active states gain beta from n-1 (n_R >= 1), gamma (n_R+1) from n+1 and
// lambda_act from the inactive partner n + N_R; inactive states gain
// lambda_ina from the active partner n - N_R (a lower index, so it comes
// first) and gamma (n_R+1) from n+1.  Coefficients of missing sources are 0.
// The death coefficient gamma (n_R+1) and the exit rate are kept per state.
__device__ inline void rate_row_coef(int kind, int n, int N, int NR, const double* th, double& dn, double& ex) {
  dn = ex = 0.0;
  if (n < 0 || n >= N) return;
  if (kind == MJP_BD1D) {
    double e = 0.0;
    if (n >= 1) e = __dadd_rn(e, __dmul_rn(th[1], (double)n));
    if (n + 1 < N) e = __dadd_rn(e, th[0]);
    ex = e;
    dn = n + 1 < N ? __dmul_rn(th[1], (double)(n + 1)) : 0.0;
    return;
  }
  const int sg = n >= NR ? 1 : 0, r = n - sg * NR;
  dn = r + 1 < NR ? __dmul_rn(th[1], (double)(r + 1)) : 0.0;
  double e = 0.0;
  if (sg == 0) {
    if (r >= 1) e = __dadd_rn(e, __dmul_rn(th[1], (double)r));
    if (r + 1 < NR) e = __dadd_rn(e, th[0]);
    e = __dadd_rn(e, th[3]);
  } else {
    e = __dadd_rn(e, th[2]);
    if (r >= 1) e = __dadd_rn(e, __dmul_rn(th[1], (double)r));
  }
  ex = e;
}
// y_n from the staged vector X (N values); xn = x_n.
__device__ inline double rate_apply_row(int kind, int n, int N, int NR, const double* th, double dn, double ex,
                                        const double* X, double xn) {
  const double left = n >= 1 ? X[n - 1] : 0.0;
  const double right = n + 1 < N ? X[n + 1] : 0.0;
  if (kind == MJP_BD1D) {
    double t = __dmul_rn(left, th[0]);
    t = __dadd_rn(t, __dmul_rn(right, dn));
    return __dsub_rn(t, __dmul_rn(xn, ex));
  }
  const bool act = n < NR;
  double t;
  if (act) {
    t = __dmul_rn(left, n >= 1 ? th[0] : 0.0);
    t = __dadd_rn(t, __dmul_rn(right, dn));
    t = __dadd_rn(t, __dmul_rn(X[n + NR], th[2]));
  } else {
    t = __dmul_rn(X[n - NR], th[3]);
    t = __dadd_rn(t, __dmul_rn(right, dn));
  }
  return __dsub_rn(t, __dmul_rn(xn, ex));
}

// Asynchronous global -> shared copy of one float or double (cp.async).
__device__ __forceinline__ void cp_async_elem(float* sdst, const float* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_elem(double* sdst, const double* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Scaled rates (rate / Omega) of one instance in the chain type.
template <typename T>
struct Coef {
  T a, b, c, d, e, f;
};

template <typename T, int KIND>
__device__ __forceinline__ Coef<T> make_coef(const double* th, double omega) {
  Coef<T> k;
  double inv = omega > 0.0 ? 1.0 / omega : 0.0;
  k.a = (T)(th[0] * inv);
  k.b = (T)(th[1] * inv);
  k.c = (KIND == MJP_BD1D) ? (T)0 : (T)(th[2] * inv);
  k.d = (KIND == MJP_BD1D) ? (T)0 : (T)(th[3] * inv);
  k.e = (KIND == MJP_AUTOREG) ? (T)(th[4] * inv) : (T)0;
  k.f = (KIND == MJP_AUTOREG) ? (T)(th[5] * inv) : (T)0;
  return k;
}

// Fixed-order arithmetic (no contraction): every thread layout and cluster
// shape produces bit-identical chains.
__device__ __forceinline__ float f_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double f_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float f_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double f_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float f_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double f_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float f_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double f_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

// Pairs of chain values (two rows of one column).  FP32 pairs use the packed
// sm_100+ FP32x2 instructions; FP64 pairs are two scalar operations.
template <typename T> struct Pair;
template <> struct Pair<float> { using type = float2; };
template <> struct Pair<double> { using type = double2; };
__device__ __forceinline__ float2 v_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ double2 v_mul(double2 a, double2 b) {
  return make_double2(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y));
}
__device__ __forceinline__ float2 v_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ double2 v_add(double2 a, double2 b) {
  return make_double2(__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y));
}
__device__ __forceinline__ float2 v_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ double2 v_fma(double2 a, double2 b, double2 c) {
  return make_double2(__fma_rn(a.x, b.x, c.x), __fma_rn(a.y, b.y, c.y));
}
__device__ __forceinline__ float2 v_make(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 v_make(double a, double b) { return make_double2(a, b); }

// Compensated FP32 jump.  A chain stored in FP32 loses about half an ulp of
// every state at every jump, and over the tens of thousands of jumps of a
// slowly relaxing chain these roundings add up coherently (relative errors of
// 1e-4 at K ~ 7e4).  The compensated jump writes the update in delta form,
//   t = lo_n + sum_{m -> n} rho_m lambda_mn / Omega - (e_n / Omega) rho_n,
//   y = rho_n + t,   lo_n <- t - (y - rho_n),
// so each state carries the part of t that the addition rounded away (its
// residual lo_n) into the next jump instead of losing it.  The value of the
// chain is rho_n + lo_n; only rho_n is read by the neighbours and by the
// weighted sum (lo_n is below half an ulp of rho_n).
//
// Column sums of B are 1 (Eq. B_def) only in exact arithmetic: the exit
// coefficient e_n / Omega, rounded to FP32, differs from the sum of the
// rounded outflow coefficients the neighbours apply by a defect d_n of up to
// half an ulp, which creates or destroys mass at every jump.  Every
// kDefectPeriod jumps each state adds kDefectPeriod d_n rho_n to its residual
// (d_n formed exactly in FP64 from the FP32 coefficients), which restores the
// conservation of B to second order in the period.  Both corrections are
// local to a state, so every thread layout, cluster shape and halo gives
// bit-identical chains.  The period is MJP_OPT_RENORM_PERIOD (default
// kDefectPeriod, a multiple of every register kernel's round length).

__device__ __forceinline__ float comp_finish(float cur, float t, float& lo) {
  const float y = __fadd_rn(cur, t);
  lo = __fsub_rn(t, __fsub_rn(y, cur));
  return y;
}
__device__ __forceinline__ float2 comp_finish(float2 cur, float2 t, float2& lo) {
  const float2 m1 = make_float2(-1.0f, -1.0f);
  const float2 y = __fadd2_rn(cur, t);
  lo = __ffma2_rn(__ffma2_rn(cur, m1, y), m1, t);  // t - (y - cur), each step exact as in comp_finish(float)
  return y;
}
// One compensated birth-death jump of a pair: inflows from the left (birth)
// and right (death), then the exit ne = -e_n / Omega.
__device__ __forceinline__ float2 comp_jump(float2 cur, float2& lo, float2 cl, float2 left, float2 cr, float2 right,
                                            float2 ne) {
  float2 t = __ffma2_rn(cl, left, lo);
  t = __ffma2_rn(cr, right, t);
  t = __ffma2_rn(ne, cur, t);
  return comp_finish(cur, t, lo);
}
__device__ __forceinline__ float comp_jump(float cur, float& lo, float cl, float left, float cr, float right,
                                           float ne) {
  float t = __fmaf_rn(cl, left, lo);
  t = __fmaf_rn(cr, right, t);
  t = __fmaf_rn(ne, cur, t);
  return comp_finish(cur, t, lo);
}

// Exit defects (exit coefficient minus the outflow coefficients that the
// neighbours apply) of the models whose FP32 chains run in more than one
// kernel; every kernel forms them with these functions, so the corrections
// agree to the bit.
//
// Birth-death state n: exit fl(fl(gamma n) + beta'), outflows beta' (to n+1,
// absent at N-1) and fl(gamma n) (to n-1); the defect is the rounding error
// of one addition, exact in FP64 and in FP32.
template <typename T>
__device__ __forceinline__ float bd_defect(const Coef<T>& co, int n, int N) {
  const float bn = __fmul_rn((float)co.b, (float)n);
  const float ain = n + 1 < N ? (float)co.a : 0.0f;
  const float e = __fadd_rn(bn, ain);
  return (float)(((double)e - (double)bn) - (double)ain);
}
// Two-state state (column m, row sigma): the active row (sigma = 0) exits by
// birth beta' (absent at m = N_R - 1), death fl(gamma m) and deactivation
// lambda_ina, summed as fl(fl(fl(gamma m) + beta') + lambda_ina); the inactive
// row by activation and death, fl(lambda_act + fl(gamma m)).  The defect is
// that exit minus its outflows, formed in FP64 and rounded.
template <typename T>
__device__ __forceinline__ float ts_defect(const Coef<T>& co, int row, int m, int M) {
  const float bm = __fmul_rn((float)co.b, (float)m);
  const float ain = m + 1 < M ? (float)co.a : 0.0f;
  if (row == 0) {
    const float e = __fadd_rn(__fadd_rn(bm, ain), (float)co.d);
    return (float)((((double)e - (double)bm) - (double)ain) - (double)co.d);
  }
  const float e = __fadd_rn((float)co.c, bm);
  return (float)(((double)e - (double)co.c) - (double)bm);
}
// mRNA/protein column m: e0 = fl(fl(fl(gamma_m m) + k_m') + fl(k_p m)) (k_m'
// = k_m below the last column), the exit without the protein decay, and its
// column defect e0 - (its three outflows), formed in FP64 and rounded.
struct MrnaCol {
  float e0, eps;
};
template <typename T>
__device__ __forceinline__ MrnaCol mrna_col(const Coef<T>& co, int m, int M) {
  const float bm = __fmul_rn((float)co.b, (float)m);
  const float ain = m + 1 < M ? (float)co.a : 0.0f;
  const float cd = __fmul_rn((float)co.c, (float)m);
  MrnaCol r;
  r.e0 = __fadd_rn(__fadd_rn(bm, ain), cd);
  r.eps = (float)((((double)r.e0 - (double)bm) - (double)ain) - (double)cd);
  return r;
}
// Defect of state (m, p): the chain's exit is e = fl(e0 + gamma_p p) (one
// fused multiply-add) and the outflow to p-1 is fl(gamma_p p); the row part
// e - e0 - fl(gamma_p p) is formed exactly (both subtractions are of numbers
// within a factor of two of each other), then added to the column part.  In
// row P-1 the exit adds k_p m back as a separate term and the outflow to p+1
// is absent, so the same defect holds there.
__device__ __forceinline__ float mrna_defect(const MrnaCol& col, float gp, int p) {
  const float fp = (float)p;
  const float e = __fmaf_rn(gp, fp, col.e0);
  const float dpf = __fmul_rn(gp, fp);
  const float row = dpf >= col.e0 ? __fsub_rn(__fsub_rn(e, dpf), col.e0) : __fsub_rn(__fsub_rn(e, col.e0), dpf);
  return __fadd_rn(col.eps, row);
}

}  // namespace
}  // namespace mjp
