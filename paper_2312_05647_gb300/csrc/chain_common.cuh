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

}  // namespace
}  // namespace mjp
