// internal.cuh -- device-side structures shared by the library's CUDA files.
// Nothing here is visible through the C ABI (include/mjp.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mjp.h"

namespace mjp {

constexpr int kMaxTimes = 256;     // observation times per call
constexpr int kMaxGroups = 8192;   // observation groups per loglik call
constexpr int kMaxTheta = 8;

// Device status word bits (first error wins; read by rate_model_check).
enum DevStatus : int {
  kStatusOk = 0,
  kStatusKcap = 1,
  kStatusNumeric = 2,
  kStatusTimeout = 3,
  kStatusArg = 4,
};

// Truncation window of one (instance, time): Algorithm 2 for x = Omega t,
// with weights Poisson(k|x) for k in [L, K] generated in the chain kernel by
// the paper's recurrence P_k = P_{k-1} x / k, started from P_L (normalised,
// log-safe) instead of exp(-x), which underflows for x > 708.
struct Win {
  double x;     // Omega * t
  double PL;    // Poisson(L | x)
  double tail;  // epsilon = sum_{k > K} Poisson(k | x) = 1 - sum_{k <= K}
  int64_t L;    // first jump index with non-negligible weight (left mass < 1e-20)
  int64_t K;    // last jump index (Algorithm 2's loop exit)
};

struct JobInfo {
  double omega;  // 1.1 * max_n e_n (0 if all rates vanish)
  int64_t Kmax;  // max_i K_i
};

// Planner inputs: B instances that share model dimensions and times.
struct PlanParams {
  int kind;
  int32_t M, P;         // stencil dims (BD1D: M = N, P = 1; TWOSTATE: M = N_R, P = 2)
  int64_t N;
  int ntheta;
  const double* theta;  // device, B x ntheta
  int B;
  int ntimes;
  const double* times;  // device, ascending
  int trunc_mode;
  double tol;
  double omega_factor;
  double omega_fixed;   // > 0: use this Omega (CSR models, computed at creation)
  int64_t kcap;
  Win* win;             // device, B x ntimes
  JobInfo* info;        // device, B
  int* status;
};

// Chain inputs (stencil models).
struct ChainParams {
  int32_t M, P;
  int64_t N;
  int ntheta;
  const double* theta;     // device, B x ntheta
  int B;
  int ntimes;
  const int32_t* orig;     // device, sorted time i -> caller's row
  const Win* win;          // device, B x ntimes
  const JobInfo* info;     // device, B
  const void* rho0;        // device, N values (T), shared by all instances
  // expv
  void* out;               // device, per instance ntimes x N (T)
  int64_t out_stride;      // elements between instances
  float* comp;             // device scratch, FP32 Kahan compensation, ntimes x N per instance
  int64_t comp_stride;
  // loglik
  const int64_t* gptr;     // device, ntimes + 1 (times sorted)
  const double* counts;    // device, G
  const int64_t* mptr;     // device, G + 1
  const int32_t* members;  // device
  int G;
  int nmem;                // members in all groups
  double* ll;              // device, B
  int renorm;              // period in jumps (0 = off)
  int64_t slab;            // states per CTA of the cluster (whole rows for 2-D models)
  int* status;
};

}  // namespace mjp

// Host-side launchers implemented in the .cu files.
namespace mjp {
cudaError_t launch_plan(const PlanParams& p, cudaStream_t s);
cudaError_t launch_chain_stencil(int kind, int precision, int loglik_mode, const ChainParams& p,
                                 int cluster, int threads, cudaStream_t s);
int64_t chain_stencil_slab(int kind, int64_t M, int64_t P, int cluster);
size_t chain_stencil_smem(int kind, int precision, int loglik_mode, int64_t M, int64_t P, int64_t slab,
                          int ntimes, int G, int nmem);
int chain_stencil_max_cluster_blocks(int kind, int precision, int loglik_mode, int cluster,
                                     int threads, size_t smem);
}  // namespace mjp
