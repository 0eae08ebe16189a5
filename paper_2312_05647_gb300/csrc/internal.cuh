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
constexpr int kWeightLead = 4;   // jumps the weight prefetch runs ahead
constexpr int kWeightRing = 6;   // ring slots (> lead + 1)
// Default period (jumps) of the exit-defect correction of the compensated
// FP32 chain (MJP_OPT_RENORM_PERIOD; chain_common.cuh).
constexpr int kDefectPeriod = 32;

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
  double x;      // Omega * t
  double PL;     // Poisson(L | x)
  double tail;   // epsilon = sum_{k > K} Poisson(k | x) = 1 - sum_{k <= K}
  int64_t L;     // first jump index with non-negligible weight (left mass < e^-50)
  int64_t K;     // last jump index (Algorithm 2's loop exit)
  int64_t woff;  // offset of P_L..P_K (tail folded into P_K) in the weight arena, -1 if absent
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
  // Batches of uneven birth-death instances (nullable): per-job state count
  // and per-job times (times + job * ntimes).
  const int32_t* jobN;
  int times_per_job;
  // Weight arena (nullable): windows are stored at offsets taken with an
  // atomic counter; a window that does not fit gets woff = -1 and sets
  // *arena_over (the chain then runs the recurrence for it).
  void* arena;
  int64_t arena_cap;                // elements
  unsigned long long* arena_used;   // element counter (zeroed before the planner)
  int* arena_over;
  int arena_fp64;                   // element type: 1 = double, 0 = float
  // 1: the chain is FP64 (weights formed to FP64 precision); 0: FP32 chain
  // (weights formed in float-float on the FP32 pipe).
  int fp64_weights;
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
  int nmem;                // length of the generic member list kept on chip (0: every group has <= 2 members)
  double* ll;              // device, B
  int renorm;              // FP32: period in jumps of the exit-defect correction (0 = off)
  int64_t slab;            // states per CTA of the cluster (whole rows for 2-D models)
  int* status;
  // Batches of uneven birth-death instances (all nullable):
  const int32_t* jobN;     // states of each job (BD1D: M = N, P = 1; slab = ceil(N / cluster))
  const int64_t* job_off;  // element offset of each job's outputs and compensation
  const int32_t* job_map;  // cluster index -> job (longest first)
  const int64_t* job_s0;   // rho0 = delta at s0 for each job (instead of rho0)
  int tile_max;            // padded tile size of the largest job in the launch
  const void* arena;       // planner's weight arena (T), indexed by Win::woff
  // Polls of a bounded wait between a kernel's warp groups before it gives up
  // (status kStatusTimeout); MJP_OPT_WAIT_LIMIT.
  long long wait_limit = 1LL << 24;
};

// One jump of the general-CSR chain (csr.cu).
struct CsrJumpParams {
  int64_t n, nslices;
  const int64_t* slice_ptr;  // first entry of each slice
  const int32_t* slice_len;  // entries per state in each slice
  const int32_t* col;        // permuted source state of each entry
  const void* val;           // lambda / Omega (T)
  const void* diag;          // 1 - e_n / Omega (T)
  const void* rho_prev;      // rho_{k-1} (T, permuted order)
  void* rho_next;            // rho_k
  int64_t k;
  bool jump;                 // form rho_k (false: only accumulate rho_{k-1})
  int tlo, thi;              // times whose window holds k-1
  const double* wtab;        // weights table
  const int64_t* woff;       // table offset per time
  const int64_t* L;          // window start per time
  const int64_t* K;          // window end per time
  void* out;                 // ntimes x n outputs (T, permuted order)
  float* comp;               // FP32 Kahan compensation, ntimes x n
};

// The whole general-CSR chain in one cooperative launch (csr.cu): every jump
// of csr_jump_kernel's body, then a grid-wide barrier with a bounded wait.
struct CsrChainParams {
  CsrJumpParams j;           // k, jump, tlo, thi, rho_prev and rho_next are set per jump in the kernel
  int ntimes;
  int64_t kmax;
  void* rho;                 // two state vectors of n elements (T), ping-pong
  unsigned* bar;             // [0] arrivals, [1] generation; zeroed before the launch
  long long wait_limit;      // polls of a waiting CTA before it gives up (status kStatusTimeout)
  int* status;
};

// Fourth-order Runge-Kutta for one birth-death distribution (rk4.cu).
struct Rk4Params {
  const double* theta;   // device, {beta, gamma} or {beta, gamma, lambda_act, lambda_ina}
  int kind;              // MJP_BD1D or MJP_TWOSTATE
  int N, M;              // states; M = N_R for the two-state model
  const double* rho0;    // device, N values
  double* out;           // device, ntimes x N (caller's time order)
  const int32_t* orig;   // device, sorted time q -> caller's row
  const int64_t* steps;  // device, steps of the interval ending at sorted time q
  const double* hstep;   // device, step length of that interval
  int ntimes;
};

}  // namespace mjp

// Host-side launchers implemented in the .cu files.
namespace mjp {
cudaError_t launch_plan(const PlanParams& p, cudaStream_t s);
// map[r] = job with the r-th largest Kmax (ties by index): longest chain first.
cudaError_t launch_order_jobs(const JobInfo* info, int B, int32_t* map, cudaStream_t s);
cudaError_t launch_chain_stencil(int kind, int precision, int loglik_mode, const ChainParams& p,
                                 int cluster, int threads, cudaStream_t s);
int64_t chain_stencil_slab(int kind, int64_t M, int64_t P, int cluster);
int chain_stencil_tile(int kind, int64_t M, int64_t P, int64_t slab);
size_t chain_stencil_smem_tile(int precision, int loglik_mode, int tile, int ntimes, int G, int nmem);
size_t chain_stencil_smem(int kind, int precision, int loglik_mode, int64_t M, int64_t P, int64_t slab,
                          int ntimes, int G, int nmem);
int chain_stencil_max_cluster_blocks(int kind, int precision, int loglik_mode, int cluster,
                                     int threads, size_t smem);
// Register-resident chain (stencil_reg.cu): mRNA/protein box, FP32, loglik.
struct RegPlan {
  int cluster;   // CTAs per instance (rows split between them)
  int rows;      // rows per CTA (a multiple of 2 qr)
  int nq;        // column quads (ceil(M / 4))
  int qr;        // row pairs per thread (4 or 5)
  int tmax;      // threads per CTA at most (384, one CTA per SM)
  int threads;   // per CTA, including the weights warp
  size_t smem;   // dynamic shared memory per CTA
};
bool chain_reg2d_plan(int64_t M, int64_t P, int ntimes, int nmem, int max_cluster, int threads, RegPlan* out);
cudaError_t launch_chain_reg2d(const ChainParams& p, const RegPlan& rp, cudaStream_t s);
// Register-resident birth-death chain (stencil_reg1d.cu): expv mode, FP32 or
// FP64, one CTA or a cluster with temporal blocking per instance.
struct Reg1dPlan {
  int cluster;   // CTAs per instance
  int threads;   // per CTA
  int qp;        // state pairs per thread
  int halo;      // halo width h (jumps between cluster exchanges); 0 for one CTA
  size_t smem;   // dynamic shared memory per CTA
};
// small: prefer one state pair per thread when the chain fits a CTA that way
// (latency of single solves); batches keep the wider runs (throughput).
bool chain_reg1d_plan(int precision, int64_t Nmax, int ntimes, int cluster, int halo, Reg1dPlan* out,
                      bool small = false);
int64_t chain_reg1d_max_states(int precision);
cudaError_t launch_chain_reg1d(int precision, const ChainParams& p, const Reg1dPlan& rp, cudaStream_t s);
// Register-resident two-state chain (stencil_regts.cu): FP32 loglik, one CTA
// per theta, groups of at most two members.
struct RegTsPlan {
  int threads;   // per CTA: chain warps and reducer warps
  int chain_warps;
  int qp;        // state pairs per thread and row (1, 3 or 7)
  int tlo;       // first chain thread holding an observed column
  int nslot;     // history slots (qp per thread from tlo on)
  size_t smem;   // dynamic shared memory per CTA
};
bool chain_regts_plan(int64_t M, int ntimes, int G, int maxmem, int col_lo, int col_hi, int threads,
                      RegTsPlan* out);
cudaError_t launch_chain_regts(const ChainParams& p, const RegTsPlan& rp, cudaStream_t s);
int64_t rk4_max_states();
// Krylov subspace steps for one birth-death distribution (krylov.cu).
struct KrylovParams {
  const double* theta;   // device, {beta, gamma} or {beta, gamma, lambda_act, lambda_ina}
  int kind;              // MJP_BD1D or MJP_TWOSTATE
  int N, M;              // states; M = N_R for the two-state model
  const double* rho0;    // device, N values
  double* out;           // device, ntimes x N (caller's time order)
  const int32_t* orig;   // device, sorted time q -> caller's row
  const int64_t* steps;  // device, steps of the interval ending at sorted time q
  const double* hstep;   // device, step length of that interval
  int ntimes;
  int kappa;             // subspace size
  double maxe;           // max_n |a_nn| (invariant-space threshold)
  double* Q;             // device scratch, kappa x N
  int* status;
};
// J-MJP state probabilities for one theta (jmjp.cu).
struct JmjpParams {
  const double* theta;       // device
  int N, M;                  // states; M = N_R for the two-state model
  const void* rho0;          // device, N values (T)
  int nobs;
  const int32_t* ksorted;    // device, jump counts sorted ascending
  const int32_t* order;      // device, sorted position -> caller's observation
  const int32_t* group_ptr;  // device, nobs + 1 (sorted order)
  const int32_t* members;    // device
  double* phi;               // device, nobs (caller's order)
  double omega;              // 1.1 max_n |a_nn|
  int nchunks;               // chunks of sorted observations staged in shared memory
  const int32_t* chunk;      // device, nchunks + 1: first observation of each chunk
  int cap_obs, cap_mem;      // shared-memory capacity of a chunk (observations, members)
  int kmax;                  // largest jump count
};
int64_t jmjp_max_states(int precision);
// Shared-memory bytes left for observation chunks beside the chain of N states.
size_t jmjp_chunk_bytes(int precision, int N);
cudaError_t launch_jmjp(int kind, int precision, const JmjpParams& p, cudaStream_t s);
int krylov_max_states();
int krylov_max_kappa();
cudaError_t launch_krylov(const KrylovParams& p, cudaStream_t s);
cudaError_t launch_rk4(const Rk4Params& p, cudaStream_t s);
cudaError_t launch_fill_weights(const Win* win, int ntimes, const int64_t* woff, double* table, cudaStream_t s);
cudaError_t launch_permute_in(int precision, const void* src, const int32_t* perm, void* dst, int64_t n,
                              cudaStream_t s);
cudaError_t launch_permute_out(int precision, const void* src, const int32_t* perm, void* dst, int64_t n,
                               int ntimes, const int32_t* orig, cudaStream_t s);
cudaError_t launch_csr_jump(int precision, const CsrJumpParams& p, cudaStream_t s);
cudaError_t launch_csr_chain(int precision, const CsrChainParams& p, cudaStream_t s);
cudaError_t launch_csr_loglik(const void* outp, int precision, int64_t n, const int64_t* gptr, int ntimes,
                              const double* counts, const int64_t* mptr, const int32_t* members,
                              const int32_t* perm, double* ll, int* status, cudaStream_t s);
}  // namespace mjp
