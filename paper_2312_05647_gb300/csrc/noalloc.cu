// noalloc.cu -- expv_series_static: the stencil series without any device
// allocation.
//
// Who needs this: callers that may not call cudaMalloc/cudaFree once they are
// running -- applications that hand all device memory to their own pool or
// fix their memory budget up front, plugins hosted by a framework that owns
// the allocator, and latency-critical loops that must not risk the device-wide
// synchronisation cudaMalloc/cudaFree can trigger.  Everything such a caller
// would otherwise get from a model handle's workspace (sorted times, the
// planner's windows, the status word, the FP32 Kahan compensation buffer)
// lives here in one file-scope __device__ array of fixed size, created when
// the library is loaded and kept by every GPU that loads it until the process
// exits.  The caller still owns rho0 and out.
//
// The same planner and chain kernels as expv_series run; only the storage of
// their scratch differs.
#include <cstdio>
#include <mutex>

#include "host_util.h"
#include "internal.cuh"

namespace {

constexpr size_t kStaticScratchBytes = (size_t)16 << 20;  // 16 MiB
constexpr size_t kAlign = 256;
constexpr int kMaxDevices = 64;
constexpr size_t kSmemMax = 227 * 1024;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch on each device (host code may not use
// the symbol itself: on the host it is only a stand-in, not a device pointer).
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

size_t up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

}  // namespace

extern "C" int expv_series_static(int kind, const int64_t* dims, int ndims, const double* theta, int ntheta,
                                  const float* rho0, const double* times, int ntimes, float* out,
                                  void* stream) try {
  using namespace mjp;
  if (!dims || !theta || !rho0 || !times || !out) return fail(MJP_ERR_ARG, "NULL argument");
  if (ntimes < 1 || ntimes > kMaxTimes) return fail(MJP_ERR_ARG, "ntimes must be in [1, 256]");
  int64_t M, P, N;
  int want_theta;
  // Each dimension is checked before any product, so N cannot wrap; the
  // chain kernels index states in 32 bits.
  constexpr int64_t kMaxN = ((int64_t)1 << 31) - 1;
  if (kind == MJP_BD1D && ndims == 1 && dims[0] >= 1 && dims[0] <= kMaxN) {
    M = dims[0]; P = 1; N = M; want_theta = 2;
  } else if (kind == MJP_TWOSTATE && ndims == 1 && dims[0] >= 2 && dims[0] <= kMaxN / 2) {
    M = dims[0]; P = 2; N = 2 * M; want_theta = 4;
  } else if (kind == MJP_MRNA_PROT2D && ndims == 2 && dims[0] >= 2 && dims[1] >= 1 && dims[0] <= kMaxN &&
             dims[1] <= kMaxN / dims[0]) {
    M = dims[0]; P = dims[1]; N = M * P; want_theta = 4;
  } else {
    return fail(MJP_ERR_ARG, "kind/dims must describe a stencil model (BD1D, TWOSTATE or MRNA_PROT2D) of at most "
                             "2^31 - 1 states");
  }
  if (ntheta != want_theta) return fail(MJP_ERR_ARG, "wrong number of parameters for this kind");
  for (int q = 0; q < ntheta; ++q)
    if (!(theta[q] >= 0.0) || !(theta[q] < 1e308)) return fail(MJP_ERR_ARG, "rates must be finite and >= 0");
  for (int i = 0; i < ntimes; ++i)
    if (!(times[i] >= 0.0) || !(times[i] < 1e308)) return fail(MJP_ERR_ARG, "times must be finite and >= 0");

  // Carve the static array: status | info | theta | times | order | windows | compensation.
  const size_t o_status = 0, o_info = up(sizeof(int)), o_theta = o_info + up(sizeof(JobInfo));
  const size_t o_times = o_theta + up(sizeof(double) * ntheta);
  const size_t o_orig = o_times + up(sizeof(double) * ntimes);
  const size_t o_win = o_orig + up(sizeof(int32_t) * ntimes);
  const size_t o_comp = o_win + up(sizeof(Win) * ntimes);
  const size_t need = o_comp + up(sizeof(float) * (size_t)ntimes * (size_t)N);
  if (need > kStaticScratchBytes) {
    char msg[192];
    snprintf(msg, sizeof(msg),
             "expv_series_static needs %zu bytes of scratch (ntimes x N x 4 plus bookkeeping); "
             "its static scratch holds %zu bytes",
             need, kStaticScratchBytes);
    return fail(MJP_ERR_ARG, msg);
  }

  // The call copies from stack memory and synchronises `stream`, neither of
  // which a stream capture accepts: refuse to run while `stream` captures.
  {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    MJP_CUDA(cudaStreamIsCapturing((cudaStream_t)stream, &cs));
    if (cs != cudaStreamCaptureStatusNone)
      return fail(MJP_ERR_UNSUPPORTED, "expv_series_static cannot run while its stream is capturing a graph");
  }

  // One-time set-up per device, with that device current.
  int dev = 0;
  MJP_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(MJP_ERR_UNSUPPORTED, "device ordinal above 63");
  unsigned char* base;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return fail(MJP_ERR_CUDA, std::string("cudaGetSymbolAddress of the static scratch: ") + cudaGetErrorString(e));
      }
      g_scratch_addr[dev] = p;
    }
    base = static_cast<unsigned char*>(g_scratch_addr[dev]);
  }

  // Launch shape: the smallest cluster whose slabs fit shared memory, one
  // column per stencil thread for the 2-D models, plus the weights warp.
  int C = 0;
  for (int c = 1; c <= 16; c *= 2)
    if (chain_stencil_smem(kind, MJP_FP32, 0, M, P, chain_stencil_slab(kind, M, P, c), ntimes, 0, 0) <= kSmemMax) {
      C = c;
      break;
    }
  if (C == 0) return fail(MJP_ERR_UNSUPPORTED, "state space too large for an on-chip stencil chain");
  const int64_t slab = chain_stencil_slab(kind, M, P, C);
  int64_t W = (kind == MJP_BD1D) ? slab : M;
  if (kind != MJP_BD1D && W > 992) return fail(MJP_ERR_UNSUPPORTED, "rows longer than 992 states are not supported");
  int64_t groups = 1;
  if (kind != MJP_BD1D) {
    int64_t pair_rows = (slab / M + 1) / 2;
    groups = (pair_rows + 19) / 20;
    if (groups > 992 / W) groups = 992 / W;
    if (groups < 1) groups = 1;
  }
  int64_t t = (W >= 992 ? 992 : W * groups);
  t = (t + 31) / 32 * 32 + 32;
  const int threads = (int)(t < 64 ? 64 : (t > 1024 ? 1024 : t));
  // The cluster must fit the GPU at all (the same check as expv_series).
  const size_t smem = chain_stencil_smem(kind, MJP_FP32, 0, M, P, slab, ntimes, 0, 0);
  if (chain_stencil_max_cluster_blocks(kind, MJP_FP32, 0, C, threads, smem) <= 0)
    return fail(MJP_ERR_UNSUPPORTED, "stencil chain configuration cannot be made resident");

  // Times in ascending order with their caller rows (no heap: fixed arrays).
  double st[kMaxTimes];
  int32_t order[kMaxTimes];
  for (int i = 0; i < ntimes; ++i) order[i] = i;
  for (int i = 1; i < ntimes; ++i)  // stable insertion sort
    for (int j = i; j > 0 && times[order[j]] < times[order[j - 1]]; --j) {
      int32_t tmp = order[j];
      order[j] = order[j - 1];
      order[j - 1] = tmp;
    }
  for (int i = 0; i < ntimes; ++i) st[i] = times[order[i]];

  cudaStream_t s = (cudaStream_t)stream;
  int* d_status = reinterpret_cast<int*>(base + o_status);
  MJP_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int), s));  // the array keeps the last call's contents
  MJP_CUDA(cudaMemcpyAsync(base + o_theta, theta, sizeof(double) * ntheta, cudaMemcpyHostToDevice, s));
  MJP_CUDA(cudaMemcpyAsync(base + o_times, st, sizeof(double) * ntimes, cudaMemcpyHostToDevice, s));
  MJP_CUDA(cudaMemcpyAsync(base + o_orig, order, sizeof(int32_t) * ntimes, cudaMemcpyHostToDevice, s));

  PlanParams pp = {};
  pp.kind = kind; pp.M = (int32_t)M; pp.P = (int32_t)P; pp.N = N;
  pp.ntheta = ntheta; pp.theta = reinterpret_cast<const double*>(base + o_theta); pp.B = 1;
  pp.ntimes = ntimes; pp.times = reinterpret_cast<const double*>(base + o_times);
  pp.trunc_mode = MJP_TRUNC_PAPER; pp.tol = 0.0; pp.omega_factor = 1.1; pp.omega_fixed = -1.0;
  pp.kcap = (int64_t)1 << 26; pp.win = reinterpret_cast<Win*>(base + o_win);
  pp.info = reinterpret_cast<JobInfo*>(base + o_info); pp.status = d_status;
  MJP_CUDA(launch_plan(pp, s));

  ChainParams cp = {};
  cp.M = (int32_t)M; cp.P = (int32_t)P; cp.N = N;
  cp.ntheta = ntheta; cp.theta = pp.theta; cp.B = 1; cp.ntimes = ntimes;
  cp.orig = reinterpret_cast<const int32_t*>(base + o_orig); cp.win = pp.win; cp.info = pp.info; cp.rho0 = rho0;
  cp.out = out; cp.out_stride = 0; cp.comp = reinterpret_cast<float*>(base + o_comp); cp.comp_stride = 0;
  cp.renorm = kDefectPeriod; cp.slab = slab; cp.status = d_status;
  MJP_CUDA(launch_chain_stencil(kind, MJP_FP32, 0, cp, C, threads, s));

  int st_host = 0;
  MJP_CUDA(cudaMemcpyAsync(&st_host, d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  MJP_CUDA(cudaStreamSynchronize(s));
  if (st_host == kStatusKcap) return fail(MJP_ERR_KCAP, "truncation index K above the cap");
  if (st_host != 0) return fail(MJP_ERR_NUMERIC, "device reported a numerical error");
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}
