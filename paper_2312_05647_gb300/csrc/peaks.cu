// peaks.cu -- measured on-chip peaks for the roofline denominators of the
// chain kernels: the FP32 fused-multiply-add rate (the better of packed FP32x2
// and scalar instructions), the shared-memory bandwidth of all SMs and the
// L2's random-gather rate.  Not part of the method; the benchmark reports the
// chain kernels against these measured numbers instead of nominal ones.
#include <cuda_runtime.h>

#include "host_util.h"
#include "internal.cuh"

namespace {

constexpr int kFmaChains = 8;  // independent FP32x2 chains per thread

// Every thread runs kFmaChains independent chains of packed FP32x2 FMAs
// (a <- a * m + c): 4 flops per instruction.  The result is written only when
// impossible in practice, so the loop is not removed.
__global__ void __launch_bounds__(512) peak_fma_kernel(float* sink, int iters) {
  float2 a[kFmaChains];
#pragma unroll
  for (int j = 0; j < kFmaChains; ++j) a[j] = make_float2(1e-3f * (threadIdx.x + j), 2e-3f * (blockIdx.x + j));
  const float2 m = make_float2(0.999999f, 0.999998f), c = make_float2(1e-7f, 2e-7f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kFmaChains; ++j) a[j] = __ffma2_rn(a[j], m, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < kFmaChains; ++j) s += a[j].x + a[j].y;
  if (s == -1.0f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The same work as scalar FP32 FMAs: 2 kFmaChains independent chains per
// thread (the instruction is emitted as written, so the chains stay scalar).
__global__ void __launch_bounds__(512) peak_fma1_kernel(float* sink, int iters) {
  float a[2 * kFmaChains];
#pragma unroll
  for (int j = 0; j < 2 * kFmaChains; ++j) a[j] = 1e-3f * (threadIdx.x + 3 * j);
  const float m = 0.999997f, c = 3e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 2 * kFmaChains; ++j) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[j]) : "f"(m), "f"(c));
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < 2 * kFmaChains; ++j) s += a[j];
  if (s == -1.0f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Every thread reads one 16-byte vector from shared memory and writes one per
// iteration, consecutive threads on consecutive vectors (no bank conflicts),
// so each warp instruction moves 512 bytes.
__global__ void __launch_bounds__(512) peak_smem_kernel(float* sink, int iters) {
  extern __shared__ __align__(16) float4 buf[];
  const int t = threadIdx.x, n = blockDim.x;
  buf[t] = make_float4((float)t, 1.0f, 2.0f, 3.0f);
  buf[t + n] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  __syncthreads();
  const unsigned rd = (unsigned)__cvta_generic_to_shared(buf + t);
  const unsigned wr = (unsigned)__cvta_generic_to_shared(buf + n + t);
  float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  for (int i = 0; i < iters; ++i) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(rd));
    acc.x += v.x;
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(wr), "f"(acc.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
  }
  if (acc.x == -1.0f) sink[blockIdx.x * blockDim.x + t] = acc.x;
}

// Every thread gathers 4-byte values at pseudo-random positions of an
// L2-resident 4 MB array (a linear congruential sequence per thread; eight
// loads per iteration, independent of each other's values): the random-access
// rate of the L2 that the general-CSR chain's gathers of rho meet.
__global__ void __launch_bounds__(512) peak_gather_kernel(const float* __restrict__ a, unsigned mask, float* sink,
                                                          int iters) {
  unsigned h = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 12345u;
  float acc[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) acc[j] = 0.0f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      h = h * 1664525u + 1013904223u;
      acc[j] += __ldg(a + ((h >> 7) & mask));
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += acc[j];
  if (s == -1.0f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int mjp_measure_peak(int which, int iters, double* result, void* stream) try {
  using namespace mjp;
  if (!result || iters < 1 || (which != MJP_PEAK_FP32_FMA && which != MJP_PEAK_SMEM && which != MJP_PEAK_L2_GATHER))
    return fail(MJP_ERR_ARG, "mjp_measure_peak: unknown quantity, iters < 1 or NULL result");
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  MJP_CUDA(cudaGetDevice(&dev));
  MJP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int threads = 512, blocks = 2 * sms;  // two CTAs of 512 threads per SM
  struct Sink {  // released on every return path
    DevBuf b;
    ~Sink() { b.release(); }
  } sk;
  DevBuf& sink = sk.b;
  int rc = sink.ensure(sizeof(float) * (size_t)blocks * threads);
  if (rc) return rc;
  constexpr unsigned kGatherN = 1u << 20;  // 4 MB of FP32, as rho of the 2^20-state CSR configuration
  struct Arr {
    DevBuf b;
    ~Arr() { b.release(); }
  } ar;
  if (which == MJP_PEAK_L2_GATHER) {
    if ((rc = ar.b.ensure(sizeof(float) * kGatherN))) return rc;
    MJP_CUDA(cudaMemsetAsync(ar.b.p, 0, sizeof(float) * kGatherN, s));
  }
  const size_t smem = (which == MJP_PEAK_SMEM) ? 2 * threads * sizeof(float4) : 0;
  // form 1: the scalar FP32 FMA kernel (the FP32 peak is the better form's).
  auto launch = [&](int form) -> cudaError_t {
    if (which == MJP_PEAK_FP32_FMA) {
      if (form == 0) peak_fma_kernel<<<blocks, threads, 0, s>>>(sink.as<float>(), iters);
      else peak_fma1_kernel<<<blocks, threads, 0, s>>>(sink.as<float>(), iters);
    } else if (which == MJP_PEAK_SMEM) {
      peak_smem_kernel<<<blocks, threads, smem, s>>>(sink.as<float>(), iters);
    } else {
      peak_gather_kernel<<<blocks, threads, 0, s>>>(ar.b.as<float>(), kGatherN - 1, sink.as<float>(), iters);
    }
    return cudaGetLastError();
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  MJP_CUDA(cudaEventCreate(&e0));
  MJP_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  const int forms = (which == MJP_PEAK_FP32_FMA) ? 2 : 1;
  for (int f = 0; f < forms; ++f) {
    MJP_CUDA(launch(f));  // warm-up (clocks, instruction cache)
    for (int r = 0; r < 3; ++r) {
      MJP_CUDA(cudaEventRecord(e0, s));
      MJP_CUDA(launch(f));
      MJP_CUDA(cudaEventRecord(e1, s));
      MJP_CUDA(cudaEventSynchronize(e1));
      float ms = 0.0f;
      MJP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) best = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double work = (double)blocks * threads * iters;
  if (which == MJP_PEAK_FP32_FMA) *result = work * kFmaChains * 4.0 / (best * 1e-3) / 1e12;  // TFLOP/s
  else if (which == MJP_PEAK_SMEM) *result = work * 32.0 / (best * 1e-3) / 1e9;            // GB/s, read + write
  else *result = work * 8.0 / (best * 1e-3) / 1e9;                                          // G gathers/s
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}
