// csr.cu -- the jump chain for a general sparse rate matrix.
//
// Storage (built once per model on the host, see api.cu): the uniformised
// matrix B = I + A/Omega (Eq. B_def) is kept as its transpose -- for every
// target state n the incoming transitions m -> n with weights lambda_mn /
// Omega -- in SELL-32 form: states are renumbered by decreasing in-degree,
// cut into slices of 32 consecutive states, and each slice stores its entries
// column-major (entry j of the slice's 32 states side by side), padded to the
// slice's largest in-degree.  A warp owns a slice; lane i owns state 32s+i,
// so every index and value load is one coalesced 128/256-byte transaction and
// the sorting keeps padding negligible.  The diagonal 1 - e_n/Omega is a
// separate array.  rho (4 MB for 2^20 FP32 states) stays resident in L2;
// neighbour values are gathered with read-only loads.
//
// Jump k accumulates rho_{k-1} into the active times' outputs
// (Kahan-compensated in FP32) and forms rho_k = rho_{k-1} B (Algorithm 2's
// loop body); rho_{k+1} depends on all of rho_k, so jumps are separated grid-
// wide.  Default: one launch per jump.  Alternative (MJP_OPT_CHAIN = 2): the
// whole chain in one cooperative launch (all CTAs co-resident), jumps
// separated by a software grid barrier whose waits are bounded (a CTA that
// polls longer than the limit records kStatusTimeout and leaves, and so do
// the others at their next barrier).  Both run the same per-jump code, so
// their results are identical.  The Poisson weights of every (time, jump)
// come from a table filled by `fill_weights_kernel` with Algorithm 2's
// recurrence P_k = P_{k-1} x/k started from the planner's P_L.
#include <algorithm>

#include "internal.cuh"

namespace mjp {

namespace {

__device__ __forceinline__ float fma_t(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_t(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_t(double a, double b) { return __dmul_rn(a, b); }

// One warp per time: table[i][k - L_i] = P_k for k in [L_i, K_i], with the
// tail 1 - sum P folded into the last entry.
__global__ void fill_weights_kernel(const Win* win, int ntimes, const int64_t* woff, double* table) {
  int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= ntimes || (threadIdx.x & 31) != 0) return;
  Win w = win[i];
  double* t = table + woff[i];
  double P = w.PL;
  for (int64_t k = w.L; k <= w.K; ++k) {
    if (k > w.L) P = __dmul_rn(P, __ddiv_rn(w.x, (double)k));
    t[k - w.L] = (k == w.K) ? P + w.tail : P;
  }
}

template <typename T>
__global__ void permute_in_kernel(const T* __restrict__ src, const int32_t* __restrict__ perm, T* __restrict__ dst,
                                  int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[perm[i]] = src[i];
}

template <typename T>
__global__ void permute_out_kernel(const T* __restrict__ src, const int32_t* __restrict__ perm, T* __restrict__ dst,
                                   int64_t n, int ntimes, const int32_t* __restrict__ orig) {
  // dst[orig[i]][s] = src[i][perm[s]]  (row-major ntimes x n)
  const int64_t total = n * ntimes;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = e / n, s = e - i * n;
    dst[(int64_t)orig[i] * n + s] = src[i * n + perm[s]];
  }
}

template <typename T>
__device__ __forceinline__ void csr_jump_body(const CsrJumpParams& p) {
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const T* __restrict__ cur = reinterpret_cast<const T*>(p.rho_prev);
  T* __restrict__ nxt = reinterpret_cast<T*>(p.rho_next);
  const T* __restrict__ val = reinterpret_cast<const T*>(p.val);
  const T* __restrict__ diag = reinterpret_cast<const T*>(p.diag);
  T* __restrict__ out = reinterpret_cast<T*>(p.out);
  const int64_t kp = p.k - 1;  // jump whose values are accumulated now
  for (int64_t s = gwarp; s < p.nslices; s += nwarps) {
    const int64_t r = s * 32 + lane;
    const bool valid = r < p.n;
    const T v = valid ? cur[r] : (T)0;
    // rho*_i += P_{k-1} rho_{k-1} for the times whose window holds k-1.
    if (valid) {
      for (int i = p.tlo; i <= p.thi; ++i) {
        const T w = (T)p.wtab[p.woff[i] + (kp - p.L[i])];
        T* o = out + (int64_t)i * p.n + r;
        if (sizeof(T) == 4) {
          float* c = p.comp + (int64_t)i * p.n + r;
          float acc, cc;
          if (kp == p.L[i]) {
            acc = __fmul_rn((float)w, (float)v);
            cc = 0.0f;
          } else {
            acc = (float)*o;
            cc = *c;
            float y = __fsub_rn(__fmul_rn((float)w, (float)v), cc);
            float t = __fadd_rn(acc, y);
            cc = __fsub_rn(__fsub_rn(t, acc), y);
            acc = t;
          }
          if (kp == p.K[i]) *o = (T)__fsub_rn(acc, cc);
          else {
            *o = (T)acc;
            *c = cc;
          }
        } else {
          *o = (kp == p.L[i]) ? mul_t(w, v) : fma_t(w, v, *o);
        }
      }
    }
    if (p.jump && valid) {
      T y = mul_t(diag[r], v);
      const int64_t base = p.slice_ptr[s] + lane;
      const int width = p.slice_len[s];
      // Entries four at a time: the index and value loads of the group, then
      // its four gathers, so each lane has several independent loads in flight
      // (the same multiply-adds in the same order as one at a time).
      int j = 0;
      for (; j + 4 <= width; j += 4) {
        const int64_t e = base + (int64_t)j * 32;
        const int32_t c0 = __ldg(p.col + e), c1 = __ldg(p.col + e + 32), c2 = __ldg(p.col + e + 64),
                      c3 = __ldg(p.col + e + 96);
        const T a0 = __ldg(val + e), a1 = __ldg(val + e + 32), a2 = __ldg(val + e + 64), a3 = __ldg(val + e + 96);
        const T g0 = __ldg(cur + c0), g1 = __ldg(cur + c1), g2 = __ldg(cur + c2), g3 = __ldg(cur + c3);
        y = fma_t(a0, g0, y);
        y = fma_t(a1, g1, y);
        y = fma_t(a2, g2, y);
        y = fma_t(a3, g3, y);
      }
      for (; j < width; ++j) {
        const int64_t e = base + (int64_t)j * 32;
        const int32_t c = __ldg(p.col + e);
        y = fma_t(__ldg(val + e), __ldg(cur + c), y);
      }
      nxt[r] = y;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(512) csr_jump_kernel(CsrJumpParams p) {
  csr_jump_body<T>(p);
}

// Grid-wide barrier with a bounded wait.  bar[0] counts arrivals, bar[1] is
// the generation: the last CTA to arrive resets the count and advances the
// generation; the others poll the generation they read before arriving, at
// most `limit` times.  Returns false (and records kStatusTimeout) when the
// wait ran out; every CTA then leaves the chain, the late ones at the latest
// at their next barrier, which can no longer complete.
__device__ bool grid_barrier(unsigned* bar, long long limit, int* status) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u) + 1u;
    int good = 1;
    if (arrived == gridDim.x) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long it = 0;
      while (*gen == g) {
        if (it++ >= limit) {
          good = 0;
          break;
        }
        __nanosleep(20);
      }
    }
    __threadfence();
    if (!good) atomicCAS(status, 0, kStatusTimeout);
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

template <typename T>
__global__ void __launch_bounds__(1024) csr_chain_kernel(CsrChainParams c) {
  CsrJumpParams p = c.j;
  const size_t n = (size_t)p.n;
  T* rho = reinterpret_cast<T*>(c.rho);
  int lo = 0, hi = -1;  // times whose window holds jump k-1 (ascending times)
  for (int64_t k = 1; k <= c.kmax + 1; ++k) {
    const int64_t kp = k - 1;
    while (lo < c.ntimes && p.K[lo] < kp) ++lo;
    while (hi + 1 < c.ntimes && p.L[hi + 1] <= kp) ++hi;
    p.k = k;
    p.jump = k <= c.kmax;
    p.tlo = lo;
    p.thi = hi;
    p.rho_prev = rho + ((kp & 1) ? n : 0);
    p.rho_next = rho + ((kp & 1) ? 0 : n);
    csr_jump_body<T>(p);
    if (k <= c.kmax && !grid_barrier(c.bar, c.wait_limit, c.status)) return;
  }
}

// Snapshot log-likelihood from the permuted outputs: one CTA.
__global__ void csr_loglik_kernel(const void* outp, int precision, int64_t n, const int64_t* gptr, int ntimes,
                                  const double* counts, const int64_t* mptr, const int32_t* members,
                                  const int32_t* perm, double* ll, int* status) {
  __shared__ double red[32];
  double acc = 0.0;
  bool bad = false;
  for (int i = 0; i < ntimes; ++i) {
    for (int64_t g = gptr[i] + threadIdx.x; g < gptr[i + 1]; g += blockDim.x) {
      double a = 0.0;
      for (int64_t q = mptr[g]; q < mptr[g + 1]; ++q) {
        int64_t idx = (int64_t)i * n + perm[members[q]];
        a += (precision == MJP_FP64) ? reinterpret_cast<const double*>(outp)[idx]
                                     : (double)reinterpret_cast<const float*>(outp)[idx];
      }
      double c = counts[g];
      if (c == 0.0) continue;
      if (a > 0.0) acc += c * log(a);
      else if (a > -1e-30) acc = -INFINITY;
      else bad = true;
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *ll = t;
    if (isnan(t) && status) atomicCAS(status, 0, kStatusNumeric);
  }
  if (bad && status) atomicCAS(status, 0, kStatusNumeric);
}

int grid_for(int64_t work, int block) {
  int64_t g = (work + block - 1) / block;
  return (int)(g < 152 * 16 ? (g < 1 ? 1 : g) : 152 * 16);
}

}  // namespace

cudaError_t launch_fill_weights(const Win* win, int ntimes, const int64_t* woff, double* table, cudaStream_t s) {
  fill_weights_kernel<<<(ntimes + 7) / 8, 256, 0, s>>>(win, ntimes, woff, table);
  return cudaGetLastError();
}

cudaError_t launch_permute_in(int precision, const void* src, const int32_t* perm, void* dst, int64_t n,
                              cudaStream_t s) {
  if (precision == MJP_FP64)
    permute_in_kernel<double><<<grid_for(n, 256), 256, 0, s>>>((const double*)src, perm, (double*)dst, n);
  else
    permute_in_kernel<float><<<grid_for(n, 256), 256, 0, s>>>((const float*)src, perm, (float*)dst, n);
  return cudaGetLastError();
}

cudaError_t launch_permute_out(int precision, const void* src, const int32_t* perm, void* dst, int64_t n,
                               int ntimes, const int32_t* orig, cudaStream_t s) {
  if (precision == MJP_FP64)
    permute_out_kernel<double><<<grid_for(n * ntimes, 256), 256, 0, s>>>((const double*)src, perm, (double*)dst, n,
                                                                          ntimes, orig);
  else
    permute_out_kernel<float><<<grid_for(n * ntimes, 256), 256, 0, s>>>((const float*)src, perm, (float*)dst, n,
                                                                         ntimes, orig);
  return cudaGetLastError();
}

cudaError_t launch_csr_jump(int precision, const CsrJumpParams& p, cudaStream_t s) {
  const int block = 512;
  int grid = grid_for(p.nslices * 32, block);
  if (precision == MJP_FP64) csr_jump_kernel<double><<<grid, block, 0, s>>>(p);
  else csr_jump_kernel<float><<<grid, block, 0, s>>>(p);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_chain_typed(const CsrChainParams& c, cudaStream_t s) {
  // 1024-thread CTAs: the fewer CTAs meet at each grid barrier, the shorter it is.
  const int block = 1024;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, csr_chain_kernel<T>, block, 0)) != cudaSuccess)
    return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  // Every CTA must be resident at once: at most the occupancy limit, and no
  // more than the slices need.
  int grid = std::min<int64_t>((int64_t)per_sm * sms, (c.j.nslices * 32 + block - 1) / block);
  if (grid < 1) grid = 1;
  void* args[] = {const_cast<CsrChainParams*>(&c)};
  return cudaLaunchCooperativeKernel((const void*)csr_chain_kernel<T>, dim3(grid), dim3(block), args, 0, s);
}

cudaError_t launch_csr_chain(int precision, const CsrChainParams& p, cudaStream_t s) {
  return precision == MJP_FP64 ? launch_chain_typed<double>(p, s) : launch_chain_typed<float>(p, s);
}

cudaError_t launch_csr_loglik(const void* outp, int precision, int64_t n, const int64_t* gptr, int ntimes,
                              const double* counts, const int64_t* mptr, const int32_t* members,
                              const int32_t* perm, double* ll, int* status, cudaStream_t s) {
  csr_loglik_kernel<<<1, 1024, 0, s>>>(outp, precision, n, gptr, ntimes, counts, mptr, members, perm, ll, status);
  return cudaGetLastError();
}

}  // namespace mjp
