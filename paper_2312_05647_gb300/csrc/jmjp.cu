// jmjp.cu -- J-MJP state probabilities (Method #2 of the paper, Sec. 2.2.2,
// Algorithm 1): phi_i = sum over observation i's group of (rho0 B^{k_i}), one
// chain rho0 B^k read at every observation's own number of virtual jumps.
//
// One CTA evolves the chain for one theta with rho double-buffered in shared
// memory (birth-death and two-state models, the paper's J-MJP examples).  The
// observations arrive sorted by k; after jump k every thread advances the same
// pointer over the observations with k_i = k and the CTA reads their groups
// (state-parallel sums from shared memory) before the next jump.
#include "chain_common.cuh"
#include "internal.cuh"

namespace mjp {

namespace {

template <typename T, int KIND>
__global__ void __launch_bounds__(1024, 1) jmjp_kernel(const JmjpParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  T* const buf0 = reinterpret_cast<T*>(smem);
  T* const buf1 = buf0 + p.N;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int N = p.N, NR = p.M;
  const double inv = p.omega > 0.0 ? 1.0 / p.omega : 0.0;
  const T b = (T)(p.theta[0] * inv), g = (T)(p.theta[1] * inv);
  const T la = KIND == MJP_TWOSTATE ? (T)(p.theta[2] * inv) : (T)0;
  const T li = KIND == MJP_TWOSTATE ? (T)(p.theta[3] * inv) : (T)0;
  const T one = (T)1;
  for (int n = tid; n < N; n += nthr) buf0[n] = reinterpret_cast<const T*>(p.rho0)[n];
  __syncthreads();
  int64_t ptr = 0;
  for (int64_t k = 0;; ++k) {
    const T* cur = (k & 1) ? buf1 : buf0;
    // Observations with k_i = k, in sorted order.
    int64_t hi = ptr;
    while (hi < p.nobs && p.ksorted[hi] == k) ++hi;
    for (int64_t o = ptr + tid; o < hi; o += nthr) {
      double v = 0.0;
      for (int64_t q = p.group_ptr[o]; q < p.group_ptr[o + 1]; ++q) v += (double)cur[p.members[q]];
      p.phi[p.order[o]] = v;
    }
    ptr = hi;
    if (ptr >= p.nobs) break;
    // rho <- rho B (gather form, rates into n scaled by 1/Omega).
    T* nxt = (k & 1) ? buf0 : buf1;
    for (int n = tid; n < N; n += nthr) {
      T y;
      if (KIND == MJP_BD1D) {
        const T fn = (T)n;
        const T e = f_add(f_mul(g, fn), n + 1 < N ? b : (T)0);
        y = f_mul(f_sub(one, e), cur[n]);
        if (n >= 1) y = f_fma(b, cur[n - 1], y);
        if (n + 1 < N) y = f_fma(f_mul(g, f_add(fn, one)), cur[n + 1], y);
      } else {  // two-state: n = n_R + sigma N_R, sigma 0 active
        const int sg = n >= NR ? 1 : 0, r = n - sg * NR;
        const T fr = (T)r;
        const T e = sg == 0 ? f_add(f_add(f_mul(g, fr), r + 1 < NR ? b : (T)0), li) : f_add(la, f_mul(g, fr));
        y = f_mul(f_sub(one, e), cur[n]);
        if (sg == 0 && r >= 1) y = f_fma(b, cur[n - 1], y);                        // birth from r-1
        if (r + 1 < NR) y = f_fma(f_mul(g, f_add(fr, one)), cur[n + 1], y);        // death from r+1
        y = f_fma(sg == 0 ? la : li, cur[sg == 0 ? n + NR : n - NR], y);           // switching in
      }
      nxt[n] = y;
    }
    __syncthreads();
  }
}

template <typename T, int KIND>
cudaError_t launch_jmjp_typed(const JmjpParams& p, cudaStream_t s) {
  const size_t smem = 2 * sizeof(T) * (size_t)p.N;
  auto kern = jmjp_kernel<T, KIND>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int threads = p.N >= 1024 ? 1024 : (p.N + 31) / 32 * 32;
  kern<<<1, threads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

int64_t jmjp_max_states(int precision) { return (int64_t)(227 * 1024 - 1024) / (2 * (precision == MJP_FP64 ? 8 : 4)); }

cudaError_t launch_jmjp(int kind, int precision, const JmjpParams& p, cudaStream_t s) {
  if (p.nobs <= 0) return cudaSuccess;
  if (kind == MJP_BD1D)
    return precision == MJP_FP64 ? launch_jmjp_typed<double, MJP_BD1D>(p, s) : launch_jmjp_typed<float, MJP_BD1D>(p, s);
  if (kind == MJP_TWOSTATE)
    return precision == MJP_FP64 ? launch_jmjp_typed<double, MJP_TWOSTATE>(p, s)
                                 : launch_jmjp_typed<float, MJP_TWOSTATE>(p, s);
  return cudaErrorInvalidValue;
}

}  // namespace mjp
