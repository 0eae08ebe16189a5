// jmjp.cu -- J-MJP state probabilities (Method #2 of the paper, Sec. 2.2.2,
// Algorithm 1): phi_i = sum over observation i's group of (rho0 B^{k_i}), one
// chain rho0 B^k read at every observation's own number of virtual jumps.
//
// One CTA evolves the chain for one theta with rho double-buffered in shared
// memory (birth-death and two-state models, the paper's J-MJP examples).  The
// observations arrive sorted by k and cut into chunks that fit the rest of
// shared memory (jump counts, caller positions, group offsets and members);
// a chunk is copied in once, so the reads of jump k touch only shared memory.
// One warp walks the sorted observations (a ballot finds those with k_i = k)
// and sums their groups (FP64) from rho_k while the other warps form
// rho_{k+1}; one CTA barrier per jump.
#include "chain_common.cuh"
#include "internal.cuh"

namespace mjp {

namespace {

constexpr size_t kJmjpSmem = 227 * 1024 - 1024;  // dynamic shared memory per CTA at most

__host__ __device__ inline size_t jmjp_rho_bytes(int N, size_t elt) { return align_up(2 * elt * (size_t)N, 16); }

// Threads [0, nupd) update the chain (R > 0: each holds the coefficients of
// its R states in registers, N <= R x nupd; R = 0 rebuilds them at every
// jump); the last warp reads the observations of each jump and loads later
// chunks, so those reads run beside the update instead of before it.
template <typename T, int KIND, int R>
__global__ void __launch_bounds__(1024, 1) jmjp_kernel(const JmjpParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  T* const buf0 = reinterpret_cast<T*>(smem);
  T* const buf1 = buf0 + p.N;
  int32_t* const s_k = reinterpret_cast<int32_t*>(smem + jmjp_rho_bytes(p.N, sizeof(T)));
  int32_t* const s_ord = s_k + p.cap_obs;
  int32_t* const s_gp = s_ord + p.cap_obs;
  int32_t* const s_mem = s_gp + p.cap_obs + 1;
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31;
  const int nupd = nthr - 32;
  const bool reader = tid >= nupd;
  const int N = p.N, NR = p.M;
  const double inv = p.omega > 0.0 ? 1.0 / p.omega : 0.0;
  const T b = (T)(p.theta[0] * inv), g = (T)(p.theta[1] * inv);
  const T la = KIND == MJP_TWOSTATE ? (T)(p.theta[2] * inv) : (T)0;
  const T li = KIND == MJP_TWOSTATE ? (T)(p.theta[3] * inv) : (T)0;
  const T one = (T)1;
  // Coefficients of state n in the gather form of rho B: y_n = d_n rho_n +
  // b rho_{n-1} + g_n rho_{n+1} (+ s rho_sw, the other gene state), built once
  // (the same operations as Eq. B_def's entries) and reused at every jump.
  struct Cf {
    T d, b, g, s;
    int lo, hi, sw;
  };
  auto coef = [&](int n) {
    Cf c;
    if (KIND == MJP_BD1D) {
      const T fn = (T)n;
      c.d = f_sub(one, f_add(f_mul(g, fn), n + 1 < N ? b : (T)0));
      c.b = b;
      c.lo = n >= 1 ? n - 1 : -1;
      c.g = n + 1 < N ? f_mul(g, f_add(fn, one)) : (T)0;
      c.hi = n + 1 < N ? n + 1 : -1;
      c.s = (T)0;
      c.sw = n;
    } else {  // two-state: n = n_R + sigma N_R, sigma 0 active
      const int sg = n >= NR ? 1 : 0, r = n - sg * NR;
      const T fr = (T)r;
      const T e = sg == 0 ? f_add(f_add(f_mul(g, fr), r + 1 < NR ? b : (T)0), li) : f_add(la, f_mul(g, fr));
      c.d = f_sub(one, e);
      c.b = b;
      c.lo = (sg == 0 && r >= 1) ? n - 1 : -1;                 // birth from r-1
      c.g = r + 1 < NR ? f_mul(g, f_add(fr, one)) : (T)0;      // death from r+1
      c.hi = r + 1 < NR ? n + 1 : -1;
      c.s = sg == 0 ? la : li;                                 // switching in
      c.sw = sg == 0 ? n + NR : n - NR;
    }
    return c;
  };
  Cf cf[R > 0 ? R : 1];
  if (!reader) {
#pragma unroll
    for (int j = 0; j < (R > 0 ? R : 1); ++j) cf[j] = coef(min(tid + j * nupd, N - 1));
  }
  for (int n = tid; n < N; n += nthr) buf0[n] = reinterpret_cast<const T*>(p.rho0)[n];
  // Chunk c: sorted observations [chunk[c], chunk[c+1]) and their members,
  // copied by threads [t0, t0 + nt) (the whole CTA for chunk 0, later the reader).
  auto load_chunk = [&](int cc, int t0, int nt) {
    const int o0 = p.chunk[cc], o1 = p.chunk[cc + 1];
    const int m0 = p.group_ptr[o0], m1 = p.group_ptr[o1];
    for (int i = tid - t0; i < o1 - o0; i += nt) {
      s_k[i] = p.ksorted[o0 + i];
      s_ord[i] = p.order[o0 + i];
    }
    for (int i = tid - t0; i <= o1 - o0; i += nt) s_gp[i] = p.group_ptr[o0 + i] - m0;
    for (int i = tid - t0; i < m1 - m0; i += nt) s_mem[i] = p.members[m0 + i];
    return o1 - o0;
  };
  int c = 0, lp = 0;
  int cn = load_chunk(0, 0, nthr);
  __syncthreads();
  for (int k = 0; k <= p.kmax; ++k) {
    const T* cur = (k & 1) ? buf1 : buf0;
    if (reader) {
      // Observations with k_i = k: a prefix of the rest of the sorted list.
      for (;;) {
        if (lp == cn && c + 1 < p.nchunks) {
          __syncwarp();  // the reader's reads of the old chunk are done
          cn = load_chunk(++c, nupd, 32);
          lp = 0;
          __syncwarp();
        }
        int hi = lp;
        for (;;) {
          const int idx = hi + lane;
          const unsigned bal = __ballot_sync(kFull, idx < cn && s_k[idx] == k);
          const int run = bal == kFull ? 32 : __ffs(~bal) - 1;
          hi += run;
          if (run < 32) break;
        }
        for (int o = lp + lane; o < hi; o += 32) {
          double v = 0.0;
          for (int q = s_gp[o]; q < s_gp[o + 1]; ++q) v += (double)cur[s_mem[q]];
          p.phi[s_ord[o]] = v;
        }
        lp = hi;
        if (lp < cn || c + 1 >= p.nchunks) break;
      }
    } else if (k < p.kmax) {
      // rho <- rho B (gather form, rates into n scaled by 1/Omega).
      T* nxt = (k & 1) ? buf0 : buf1;
      if (R > 0) {
#pragma unroll
        for (int j = 0; j < (R > 0 ? R : 1); ++j) {
          const int n = tid + j * nupd;
          if (n < N) {
            T y = f_mul(cf[j].d, cur[n]);
            if (cf[j].lo >= 0) y = f_fma(cf[j].b, cur[cf[j].lo], y);
            if (cf[j].hi >= 0) y = f_fma(cf[j].g, cur[cf[j].hi], y);
            if (KIND == MJP_TWOSTATE) y = f_fma(cf[j].s, cur[cf[j].sw], y);
            nxt[n] = y;
          }
        }
      } else {
        for (int n = tid; n < N; n += nupd) {
          const Cf cc = coef(n);
          T y = f_mul(cc.d, cur[n]);
          if (cc.lo >= 0) y = f_fma(cc.b, cur[cc.lo], y);
          if (cc.hi >= 0) y = f_fma(cc.g, cur[cc.hi], y);
          if (KIND == MJP_TWOSTATE) y = f_fma(cc.s, cur[cc.sw], y);
          nxt[n] = y;
        }
      }
    }
    __syncthreads();
  }
}

template <typename T, int KIND>
cudaError_t launch_jmjp_typed(const JmjpParams& p, cudaStream_t s) {
  const size_t smem = jmjp_rho_bytes(p.N, sizeof(T)) + 4 * (3 * (size_t)p.cap_obs + 1 + (size_t)p.cap_mem);
  if (smem > kJmjpSmem) return cudaErrorInvalidValue;
  const int nupd = p.N >= 992 ? 992 : (p.N + 31) / 32 * 32;  // updaters; one more warp reads
  auto kern = p.N <= nupd ? jmjp_kernel<T, KIND, 1> : p.N <= 4 * nupd ? jmjp_kernel<T, KIND, 4> : jmjp_kernel<T, KIND, 0>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kJmjpSmem);
  if (e != cudaSuccess) return e;
  kern<<<1, nupd + 32, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

// Leaves room for chunks of at least 256 observations of 4 members.
int64_t jmjp_max_states(int precision) {
  const size_t elt = precision == MJP_FP64 ? 8 : 4;
  return (int64_t)((kJmjpSmem - 4 * (3 * 256 + 1 + 1024)) / (2 * elt)) / 4 * 4;
}

size_t jmjp_chunk_bytes(int precision, int N) {
  const size_t used = jmjp_rho_bytes(N, precision == MJP_FP64 ? 8 : 4);
  return used < kJmjpSmem ? kJmjpSmem - used : 0;
}

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
