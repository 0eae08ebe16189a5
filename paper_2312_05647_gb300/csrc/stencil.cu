// stencil.cu -- persistent jump-chain kernels for the stencil rate models.
//
// One thread-block cluster per instance (theta).  The probability vector rho
// lives in shared memory for all K jumps: the cluster's C CTAs each own a
// contiguous slab of states, double-buffered (ping-pong), and read the few
// neighbour states outside their slab straight from the owning CTA's shared
// memory (distributed shared memory).  One cluster barrier per jump.
//
// Per jump (Algorithm 2's loop body, gather form of rho <- rho B):
//   y_n = rho_n (1 - e_n / Omega) + sum_{m -> n} rho_m lambda_{mn} / Omega,
// with the rates built matrix-free from theta (Eqs. BD_def, Gene_def and the
// mRNA/protein reactions), and the weighted accumulation
//   rho*_i += P_k rho_k   for every time i whose window [L_i, K_i] holds k,
// plus the tail (1 - sum P) at k = K_i.  The weights follow Algorithm 2's
// recurrence P_k = P_{k-1} x_i / k in FP64 (one lane per active time, one jump
// ahead), started from the planner's P_{L_i}.
//
// Modes: EXPV writes rho*(t_i) (FP32: Kahan-compensated, compensation in a
// global scratch buffer; FP64: plain), LOGLIK accumulates only the observed
// groups in shared memory and finishes with sum_g c_g log(a_g).
#include <cooperative_groups.h>

#include "internal.cuh"

namespace cg = cooperative_groups;

namespace mjp {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ void set_status(int* st, int code) {
  if (st) atomicCAS(st, 0, code);
}

// Scaled rate coefficients of one instance: rate / Omega in the chain type.
template <typename T>
struct Coef {
  T a, b, c, d;
};

template <typename T, int KIND>
__device__ __forceinline__ Coef<T> make_coef(const double* th, double omega) {
  Coef<T> k;
  double inv = omega > 0.0 ? 1.0 / omega : 0.0;
  k.a = (T)(th[0] * inv);
  k.b = (T)(th[1] * inv);
  if (KIND == MJP_BD1D) {
    k.c = (T)0;
    k.d = (T)0;
  } else {
    k.c = (T)(th[2] * inv);
    k.d = (T)(th[3] * inv);
  }
  return k;
}

// One gather-form jump for state n = m + M p; `nb(idx)` reads rho_k[idx].
// BD1D:     a = beta, b = gamma.
// TWOSTATE: a = beta, b = gamma, c = lambda_act, d = lambda_ina (p = sigma).
// MRNA:     a = k_m, b = gamma_m, c = k_p, d = gamma_p.
template <typename T, int KIND, typename NB>
__device__ __forceinline__ T jump(const Coef<T>& k, int64_t n, int64_t m, int64_t p, int64_t M,
                                  int64_t P, T self, NB nb) {
  const T one = (T)1;
  if (KIND == MJP_BD1D) {
    T e = (m >= 1 ? k.b * (T)m : (T)0) + (m + 1 < M ? k.a : (T)0);
    T y = (one - e) * self;
    if (m >= 1) y += k.a * nb(n - 1);
    if (m + 1 < M) y += k.b * (T)(m + 1) * nb(n + 1);
    return y;
  } else if (KIND == MJP_TWOSTATE) {
    if (p == 0) {
      T e = k.b * (T)m + (m + 1 < M ? k.a : (T)0) + k.d;
      T y = (one - e) * self;
      if (m >= 1) y += k.a * nb(n - 1);
      if (m + 1 < M) y += k.b * (T)(m + 1) * nb(n + 1);
      y += k.c * nb(n + M);  // inactive -> active
      return y;
    } else {
      T e = k.c + k.b * (T)m;
      T y = (one - e) * self;
      if (m + 1 < M) y += k.b * (T)(m + 1) * nb(n + 1);
      y += k.d * nb(n - M);  // active -> inactive
      return y;
    }
  } else {
    T e = k.d * (T)p + k.b * (T)m + (m + 1 < M ? k.a : (T)0) + (p + 1 < P ? k.c * (T)m : (T)0);
    T y = (one - e) * self;
    if (m >= 1) y += k.a * nb(n - 1);
    if (m + 1 < M) y += k.b * (T)(m + 1) * nb(n + 1);
    if (p >= 1) y += k.c * (T)m * nb(n - M);
    if (p + 1 < P) y += k.d * (T)(p + 1) * nb(n + M);
    return y;
  }
}

struct Smem {
  // Byte offsets of the pieces of dynamic shared memory.
  size_t buf1, tx, tPL, ttail, tL, tK, torig, pw, red, acc_s, acc_c, total;
};

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

__host__ __device__ inline Smem smem_layout(size_t elt, int64_t slab, int nt, int G, bool ll) {
  Smem s;
  size_t bufbytes = align_up((size_t)slab * elt, 16);
  s.buf1 = bufbytes;
  size_t o = 2 * bufbytes;
  s.tx = o; o += 8 * (size_t)nt;
  s.tPL = o; o += 8 * (size_t)nt;
  s.ttail = o; o += 8 * (size_t)nt;
  s.tL = o; o += 8 * (size_t)nt;
  s.tK = o; o += 8 * (size_t)nt;
  s.torig = o; o += align_up(4 * (size_t)nt, 8);
  s.pw = o; o += 16 * (size_t)nt;
  s.red = o; o += 8 * 2 * 33;
  s.acc_s = o;
  if (ll) {
    o += align_up(elt * (size_t)G, 8);
    s.acc_c = o;
    if (elt == 4) o += align_up(4 * (size_t)G, 8);
  } else {
    s.acc_c = o;
  }
  s.total = align_up(o, 16);
  return s;
}

template <typename T, int KIND, bool LL>
__global__ void __launch_bounds__(1024, 1) chain_kernel(ChainParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int job = blockIdx.x / C;
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = nthr >> 5;
  const int nt = p.ntimes;
  const int64_t N = p.N, M = p.M, P = p.P, S = p.slab;
  const int64_t n0 = (int64_t)rank * S;
  const int64_t n1 = (n0 + S < N) ? n0 + S : N;
  const int64_t nloc = n1 > n0 ? n1 - n0 : 0;

  const Smem L = smem_layout(sizeof(T), S, nt, p.G, LL);
  T* buf[2] = {reinterpret_cast<T*>(smem), reinterpret_cast<T*>(smem + L.buf1)};
  double* t_x = reinterpret_cast<double*>(smem + L.tx);
  double* t_PL = reinterpret_cast<double*>(smem + L.tPL);
  double* t_tail = reinterpret_cast<double*>(smem + L.ttail);
  long long* t_L = reinterpret_cast<long long*>(smem + L.tL);
  long long* t_K = reinterpret_cast<long long*>(smem + L.tK);
  int* t_orig = reinterpret_cast<int*>(smem + L.torig);
  double* pw = reinterpret_cast<double*>(smem + L.pw);   // [2][nt]
  double* red = reinterpret_cast<double*>(smem + L.red);  // [2][33]
  T* acc_s = reinterpret_cast<T*>(smem + L.acc_s);
  float* acc_c = reinterpret_cast<float*>(smem + L.acc_c);

  auto sync = [&]() {
    if (C == 1) __syncthreads();
    else cluster.sync();
  };

  // ---- prologue: instance data into shared memory -------------------------
  const Win* wj = p.win + (int64_t)job * nt;
  for (int i = tid; i < nt; i += nthr) {
    Win w = wj[i];
    t_x[i] = w.x;
    t_PL[i] = w.PL;
    t_tail[i] = w.tail;
    t_L[i] = w.L;
    t_K[i] = w.K;
    t_orig[i] = p.orig ? p.orig[i] : i;
    pw[i] = (w.L == 0) ? w.PL : 0.0;  // weights of jump 0
  }
  const double omega = p.info[job].omega;
  const int64_t Kmax = p.info[job].Kmax;
  const Coef<T> co = make_coef<T, KIND>(p.theta + (int64_t)job * p.ntheta, omega);
  const T* rho0 = reinterpret_cast<const T*>(p.rho0);
  T msum = (T)0;
  for (int64_t j = tid; j < nloc; j += nthr) {
    T v = rho0[n0 + j];
    buf[0][j] = v;
    msum += v;
  }
  if (LL) {
    for (int g = tid; g < p.G; g += nthr) {
      acc_s[g] = (T)0;
      if (sizeof(T) == 4) acc_c[g] = 0.0f;
    }
  }
  double mass0 = 1.0;
  if (p.renorm > 0) {
    double v = (double)msum;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if (lane == 0) red[warp] = v;
  }
  sync();
  if (p.renorm > 0) {
    double tot = 0.0;
    for (int r = 0; r < C; ++r) {
      const double* rr = (C == 1) ? red : cluster.map_shared_rank(red, r);
      for (int w = 0; w < nwarps; ++w) tot += rr[w];
    }
    mass0 = tot;
  }

  // Active window bookkeeping: times are sorted, so the times whose window
  // holds jump k form a contiguous range [lo, hi].
  int lo = 0, hi = -1;
  auto advance = [&](int64_t k, int& l, int& h) {
    while (l < nt && t_K[l] < k) ++l;
    while (h + 1 < nt && t_L[h + 1] <= k) ++h;
  };
  advance(0, lo, hi);

  // Per-thread state iteration: n = n0 + tid + j*nthr, (m, p) tracked.
  const int64_t dm = nthr % M, dp = nthr / M;
  int64_t m_start = (n0 + tid) % M, p_start = (n0 + tid) / M;

  // LOGLIK: add weight w times the group sums of rho_k (from `cur`).
  auto group_accumulate = [&](const T* cur, int l, int h, int64_t k, const double* wts) {
    for (int i = l; i <= h; ++i) {
      double wd = wts[i] + (k == t_K[i] ? t_tail[i] : 0.0);
      T w = (T)wd;
      int64_t g0 = p.gptr[i], g1 = p.gptr[i + 1];
      for (int64_t g = g0 + tid; g < g1; g += nthr) {
        T v = (T)0;
        bool any = false;
        for (int64_t q = p.mptr[g]; q < p.mptr[g + 1]; ++q) {
          int64_t s = p.members[q];
          if (s >= n0 && s < n1) {
            v += cur[s - n0];
            any = true;
          }
        }
        if (!any) continue;
        if (sizeof(T) == 4) {
          float y = (float)w * (float)v - acc_c[g];
          float t = (float)acc_s[g] + y;
          acc_c[g] = (t - (float)acc_s[g]) - y;
          acc_s[g] = (T)t;
        } else {
          acc_s[g] += w * v;
        }
      }
    }
  };

  double f_prev = 1.0;  // renormalisation factor carried onto rho_{k-1}
  if (LL) group_accumulate(buf[0], lo, hi, 0, pw);

  // ---- the jump chain -----------------------------------------------------
  for (int64_t k = 1; k <= Kmax + (LL ? 0 : 1); ++k) {
    const T* src = buf[(k - 1) & 1];
    T* dst = buf[k & 1];
    const double* wprev = pw + ((k - 1) & 1) * nt;
    double* wcur = pw + (k & 1) * nt;
    int plo = lo, phi = hi;  // active times of jump k-1
    int clo = lo, chi = hi;
    advance(k, clo, chi);    // active times of jump k
    // Weights of jump k, one lane per active time (Algorithm 2: P *= x/k).
    if (warp == 0 && k <= Kmax) {
      for (int i = clo + lane; i <= chi; i += 32) {
        wcur[i] = (k == t_L[i]) ? t_PL[i] : __dmul_rn(wprev[i], __ddiv_rn(t_x[i], (double)k));
      }
    }
    const T f = (T)f_prev;
    T part = (T)0;
    int64_t mm = m_start, pp = p_start;
    for (int64_t j = tid; j < nloc; j += nthr) {
      const int64_t n = n0 + j;
      T r = src[j];
      if (!LL) {
        // EXPV: accumulate rho_{k-1} (fused with the read of the jump).
        const int64_t kp = k - 1;
        T rv = r * f;
        for (int i = plo; i <= phi; ++i) {
          double wd = wprev[i] + (kp == t_K[i] ? t_tail[i] : 0.0);
          T w = (T)wd;
          int64_t base = (int64_t)job * p.out_stride + (int64_t)t_orig[i] * N + n;
          T* o = reinterpret_cast<T*>(p.out) + base;
          if (sizeof(T) == 4) {
            float* c = p.comp + (int64_t)job * p.comp_stride + (int64_t)i * N + n;
            float s, cc;
            if (kp == t_L[i]) {
              s = (float)w * (float)rv;
              cc = 0.0f;
            } else {
              s = (float)*o;
              cc = *c;
              float y = (float)w * (float)rv - cc;
              float t = s + y;
              cc = (t - s) - y;
              s = t;
            }
            if (kp == t_K[i]) *o = (T)(s - cc);
            else {
              *o = (T)s;
              *c = cc;
            }
          } else {
            if (kp == t_L[i]) *o = w * rv;
            else *o += w * rv;
          }
        }
      }
      if (k <= Kmax) {
        auto nb = [&](int64_t idx) -> T {
          int64_t li = idx - n0;
          if (li >= 0 && li < S) return src[li];
          int owner = (int)(idx / S);
          const T* rs = cluster.map_shared_rank(src, owner);
          return rs[idx - (int64_t)owner * S];
        };
        T y = jump<T, KIND>(co, n, mm, pp, M, P, r, nb);
        if (p.renorm > 0) {
          y *= f;
          part += y;
        }
        dst[j] = y;
      }
      mm += dm;
      pp += dp;
      if (mm >= M) {
        mm -= M;
        pp += 1;
      }
    }
    const bool do_renorm = p.renorm > 0 && k <= Kmax && (k % p.renorm) == 0;
    double* redk = red + (k & 1) * 33;
    if (do_renorm) {
      double v = (double)part;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
      if (lane == 0) redk[warp] = v;
    }
    sync();
    lo = clo;
    hi = chi;
    if (k > Kmax) break;
    f_prev = 1.0;
    if (do_renorm) {
      double tot = 0.0;
      for (int r = 0; r < C; ++r) {
        const double* rr = (C == 1) ? redk : cluster.map_shared_rank(redk, r);
        for (int w = 0; w < nwarps; ++w) tot += rr[w];
      }
      f_prev = tot > 0.0 ? mass0 / tot : 1.0;
    } else if (p.renorm > 0) {
      f_prev = 1.0;
    }
    if (LL) {
      if (f_prev != 1.0) {
        // Apply the factor to rho_k in place before it is read again.
        for (int64_t j = tid; j < nloc; j += nthr) dst[j] = (T)(dst[j] * (T)f_prev);
        f_prev = 1.0;
        sync();
      }
      group_accumulate(dst, lo, hi, k, wcur);
    }
  }

  if (LL) {
    // ---- epilogue: sum_g c_g log(a_g), partial sums of all CTAs ------------
    sync();
    if (rank == 0) {
      double ll = 0.0;
      bool bad = false;
      for (int g = tid; g < p.G; g += nthr) {
        double a = 0.0;
        for (int r = 0; r < C; ++r) {
          const T* rs = (C == 1) ? acc_s : cluster.map_shared_rank(acc_s, r);
          double v = (double)rs[g];
          if (sizeof(T) == 4) {
            const float* rc = (C == 1) ? acc_c : cluster.map_shared_rank(acc_c, r);
            v -= (double)rc[g];
          }
          a += v;
        }
        double c = p.counts[g];
        if (c == 0.0) continue;
        if (a > 0.0) ll += c * log(a);
        else if (a == 0.0 || a > -1e-30) ll = -INFINITY;
        else bad = true;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ll += __shfl_xor_sync(kFull, ll, o);
      __syncthreads();
      if (lane == 0) red[warp] = ll;
      __syncthreads();
      if (tid == 0) {
        double tot = 0.0;
        for (int w = 0; w < nwarps; ++w) tot += red[w];
        if (isnan(tot)) set_status(p.status, kStatusNumeric);
        p.ll[job] = tot;
      }
      if (bad) set_status(p.status, kStatusNumeric);
    }
    sync();  // keep every CTA's shared memory alive until rank 0 is done
  }
}

template <typename T, int KIND, bool LL>
cudaError_t launch_typed(const ChainParams& p, int cluster, int threads, cudaStream_t s) {
  size_t smem = smem_layout(sizeof(T), p.slab, p.ntimes, p.G, LL).total;
  auto kern = chain_kernel<T, KIND, LL>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (cluster > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(p.B * cluster), 1, 1);
  cfg.blockDim = dim3((unsigned)threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, p);
}

template <typename T, bool LL>
cudaError_t launch_kind(int kind, const ChainParams& p, int cluster, int threads, cudaStream_t s) {
  switch (kind) {
    case MJP_BD1D: return launch_typed<T, MJP_BD1D, LL>(p, cluster, threads, s);
    case MJP_TWOSTATE: return launch_typed<T, MJP_TWOSTATE, LL>(p, cluster, threads, s);
    case MJP_MRNA_PROT2D: return launch_typed<T, MJP_MRNA_PROT2D, LL>(p, cluster, threads, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int KIND, bool LL>
int max_clusters_typed(int cluster, int threads, size_t smem) {
  auto kern = chain_kernel<T, KIND, LL>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  if (cluster > 8) cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)cluster, 1, 1);
  cfg.blockDim = dim3((unsigned)threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace

size_t chain_stencil_smem(int precision, int loglik_mode, int64_t slab, int ntimes, int G) {
  return smem_layout(precision == MJP_FP64 ? 8 : 4, slab, ntimes, G, loglik_mode != 0).total;
}

cudaError_t launch_chain_stencil(int kind, int precision, int loglik_mode, const ChainParams& p,
                                 int cluster, int threads, cudaStream_t s) {
  if (p.B <= 0) return cudaSuccess;
  if (precision == MJP_FP64) {
    return loglik_mode ? launch_kind<double, true>(kind, p, cluster, threads, s)
                       : launch_kind<double, false>(kind, p, cluster, threads, s);
  }
  return loglik_mode ? launch_kind<float, true>(kind, p, cluster, threads, s)
                     : launch_kind<float, false>(kind, p, cluster, threads, s);
}

int chain_stencil_max_cluster_blocks(int kind, int precision, int loglik_mode, int cluster,
                                     int threads, size_t smem) {
  bool ll = loglik_mode != 0;
  if (precision == MJP_FP64) {
    switch (kind) {
      case MJP_BD1D: return ll ? max_clusters_typed<double, MJP_BD1D, true>(cluster, threads, smem) : max_clusters_typed<double, MJP_BD1D, false>(cluster, threads, smem);
      case MJP_TWOSTATE: return ll ? max_clusters_typed<double, MJP_TWOSTATE, true>(cluster, threads, smem) : max_clusters_typed<double, MJP_TWOSTATE, false>(cluster, threads, smem);
      default: return ll ? max_clusters_typed<double, MJP_MRNA_PROT2D, true>(cluster, threads, smem) : max_clusters_typed<double, MJP_MRNA_PROT2D, false>(cluster, threads, smem);
    }
  }
  switch (kind) {
    case MJP_BD1D: return ll ? max_clusters_typed<float, MJP_BD1D, true>(cluster, threads, smem) : max_clusters_typed<float, MJP_BD1D, false>(cluster, threads, smem);
    case MJP_TWOSTATE: return ll ? max_clusters_typed<float, MJP_TWOSTATE, true>(cluster, threads, smem) : max_clusters_typed<float, MJP_TWOSTATE, false>(cluster, threads, smem);
    default: return ll ? max_clusters_typed<float, MJP_MRNA_PROT2D, true>(cluster, threads, smem) : max_clusters_typed<float, MJP_MRNA_PROT2D, false>(cluster, threads, smem);
  }
}

}  // namespace mjp
