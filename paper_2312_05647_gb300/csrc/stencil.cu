// stencil.cu -- persistent jump-chain kernels for the stencil rate models.
//
// One thread-block cluster per instance (theta).  The probability vector rho
// lives in shared memory for all K jumps.  States are laid out as rows of M
// (n = m + M p); each CTA of the cluster owns a contiguous slab -- whole rows
// for the two-dimensional models, a run of columns for the birth-death chain
// -- stored double-buffered (ping-pong) with a ring of zero padding, so that
// interior stencil reads need no bounds checks.  Rows or columns just outside
// a slab are read straight from the neighbouring CTA's shared memory
// (distributed shared memory).  One CTA barrier and, for clusters, one split
// cluster barrier (arrive ... wait) per jump.
//
// Thread layout: thread (tx, ty) owns column m = tx (+ multiples of TX when
// the slab is wider than the CTA) and a contiguous run of rows, walked with a
// sliding window (down, cur, up) so every value is loaded once per jump.  The
// rate coefficients of a column are built matrix-free from theta (Eqs.
// BD_def, Gene_def, the mRNA/protein reactions) once per column.
//
// Per jump (Algorithm 2's loop body, gather form of rho <- rho B):
//   y_n = rho_n (1 - e_n / Omega) + sum_{m -> n} rho_m lambda_{mn} / Omega,
// then the weighted accumulation rho*_i += P_k rho_k for every time i whose
// window [L_i, K_i] holds k, plus the tail (1 - sum P) at k = K_i.  The
// weights follow Algorithm 2's recurrence P_k = P_{k-1} x_i / k in FP64 (one
// lane per active time, one jump ahead), started from the planner's P_{L_i}.
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

__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Local tile geometry of one CTA: a padded (rows + 2) x (width + 2) array.
struct Geo {
  int p0, p1, m0, m1;  // owned rows [p0, p1) and columns [m0, m1)
  int W, H;            // width and height of the owned block
  int Wp;              // padded row stride (W + 2)
  int size;            // padded elements ((H + 2) * Wp)
};

__host__ __device__ inline Geo geometry(int kind, int M, int P, int N, int slab, int rank) {
  Geo g;
  int n0 = rank * slab;
  int n1 = n0 + slab < N ? n0 + slab : N;
  if (n1 < n0) n1 = n0;
  if (kind == MJP_BD1D) {
    g.p0 = 0; g.p1 = 1; g.m0 = n0; g.m1 = n1;
  } else {  // slab is a whole number of rows
    g.p0 = n0 / M; g.p1 = (n1 + M - 1) / M; g.m0 = 0; g.m1 = M;
    if (g.p1 < g.p0) g.p1 = g.p0;
  }
  g.W = g.m1 - g.m0;
  g.H = g.p1 - g.p0;
  g.Wp = g.W + 2;
  // The birth-death chain has no vertical neighbours: no pad rows.
  g.size = (kind == MJP_BD1D) ? g.Wp : (g.H + 2) * g.Wp;
  return g;
}

// Padded-row offset of owned row 0 in the local tile.
template <int KIND>
__device__ __forceinline__ int row_off() {
  return KIND == MJP_BD1D ? 0 : 1;
}

// Largest padded tile over the ranks of a cluster (rank 0 is never smaller).
__host__ __device__ inline int tile_elems(int kind, int M, int P, int N, int slab) {
  Geo g = geometry(kind, M, P, N, slab, 0);
  return g.size;
}

struct Smem {
  size_t buf1, tx, tPL, ttail, tL, tK, torig, pw, red, memloc, acc_s, acc_c, total;
};

__host__ __device__ inline Smem smem_layout(size_t elt, int tile, int nt, int G, int nmem, bool ll) {
  Smem s;
  size_t bufbytes = align_up((size_t)tile * elt, 16);
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
  s.memloc = o;
  if (ll) o += align_up(4 * (size_t)nmem, 8);
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

// Scaled rates (rate / Omega) of one instance in the chain type.
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
  k.c = (KIND == MJP_BD1D) ? (T)0 : (T)(th[2] * inv);
  k.d = (KIND == MJP_BD1D) ? (T)0 : (T)(th[3] * inv);
  return k;
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
  const int M = p.M, P = p.P, N = (int)p.N, S = (int)p.slab;
  const Geo g = geometry(KIND, M, P, N, S, rank);
  const int tile = tile_elems(KIND, M, P, N, S);

  const Smem L = smem_layout(sizeof(T), tile, nt, p.G, p.nmem, LL);
  T* buf[2] = {reinterpret_cast<T*>(smem), reinterpret_cast<T*>(smem + L.buf1)};
  double* t_x = reinterpret_cast<double*>(smem + L.tx);
  double* t_PL = reinterpret_cast<double*>(smem + L.tPL);
  double* t_tail = reinterpret_cast<double*>(smem + L.ttail);
  long long* t_L = reinterpret_cast<long long*>(smem + L.tL);
  long long* t_K = reinterpret_cast<long long*>(smem + L.tK);
  int* t_orig = reinterpret_cast<int*>(smem + L.torig);
  double* pw = reinterpret_cast<double*>(smem + L.pw);   // [2][nt]
  double* red = reinterpret_cast<double*>(smem + L.red);  // [2][33]
  int* memloc = reinterpret_cast<int*>(smem + L.memloc);
  T* acc_s = reinterpret_cast<T*>(smem + L.acc_s);
  float* acc_c = reinterpret_cast<float*>(smem + L.acc_c);

  // Remote tiles of the neighbouring CTAs (same layout, same offsets).
  const T* up_rem[2] = {nullptr, nullptr};
  const T* dn_rem[2] = {nullptr, nullptr};
  int up_W = 0, dn_W = 0, dn_H = 0;
  if (C > 1) {
    if (rank + 1 < C) {
      up_rem[0] = cluster.map_shared_rank(buf[0], rank + 1);
      up_rem[1] = cluster.map_shared_rank(buf[1], rank + 1);
      up_W = geometry(KIND, M, P, N, S, rank + 1).Wp;
    }
    if (rank > 0) {
      dn_rem[0] = cluster.map_shared_rank(buf[0], rank - 1);
      dn_rem[1] = cluster.map_shared_rank(buf[1], rank - 1);
      Geo gd = geometry(KIND, M, P, N, S, rank - 1);
      dn_W = gd.Wp;
      dn_H = gd.H;
    }
  }

  // ---- prologue ------------------------------------------------------------
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
  for (int j = tid; j < 2 * tile; j += nthr) (j < tile ? buf[0] : buf[1])[j < tile ? j : j - tile] = (T)0;
  __syncthreads();
  T msum = (T)0;
  for (int j = tid; j < g.W * g.H; j += nthr) {
    int r = j / g.W, c = j - r * g.W;
    int gi = (g.p0 + r) * M + g.m0 + c;
    T v = rho0[gi];
    buf[0][(r + row_off<KIND>()) * g.Wp + c + 1] = v;
    msum += v;
  }
  if (LL) {
    for (int q = tid; q < p.nmem; q += nthr) {
      int s = p.members[q];
      int ps = s / M, ms = s - ps * M;
      bool mine = ps >= g.p0 && ps < g.p1 && ms >= g.m0 && ms < g.m1;
      memloc[q] = mine ? (ps - g.p0 + row_off<KIND>()) * g.Wp + (ms - g.m0) + 1 : -1;
    }
    for (int q = tid; q < p.G; q += nthr) {
      acc_s[q] = (T)0;
      if (sizeof(T) == 4) acc_c[q] = 0.0f;
    }
  }
  double mass0 = 1.0;
  if (p.renorm > 0) {
    double v = (double)msum;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    if (lane == 0) red[warp] = v;
  }
  if (C > 1) cluster.sync();
  else __syncthreads();
  if (p.renorm > 0) {
    double tot = 0.0;
    for (int r = 0; r < C; ++r) {
      const double* rr = (C == 1) ? red : cluster.map_shared_rank(red, r);
      for (int w = 0; w < nwarps; ++w) tot += rr[w];
    }
    mass0 = tot;
  }

  // Active times of jump k form a contiguous range [lo, hi] (times sorted).
  int lo = 0, hi = -1;
  auto advance = [&](int64_t k, int& l, int& h) {
    while (l < nt && t_K[l] < k) ++l;
    while (h + 1 < nt && t_L[h + 1] <= k) ++h;
  };
  advance(0, lo, hi);

  // LOGLIK: acc_g += w_i * sum_{s in g} rho_k[s] over this CTA's states.
  auto group_accumulate = [&](const T* cur, int l, int h, int64_t k, const double* wts) {
    for (int i = l; i <= h; ++i) {
      double wd = wts[i] + (k == t_K[i] ? t_tail[i] : 0.0);
      T w = (T)wd;
      int g0 = (int)p.gptr[i], g1 = (int)p.gptr[i + 1];
      for (int gq = g0 + tid; gq < g1; gq += nthr) {
        int q0 = (int)p.mptr[gq], q1 = (int)p.mptr[gq + 1];
        T v = (T)0;
        bool any = false;
        for (int q = q0; q < q1; ++q) {
          int li = memloc[q];
          if (li >= 0) {
            v += cur[li];
            any = true;
          }
        }
        if (!any) continue;
        if (sizeof(T) == 4) {
          float y = (float)w * (float)v - acc_c[gq];
          float t = (float)acc_s[gq] + y;
          acc_c[gq] = (t - (float)acc_s[gq]) - y;
          acc_s[gq] = (T)t;
        } else {
          acc_s[gq] += w * v;
        }
      }
    }
  };

  // Thread layout over the owned block.
  const int TX = g.W < nthr ? (g.W > 0 ? g.W : 1) : nthr;
  const int TY = nthr / TX;
  const int tx = tid % TX, ty = tid / TX;
  const int R = (g.H + TY - 1) / TY;
  const int ra = g.p0 + ty * R;
  const int rb = (ty < TY) ? min(g.p1, ra + R) : ra;
  const T one = (T)1;

  double f_prev = 1.0;  // renormalisation factor carried onto rho_{k-1}
  if (LL) group_accumulate(buf[0], lo, hi, 0, pw);

  // ---- the jump chain -----------------------------------------------------
  for (int64_t k = 1; k <= Kmax + (LL ? 0 : 1); ++k) {
    const int par = (int)((k - 1) & 1);
    const T* src = buf[par];
    T* dst = buf[par ^ 1];
    const double* wprev = pw + par * nt;
    double* wcur = pw + (par ^ 1) * nt;
    const int plo = lo, phi = hi;
    int clo = lo, chi = hi;
    advance(k, clo, chi);
    if (warp == 0 && k <= Kmax) {  // weights of jump k (Algorithm 2: P *= x/k)
      for (int i = clo + lane; i <= chi; i += 32)
        wcur[i] = (k == t_L[i]) ? t_PL[i] : __dmul_rn(wprev[i], __ddiv_rn(t_x[i], (double)k));
    }
    const T f = (T)f_prev;
    const bool jump = k <= Kmax;
    T part = (T)0;
    for (int m = g.m0 + tx; m < g.m1; m += TX) {
      const int lc = m - g.m0 + 1;  // local column (padded)
      // Column coefficients (scaled rates into this column's states).
      T cl, cr, cd, cu, ebase;
      if (KIND == MJP_BD1D) {
        cl = co.a;                                   // birth from m-1
        cr = co.b * (T)(m + 1);                      // death from m+1
        cd = (T)0;
        cu = (T)0;
        ebase = co.b * (T)m + (m + 1 < M ? co.a : (T)0);
      } else if (KIND == MJP_TWOSTATE) {
        cl = co.a;                                   // birth (active row only)
        cr = co.b * (T)(m + 1);                      // death from m+1
        cd = co.d;                                   // row 1 <- row 0 at lambda_ina
        cu = co.c;                                   // row 0 <- row 1 at lambda_act
        ebase = co.b * (T)m;
      } else {
        cl = co.a;                                   // k_m from m-1
        cr = co.b * (T)(m + 1);                      // gamma_m (m+1) from m+1
        cd = co.c * (T)m;                            // k_p m from p-1
        cu = (T)0;                                   // gamma_p (p+1), per row
        ebase = co.b * (T)m + (m + 1 < M ? co.a : (T)0) + co.c * (T)m;
      }
      // Left/right neighbours outside a column slab (birth-death clusters).
      T left_rem = (T)0, right_rem = (T)0;
      if (KIND == MJP_BD1D && C > 1 && jump) {
        // A neighbour's tile is one padded row: its last owned column sits at
        // Wp - 2, its first at 1.
        if (m == g.m0 && m >= 1 && dn_rem[par]) left_rem = dn_rem[par][dn_W - 2];
        if (m == g.m1 - 1 && m + 1 < M && up_rem[par]) right_rem = up_rem[par][1];
      }
      int li = (ra - g.p0 + row_off<KIND>()) * g.Wp + lc;
      T down = (T)0;
      if (KIND != MJP_BD1D && ra < rb && ra >= 1) {
        if (ra - 1 >= g.p0) down = src[li - g.Wp];
        else if (dn_rem[par]) down = dn_rem[par][dn_H * dn_W + lc];  // last owned row of rank-1
      }
      T cur = (ra < rb) ? src[li] : (T)0;
      for (int pp = ra; pp < rb; ++pp, li += g.Wp) {
        T up = (T)0;
        if (KIND != MJP_BD1D && pp + 1 < P) {
          if (pp + 1 < g.p1) up = src[li + g.Wp];
          else if (up_rem[par]) up = up_rem[par][g.Wp + lc];  // first owned row of rank+1
        }
        T left = src[li - 1], right = src[li + 1];
        if (KIND == MJP_BD1D && C > 1) {
          if (m == g.m0) left = left_rem;
          if (m == g.m1 - 1) right = right_rem;
        }
        if (!LL) {
          // EXPV: accumulate rho_{k-1} (its value is `cur`).
          const int64_t kp = k - 1;
          const T rv = cur * f;
          const int64_t gidx = (int64_t)pp * M + m;
          for (int i = plo; i <= phi; ++i) {
            double wd = wprev[i] + (kp == t_K[i] ? t_tail[i] : 0.0);
            T w = (T)wd;
            T* o = reinterpret_cast<T*>(p.out) + (int64_t)job * p.out_stride + (int64_t)t_orig[i] * N + gidx;
            if (sizeof(T) == 4) {
              float* c = p.comp + (int64_t)job * p.comp_stride + (int64_t)i * N + gidx;
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
        if (jump) {
          T y;
          if (KIND == MJP_BD1D) {
            y = (one - ebase) * cur + cl * left + cr * right;
          } else if (KIND == MJP_TWOSTATE) {
            if (pp == 0) {  // active: births, deaths, reactivation from row 1
              T e = ebase + (m + 1 < M ? co.a : (T)0) + co.d;
              y = (one - e) * cur + cl * left + cr * right + cu * up;
            } else {        // inactive: deaths, deactivation from row 0
              T e = ebase + co.c;
              y = (one - e) * cur + cr * right + cd * down;
            }
          } else {
            const T gp = co.d * (T)pp;
            T e = ebase + gp - (pp + 1 < P ? (T)0 : cd);  // no protein birth in the top row
            T cup = co.d * (T)(pp + 1);
            y = (one - e) * cur + cl * left + cr * right + cd * down + cup * up;
          }
          if (p.renorm > 0) {
            y *= f;
            part += y;
          }
          dst[li] = y;
        }
        down = cur;
        cur = up;
      }
    }
    const bool do_renorm = p.renorm > 0 && jump && (k % p.renorm) == 0;
    double* redk = red + (k & 1) * 33;
    if (do_renorm) {
      double v = (double)part;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
      if (lane == 0) redk[warp] = v;
    }
    __syncthreads();
    lo = clo;
    hi = chi;
    if (!jump) break;
    f_prev = 1.0;
    if (do_renorm) {
      if (C > 1) cluster.sync();
      double tot = 0.0;
      for (int r = 0; r < C; ++r) {
        const double* rr = (C == 1) ? redk : cluster.map_shared_rank(redk, r);
        for (int w = 0; w < nwarps; ++w) tot += rr[w];
      }
      f_prev = tot > 0.0 ? mass0 / tot : 1.0;
      if (LL && f_prev != 1.0) {
        for (int j = tid; j < tile; j += nthr) dst[j] = (T)(dst[j] * (T)f_prev);
        f_prev = 1.0;
        __syncthreads();
      }
      if (LL) group_accumulate(dst, lo, hi, k, wcur);
      if (C > 1) cluster.sync();  // remote reads of red and of dst are complete
    } else {
      if (C > 1) cluster_arrive();
      if (LL) group_accumulate(dst, lo, hi, k, wcur);
      if (C > 1) cluster_wait();
    }
  }

  if (LL) {
    // ---- epilogue: sum_g c_g log(a_g), partial sums of all CTAs ------------
    if (C > 1) cluster.sync();
    else __syncthreads();
    if (rank == 0) {
      double ll = 0.0;
      bool bad = false;
      for (int gq = tid; gq < p.G; gq += nthr) {
        double a = 0.0;
        for (int r = 0; r < C; ++r) {
          const T* rs = (C == 1) ? acc_s : cluster.map_shared_rank(acc_s, r);
          double v = (double)rs[gq];
          if (sizeof(T) == 4) {
            const float* rc = (C == 1) ? acc_c : cluster.map_shared_rank(acc_c, r);
            v -= (double)rc[gq];
          }
          a += v;
        }
        double c = p.counts[gq];
        if (c == 0.0) continue;
        if (a > 0.0) ll += c * log(a);
        else if (a > -1e-30) ll = -INFINITY;
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
    if (C > 1) cluster.sync();  // keep every CTA's shared memory alive until rank 0 is done
  }
}

template <typename T, int KIND, bool LL>
cudaError_t launch_typed(const ChainParams& p, int cluster, int threads, cudaStream_t s) {
  int tile = tile_elems(KIND, p.M, p.P, (int)p.N, (int)p.slab);
  size_t smem = smem_layout(sizeof(T), tile, p.ntimes, p.G, p.nmem, LL).total;
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
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
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

template <typename T, bool LL>
int max_clusters_kind(int kind, int cluster, int threads, size_t smem) {
  switch (kind) {
    case MJP_BD1D: return max_clusters_typed<T, MJP_BD1D, LL>(cluster, threads, smem);
    case MJP_TWOSTATE: return max_clusters_typed<T, MJP_TWOSTATE, LL>(cluster, threads, smem);
    default: return max_clusters_typed<T, MJP_MRNA_PROT2D, LL>(cluster, threads, smem);
  }
}

}  // namespace

int64_t chain_stencil_slab(int kind, int64_t M, int64_t P, int cluster) {
  int64_t N = M * P;
  if (kind == MJP_BD1D) return (N + cluster - 1) / cluster;
  int64_t rows = (P + cluster - 1) / cluster;
  return rows * M;
}

size_t chain_stencil_smem(int kind, int precision, int loglik_mode, int64_t M, int64_t P, int64_t slab,
                          int ntimes, int G, int nmem) {
  int tile = tile_elems(kind, (int)M, (int)P, (int)(M * P), (int)slab);
  return smem_layout(precision == MJP_FP64 ? 8 : 4, tile, ntimes, G, nmem, loglik_mode != 0).total;
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
  if (precision == MJP_FP64)
    return ll ? max_clusters_kind<double, true>(kind, cluster, threads, smem)
              : max_clusters_kind<double, false>(kind, cluster, threads, smem);
  return ll ? max_clusters_kind<float, true>(kind, cluster, threads, smem)
            : max_clusters_kind<float, false>(kind, cluster, threads, smem);
}

}  // namespace mjp
