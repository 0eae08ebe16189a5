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
//
// FP32 chains run the compensated jump of chain_common.cuh: every state
// carries its rounding residual (a third tile, single-buffered: only the
// state's owner touches it) and, every p.renorm jumps, adds back the defect
// of its exit coefficient (a fourth tile, formed once in the prologue).
#include <cooperative_groups.h>

#include "chain_common.cuh"
#include "internal.cuh"

namespace cg = cooperative_groups;

namespace mjp {

namespace {

// Local tile geometry of one CTA.
//  - birth-death chain: one row of W owned columns plus one zero pad cell on
//    each side;
//  - two-dimensional models: owned rows [p0, p1) stored as row PAIRS
//    (rows 2j and 2j+1 of a column side by side, i.e. a float2/double2 per
//    column), with a pad pair-row below and above and a pad column on each
//    side, so a thread updates two states with packed arithmetic.
struct Geo {
  int p0, p1, m0, m1;  // owned rows [p0, p1) and columns [m0, m1)
  int W, H;            // width and height of the owned block
  int Hp;              // owned pair-rows (2-D)
  int Wp;              // padded row stride in cells (W + 2)
  int size;            // padded tile in scalar elements
};

__host__ __device__ inline Geo geometry(int kind, int M, int P, int N, int slab, int rank) {
  Geo g;
  int n0 = rank * slab;
  int n1 = n0 + slab < N ? n0 + slab : N;
  if (n1 < n0) n1 = n0;
  if (kind == MJP_BD1D) {
    g.p0 = 0; g.p1 = 1; g.m0 = n0; g.m1 = n1;
  } else {  // slab is an even number of whole rows
    g.p0 = n0 / M; g.p1 = (n1 + M - 1) / M; g.m0 = 0; g.m1 = M;
    if (g.p1 < g.p0) g.p1 = g.p0;
  }
  g.W = g.m1 - g.m0;
  g.H = g.p1 - g.p0;
  g.Hp = (g.H + 1) / 2;
  g.Wp = g.W + 2;
  g.size = (kind == MJP_BD1D) ? g.Wp : (g.Hp + 2) * g.Wp * 2;
  return g;
}

// Scalar element of owned local row r, local column c of a 2-D tile.
__host__ __device__ inline int elem2d(const Geo& g, int r, int c) {
  return (((r >> 1) + 1) * g.Wp + c + 1) * 2 + (r & 1);
}

// Largest padded tile over the ranks of a cluster (rank 0 is never smaller).
__host__ __device__ inline int tile_elems(int kind, int M, int P, int N, int slab) {
  Geo g = geometry(kind, M, P, N, slab, 0);
  return g.size;
}

struct Smem {
  size_t buf1, lo, cb, tx, tPL, ttail, tL, tK, twoff, twb, torig, pw, ring, red, memloc, gptr, mptr, gloc, gtime, acc_s,
      acc_c, total;
};

__host__ __device__ inline Smem smem_layout(size_t elt, int tile, int nt, int G, int nmem, bool ll) {
  Smem s;
  size_t bufbytes = align_up((size_t)tile * elt, 16);
  s.buf1 = bufbytes;
  size_t o = 2 * bufbytes;
  // FP32: residual and defect of every state, tile-shaped.
  s.lo = o;
  if (elt == 4) o += bufbytes;
  s.cb = o;
  if (elt == 4) o += bufbytes;
  s.tx = o; o += 8 * (size_t)nt;
  s.tPL = o; o += 8 * (size_t)nt;
  s.ttail = o; o += 8 * (size_t)nt;
  s.tL = o; o += 8 * (size_t)nt;
  s.tK = o; o += 8 * (size_t)nt;
  s.torig = o; o += align_up(4 * (size_t)nt, 8);
  s.twoff = o; o += 8 * (size_t)nt;
  s.twb = o; o += 8 * (size_t)nt;
  s.pw = o; o += 16 * (size_t)nt;
  s.ring = o; o += align_up(elt * kWeightRing * (size_t)nt, 8);
  s.red = o; o += 8 * 2 * 33;
  // nmem > 0 only when some group has more than two members: the generic
  // member list; otherwise each group's (at most two) members are resolved
  // once into gloc.
  s.memloc = o;
  if (ll) o += align_up(4 * (size_t)nmem, 8);
  s.gptr = o;
  if (ll) o += align_up(4 * (size_t)(nt + 1), 8);
  s.mptr = o;
  if (ll && nmem > 0) o += align_up(4 * (size_t)(G + 1), 8);
  s.gloc = o;
  if (ll) o += 8 * (size_t)G;
  s.gtime = o;
  if (ll) o += align_up(2 * (size_t)G, 8);
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

// Exit defect of the state in tile row `row`, column `col` for the compensated
// FP32 chain (see chain_common.cuh): the exit coefficient the update applies
// minus the sum of the outflow coefficients its neighbours apply.  Birth-death
// and mRNA/protein use the shared forms (their chains also run in the
// register-resident kernels); the two-state and autoregulatory models form it
// in FP64 from the FP32 coefficients of the update below.
template <int KIND, typename T>
__device__ float exit_defect(const Coef<T>& co, int row, int col, int M, int P) {
  if (KIND == MJP_BD1D) return bd_defect(co, col, M);
  if (KIND == MJP_MRNA_PROT2D) return mrna_defect(mrna_col(co, col, M), (float)co.d, row);
  if (KIND == MJP_TWOSTATE) return ts_defect(co, row, col, M);
  const float fm = (float)col;
  // Autoregulatory network, tile row 2 q + sigma (Pm = P / 2 protein counts).
  const int q = row >> 1, Pm = P / 2;
  const float fq = (float)q;
  const bool qtop = q + 1 >= Pm;
  const float a_gm = __fmul_rn((float)co.c, fm);                // gamma_R m (to m-1)
  const float a_tx = col + 1 < M ? (float)co.a : 0.0f;          // beta_R (to m+1, active)
  const float tr = qtop ? 0.0f : __fmul_rn((float)co.b, fm);    // beta_P m (to q+1)
  const float pd = __fmul_rn((float)co.d, fq);                  // gamma_P q (to q-1)
  const float decay = __fadd_rn(pd, a_gm);
  if ((row & 1) == 0) {
    const float bind = __fmul_rn((float)co.f, fq);              // lambda_ina q (to q-1, inactive)
    const float e = __fadd_rn(__fadd_rn(__fadd_rn(decay, a_tx), tr), bind);
    return (float)(((((double)e - (double)a_tx) - (double)a_gm) - (double)tr) - (double)pd - (double)bind);
  }
  const float unb = qtop ? 0.0f : (float)co.e;                  // lambda_act (to q+1, active)
  const float e = __fadd_rn(__fadd_rn(decay, tr), unb);
  return (float)(((((double)e - (double)a_gm) - (double)tr) - (double)pd) - (double)unb);
}

template <typename T, int KIND, bool LL>
__global__ void __launch_bounds__(1024, 1) chain_kernel(ChainParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int job = p.job_map ? p.job_map[blockIdx.x / C] : blockIdx.x / C;
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = nthr >> 5;
  const int nt = p.ntimes;
  // Batches of uneven birth-death instances carry their own state count.
  const int N = p.jobN ? p.jobN[job] : (int)p.N;
  const int M = p.jobN ? N : p.M, P = p.P;
  const int S = p.jobN ? (N + C - 1) / C : (int)p.slab;
  const Geo g = geometry(KIND, M, P, N, S, rank);
  const int tile = p.tile_max > 0 ? p.tile_max : tile_elems(KIND, M, P, N, S);
  const int64_t out_base = p.job_off ? p.job_off[job] : (int64_t)job * p.out_stride;
  const int64_t comp_base = p.job_off ? p.job_off[job] : (int64_t)job * p.comp_stride;

  const Smem L = smem_layout(sizeof(T), tile, nt, p.G, p.nmem, LL);
  // Tile buffers are always formed from the __shared__ base (never through a
  // runtime-indexed pointer array), so accesses compile to shared-memory
  // instructions with 32-bit addressing.
  const unsigned buf_off[2] = {0u, (unsigned)L.buf1};
  T* const buf0 = reinterpret_cast<T*>(smem);
  T* const buf1 = reinterpret_cast<T*>(smem + L.buf1);
  constexpr bool kComp = sizeof(T) == 4;  // compensated FP32 chain
  float* const lo_t = reinterpret_cast<float*>(smem + L.lo);  // residual of each state (FP32)
  float* const cb_t = reinterpret_cast<float*>(smem + L.cb);  // p.renorm x exit defect (FP32)
  double* t_x = reinterpret_cast<double*>(smem + L.tx);
  double* t_PL = reinterpret_cast<double*>(smem + L.tPL);
  double* t_tail = reinterpret_cast<double*>(smem + L.ttail);
  long long* t_L = reinterpret_cast<long long*>(smem + L.tL);
  long long* t_K = reinterpret_cast<long long*>(smem + L.tK);
  int* t_orig = reinterpret_cast<int*>(smem + L.torig);
  double* pw = reinterpret_cast<double*>(smem + L.pw);   // [2][nt] FP64 recurrence state
  long long* t_woff = reinterpret_cast<long long*>(smem + L.twoff);
  T* ring = reinterpret_cast<T*>(smem + L.ring);         // [kWeightRing][nt] weight of each jump
  const T* arena = reinterpret_cast<const T*>(p.arena);
  double* red = reinterpret_cast<double*>(smem + L.red);  // [2][33]
  int* memloc = reinterpret_cast<int*>(smem + L.memloc);
  int2* gloc = reinterpret_cast<int2*>(smem + L.gloc);     // tile index of a group's first two members
  short* gtime = reinterpret_cast<short*>(smem + L.gtime);  // time of each group
  const T** t_wb = reinterpret_cast<const T**>(smem + L.twb);  // arena + woff - L per time
  int* s_gptr = reinterpret_cast<int*>(smem + L.gptr);  // group ranges per time
  int* s_mptr = reinterpret_cast<int*>(smem + L.mptr);  // member ranges per group
  T* acc_s = reinterpret_cast<T*>(smem + L.acc_s);
  float* acc_c = reinterpret_cast<float*>(smem + L.acc_c);

  // Pad cells of the neighbouring CTAs that receive this CTA's boundary
  // values after every jump (pushed through distributed shared memory), so
  // that every stencil read is a local one.
  T* push_dn[2] = {nullptr, nullptr};  // rank-1: top pad pair-row (2-D) / right pad cell (1-D)
  T* push_up[2] = {nullptr, nullptr};  // rank+1: bottom pad pair-row (2-D) / left pad cell (1-D)
  if (C > 1) {
    if (rank > 0) {
      Geo gd = geometry(KIND, M, P, N, S, rank - 1);
      int off = (KIND == MJP_BD1D) ? gd.Wp - 1 : (gd.Hp + 1) * gd.Wp * 2;
      push_dn[0] = cluster.map_shared_rank(buf0, rank - 1) + off;
      push_dn[1] = cluster.map_shared_rank(buf1, rank - 1) + off;
    }
    if (rank + 1 < C) {
      Geo gu = geometry(KIND, M, P, N, S, rank + 1);
      if (gu.W > 0 && gu.H > 0)
      {
        push_up[0] = cluster.map_shared_rank(buf0, rank + 1);
        push_up[1] = cluster.map_shared_rank(buf1, rank + 1);
      }
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
    t_woff[i] = w.woff;
    t_wb[i] = (w.woff >= 0 && arena) ? arena + (w.woff - w.L) : nullptr;
    pw[i] = (w.L == 0) ? w.PL : 0.0;  // recurrence state at jump 0
    if (w.L == 0)                     // weight of jump 0 (tail folded in)
      ring[i] = (w.woff >= 0 && arena) ? arena[w.woff] : (T)(w.PL + (w.K == 0 ? w.tail : 0.0));
  }
  const double omega = p.info[job].omega;
  const int64_t Kmax = p.info[job].Kmax;
  const Coef<T> co = make_coef<T, KIND>(p.theta + (int64_t)job * p.ntheta, omega);
  const T* rho0 = reinterpret_cast<const T*>(p.rho0);
  const int64_t s0 = p.job_s0 ? p.job_s0[job] : -1;  // rho0 = delta at s0
  auto rho0_at = [&](int64_t n) -> T { return s0 >= 0 ? (T)(n == s0 ? 1 : 0) : rho0[n]; };
  // Model index of tile row `row`, column `col`.  The autoregulatory model's
  // tile rows interleave the gene states (row 2 n_P + sigma), so a row pair
  // holds both gene states of one protein count; its model index is
  // n_R + N_R n_P + N_R N_P sigma (Sec. 3.1.3).
  const int Pm = (KIND == MJP_AUTOREG) ? P / 2 : P;
  auto gidx = [&](int64_t row, int64_t col) -> int64_t {
    return KIND == MJP_AUTOREG ? col + (int64_t)M * (row >> 1) + (int64_t)M * Pm * (row & 1) : row * M + col;
  };
  for (int j = tid; j < tile; j += nthr) {
    buf0[j] = (T)0;
    buf1[j] = (T)0;
    if (kComp) {
      lo_t[j] = 0.0f;
      cb_t[j] = 0.0f;
    }
  }
  __syncthreads();
  for (int j = tid; j < g.W * g.H; j += nthr) {
    int r = j / g.W, c = j - r * g.W;
    const int li = KIND == MJP_BD1D ? c + 1 : elem2d(g, r, c);
    T v = rho0_at(gidx(g.p0 + r, g.m0 + c));
    buf0[li] = v;
    if (kComp && p.renorm > 0) cb_t[li] = (float)p.renorm * exit_defect<KIND>(co, g.p0 + r, g.m0 + c, M, P);
  }
  // Halo of rho0 from global memory (later jumps receive it by push): the
  // row below a 2-D slab is the odd half of the bottom pad pair, the row above
  // the even half of the top pad pair.
  if (KIND == MJP_BD1D) {
    if (tid == 0 && g.W > 0 && g.m0 >= 1) buf0[0] = rho0_at(g.m0 - 1);
    if (tid == 0 && g.W > 0 && g.m1 < M) buf0[g.Wp - 1] = rho0_at(g.m1);
  } else if (g.H > 0) {
    for (int c = tid; c < g.W; c += nthr) {
      if (g.p0 >= 1) buf0[(c + 1) * 2 + 1] = rho0_at(gidx(g.p0 - 1, c));
      if (g.p1 < P) buf0[((g.Hp + 1) * g.Wp + c + 1) * 2] = rho0_at(gidx(g.p1, c));
      // The autoregulatory update reads both gene states of the neighbouring
      // protein counts, i.e. whole pad pairs.
      if (KIND == MJP_AUTOREG && g.p0 >= 2) buf0[(c + 1) * 2] = rho0_at(gidx(g.p0 - 2, c));
      if (KIND == MJP_AUTOREG && g.p1 + 1 < P) buf0[((g.Hp + 1) * g.Wp + c + 1) * 2 + 1] = rho0_at(gidx(g.p1 + 1, c));
    }
  }
  if (LL) {
    // Tile index of state s in this CTA, or -1 when another CTA owns it.
    auto loc_of = [&](int s) -> int {
      int ps = s / M, ms = s - ps * M;
      if (KIND == MJP_AUTOREG) {  // tile row 2 n_P + sigma
        const int sg = s / (M * Pm), rem = s - sg * M * Pm, pm = rem / M;
        ms = rem - pm * M;
        ps = 2 * pm + sg;
      }
      bool mine = ps >= g.p0 && ps < g.p1 && ms >= g.m0 && ms < g.m1;
      return !mine ? -1 : (KIND == MJP_BD1D ? ms - g.m0 + 1 : elem2d(g, ps - g.p0, ms));
    };
    for (int q = tid; q < p.nmem; q += nthr) memloc[q] = loc_of(p.members[q]);
    for (int q = tid; q < p.G; q += nthr) {
      acc_s[q] = (T)0;
      if (sizeof(T) == 4) acc_c[q] = 0.0f;
      const int q0 = (int)p.mptr[q], q1 = (int)p.mptr[q + 1];
      gloc[q] = make_int2(q1 > q0 ? loc_of(p.members[q0]) : -1, q1 > q0 + 1 ? loc_of(p.members[q0 + 1]) : -1);
      if (p.nmem > 0) s_mptr[q] = q0;
    }
    if (p.nmem > 0 && tid == 0) s_mptr[p.G] = (int)p.mptr[p.G];
    for (int q = tid; q <= nt; q += nthr) s_gptr[q] = (int)p.gptr[q];
    for (int i = warp; i < nt; i += nwarps)
      for (int q = (int)p.gptr[i] + lane; q < (int)p.gptr[i + 1]; q += 32) gtime[q] = (short)i;
  }
  if (C > 1) cluster.sync();
  else __syncthreads();
  // Does any window lack a stored copy of its weights (arena overflow)?
  bool mine_rec = false;
  for (int i = tid; i < nt; i += nthr) mine_rec |= t_woff[i] < 0;
  const bool any_rec = __syncthreads_or(mine_rec) != 0;

  // Active times of jump k form a contiguous range [lo, hi] (times sorted).
  int lo = 0, hi = -1;
  auto advance = [&](int64_t k, int& l, int& h) {
    while (l < nt && t_K[l] < k) ++l;
    while (h + 1 < nt && t_L[h + 1] <= k) ++h;
  };
  advance(0, lo, hi);
  // Weight prefetch pointer: active times of jump k + lead.
  int flo = 0, fhi = -1;
  if (warp == nwarps - 1) {  // the weights warp
    for (int64_t kf = 1; kf <= kWeightLead; ++kf) {
      advance(kf, flo, fhi);
      if (kf <= Kmax)
        for (int i = flo + lane; i <= fhi; i += 32)
          if (t_wb[i]) cp_async_elem(ring + (int)(kf % kWeightRing) * nt + i, t_wb[i] + kf);
      cp_async_commit();
    }
  }

  // Thread layout: the last warp forms the Poisson weights (FP64, off the
  // stencil's critical path); the other warps own columns and runs of rows.
  const int nthr_c = nthr - 32;
  const bool wwarp = warp == nwarps - 1;
  // Birth-death tiles are one row: every stencil thread takes columns
  // tid, tid + nthr_c, ... (threads past the row stay idle), so no state has
  // two owners.
  const int TX = (KIND == MJP_BD1D) ? nthr_c : (g.W > 0 ? g.W : 1);
  const int TY = nthr_c / TX > 0 ? nthr_c / TX : 1;
  const int tx = tid % TX, ty = wwarp ? TY : tid / TX;
  // 2-D threads walk a run of R pair-rows [ja, jb) of their column.
  const int R = (KIND == MJP_BD1D) ? 1 : (g.Hp + TY - 1) / TY;
  const int ja = ty * R;
  const int jb = (ty < TY) ? min(g.Hp, ja + R) : ja;
  const bool rows = !wwarp && tx < g.W && ja < jb;  // 2-D models
  // Observation groups are folded in by the weights warp when the stencil
  // threads are busy (>= 8 states each), otherwise by every thread.
  const int spt = (KIND == MJP_BD1D) ? (g.W + nthr_c - 1) / nthr_c : 2 * R;
  const bool acc_ww = spt >= 8;
  const bool acc_me = acc_ww ? wwarp : true;
  const int acc_id = acc_ww ? lane : tid, acc_stride = acc_ww ? 32 : nthr;

  // LOGLIK: acc_g += w_i f sum_{s in g} rho_k[s] over this CTA's states.
  // The groups of the active times [l, h] are one contiguous index range
  // (groups are stored time by time), so threads take groups directly.
  auto group_accumulate = [&](const T* cur, int l, int h, const T* wts) {
    if (h < l) return;
    const int ga = s_gptr[l], gb = s_gptr[h + 1];
    for (int gq = ga + acc_id; gq < gb; gq += acc_stride) {
      const int2 lq = gloc[gq];
      bool any = lq.x >= 0 || lq.y >= 0;
      T v = lq.x >= 0 ? cur[lq.x] : (T)0;
      if (lq.y >= 0) v = f_add(v, cur[lq.y]);
      if (p.nmem > 0) {  // members beyond the second
        const int q1 = s_mptr[gq + 1];
        for (int q = s_mptr[gq] + 2; q < q1; ++q) {
          const int li = memloc[q];
          if (li >= 0) {
            v = f_add(v, cur[li]);
            any = true;
          }
        }
      }
      if (!any) continue;
      const T w = wts[gtime[gq]];
      {
        if (sizeof(T) == 4) {
          float y = __fsub_rn(__fmul_rn((float)w, (float)v), acc_c[gq]);
          float s0 = (float)acc_s[gq];
          float t = __fadd_rn(s0, y);
          acc_c[gq] = __fsub_rn(__fsub_rn(t, s0), y);
          acc_s[gq] = (T)t;
        } else {
          acc_s[gq] = f_fma(w, v, acc_s[gq]);
        }
      }
    }
  };

  // EXPV: rho*_i += w rho_{k-1}[n] for the active times (Kahan in FP32).
  auto expv_accumulate = [&](T rv, int64_t gidx, int64_t kp, int l, int h, const T* wts) {
    for (int i = l; i <= h; ++i) {
      const T w = wts[i];
      T* o = reinterpret_cast<T*>(p.out) + out_base + (int64_t)t_orig[i] * N + gidx;
      if (sizeof(T) == 4) {
        float* cp = p.comp + comp_base + (int64_t)i * N + gidx;
        float s, cc;
        if (kp == t_L[i]) {
          s = __fmul_rn((float)w, (float)rv);
          cc = 0.0f;
        } else {
          s = (float)*o;
          cc = *cp;
          float y = __fsub_rn(__fmul_rn((float)w, (float)rv), cc);
          float t = __fadd_rn(s, y);
          cc = __fsub_rn(__fsub_rn(t, s), y);
          s = t;
        }
        if (kp == t_K[i]) *o = (T)__fsub_rn(s, cc);
        else {
          *o = (T)s;
          *cp = cc;
        }
      } else {
        if (kp == t_L[i]) *o = f_mul(w, rv);
        else *o = f_fma(w, rv, *o);
      }
    }
  };

  // Column constants of a 2-D thread as pairs (rates into column m, scaled
  // by 1/Omega); the pair holds the values for rows 2j and 2j+1.
  using T2 = typename Pair<T>::type;
  const int mc = tx;  // 2-D slabs span all columns (m0 = 0)
  const T one = (T)1;
  T cd = (T)0;
  T2 c_l = v_make((T)0, (T)0), c_r = c_l, c_d = c_l, c_dg = c_l, c_sw = c_l, c_gp = c_l, c_ngp = c_l;
  // Autoregulatory column constants: gamma_R m, beta_R (if m+1 < N_R), beta_P m.
  const T a_gm = (KIND == MJP_AUTOREG) ? f_mul(co.c, (T)mc) : (T)0;
  const T a_tx = (KIND == MJP_AUTOREG && mc + 1 < M) ? co.a : (T)0;
  const T a_tl = (KIND == MJP_AUTOREG) ? f_mul(co.b, (T)mc) : (T)0;
  if (KIND == MJP_TWOSTATE) {
    // Active row (x): birth from m-1, death from m+1, reactivation of the
    // inactive state; inactive row (y): death from m+1, deactivation.
    const T bm = f_mul(co.b, (T)mc);
    const T cr = f_mul(co.b, (T)(mc + 1));
    c_l = v_make(co.a, (T)0);
    c_r = v_make(cr, cr);
    const T ex = f_add(f_add(bm, mc + 1 < M ? co.a : (T)0), co.d), ey = f_add(co.c, bm);
    c_dg = kComp ? v_make(-ex, -ey) : v_make(f_sub(one, ex), f_sub(one, ey));  // 1 - e (FP32: -e)
    c_sw = v_make(co.c, co.d);
  } else if (KIND == MJP_AUTOREG) {
    const T cr = f_mul(co.c, (T)(mc + 1));                 // gamma_R (m+1) from m+1
    c_r = v_make(cr, cr);
  }
  if (KIND == MJP_MRNA_PROT2D) {
    const T fm = (T)mc;
    const T cr = f_mul(co.b, (T)(mc + 1));                 // gamma_m (m+1) from m+1
    cd = f_mul(co.c, fm);                                  // k_p m from p-1
    const T e0 = f_add(f_add(f_mul(co.b, fm), mc + 1 < M ? co.a : (T)0), cd);
    const T d0 = kComp ? -e0 : f_sub(one, e0);
    c_l = v_make(co.a, co.a);                              // k_m from m-1
    c_r = v_make(cr, cr);
    c_d = v_make(cd, cd);
    c_dg = v_make(d0, d0);                                 // 1 - e without gamma_p p (FP32: -e)
    c_gp = v_make(co.d, co.d);                             // gamma_p
    c_ngp = v_make(-co.d, -co.d);
  }
  const T2 two2 = v_make((T)2, (T)2);

  // ---- the jump chain -----------------------------------------------------
  // Ring slots of jumps k - 1, k and k + lead, and the jumps left until the
  // next exit-defect correction, kept as counters (no 64-bit modulo per jump).
  int sprev = 0, scur = 1 % kWeightRing, sfut = (1 + kWeightLead) % kWeightRing;
  int dleft = p.renorm;
  for (int64_t k = 1; k <= Kmax + 1; ++k) {
    const int par = (int)((k - 1) & 1);
    const T* src = reinterpret_cast<const T*>(smem + buf_off[par]);
    T* dst = reinterpret_cast<T*>(smem + buf_off[par ^ 1]);
    const double* rprev = pw + par * nt;    // FP64 recurrence state, jump k-1
    double* rcur = pw + (par ^ 1) * nt;     // jump k
    const T* wprev = ring + sprev * nt;     // weights of jump k-1
    T* wcur = ring + scur * nt;
    const int plo = lo, phi = hi;
    int clo = lo, chi = hi;
    advance(k, clo, chi);
    const bool jump = k <= Kmax;
    // FP32: the exit defects are added back after jumps that are multiples of p.renorm.
    bool dfix = false;
    if (kComp && p.renorm > 0 && --dleft == 0) {
      dfix = jump;
      dleft = p.renorm;
    }
    if (wwarp) {
      // Weights of jump k + lead from the planner's arena, copied straight
      // into the ring (cp.async, one group per jump) ...
      const int64_t kf = k + kWeightLead;
      advance(kf, flo, fhi);
      if (kf <= Kmax)
        for (int i = flo + lane; i <= fhi; i += 32)
          if (t_wb[i]) cp_async_elem(ring + sfut * nt + i, t_wb[i] + kf);
      cp_async_commit();
      // ... and, for windows without a stored copy, Algorithm 2's recurrence
      // P_k = P_{k-1} x / k (the tail is added at k = K).
      if (jump && any_rec)
        for (int i = clo + lane; i <= chi; i += 32) {
          if (t_woff[i] >= 0) continue;
          const double P = (k == t_L[i]) ? t_PL[i] : __dmul_rn(rprev[i], __ddiv_rn(t_x[i], (double)k));
          rcur[i] = P;
          wcur[i] = (T)(P + (k == t_K[i] ? t_tail[i] : 0.0));
        }
      cp_async_wait<kWeightLead>();  // jump k's copy (issued lead jumps ago) has landed
    }
    if (LL && acc_me) group_accumulate(src, plo, phi, wprev);
    if (KIND == MJP_BD1D) {
      for (int m = wwarp ? g.m1 : g.m0 + tx; m < g.m1; m += TX) {
        const int li = m - g.m0 + 1;
        const T cur = src[li];
        if (!LL) expv_accumulate(cur, m, k - 1, plo, phi, wprev);
        if (jump) {
          const T fm = (T)m;
          const T e = f_add(f_mul(co.b, fm), m + 1 < M ? co.a : (T)0);
          const T cr = f_mul(co.b, f_add(fm, one));
          T y;
          if constexpr (kComp) {
            float l = lo_t[li];
            y = comp_jump(cur, l, co.a, src[li - 1], cr, src[li + 1], -e);
            if (dfix) l = __fmaf_rn(cb_t[li], y, l);
            lo_t[li] = l;
          } else {
            y = f_mul(f_sub(one, e), cur);
            y = f_fma(co.a, src[li - 1], y);
            y = f_fma(cr, src[li + 1], y);
          }
          dst[li] = y;
          if (m == g.m0 && push_dn[par ^ 1]) *push_dn[par ^ 1] = y;
          if (m == g.m1 - 1 && push_up[par ^ 1]) *push_up[par ^ 1] = y;
        }
      }
    } else if (rows) {
      // The two ping-pong buffers never overlap.
      const T2* __restrict__ sp = reinterpret_cast<const T2*>(src) + (ja + 1) * g.Wp + mc + 1;
      T2* __restrict__ dp = reinterpret_cast<T2*>(dst) + (ja + 1) * g.Wp + mc + 1;
      T2* const dfirst = dp;
      const int W2 = g.Wp;
      int pp = g.p0 + 2 * ja;  // row of the pair's first half
      T2 prev = sp[-W2];
      T2 cur = sp[0];
      T2 fpp = v_make((T)pp, (T)(pp + 1));
      T2 y = v_make((T)0, (T)0);
      float2* lp = kComp ? reinterpret_cast<float2*>(lo_t) + (ja + 1) * g.Wp + mc + 1 : nullptr;
      const float2* cbp = kComp ? reinterpret_cast<const float2*>(cb_t) + (ja + 1) * g.Wp + mc + 1 : nullptr;
      // One pair-row: rows pp and pp+1 of column mc.  `top` marks the pair
      // that holds row P-1 (no protein birth out of it; row P absent).
      auto pair_row = [&](bool top) {
        const T2 next = sp[W2];
        const T2 left = sp[-1], right = sp[1];
        if (!LL) {
          expv_accumulate(cur.x, gidx(pp, mc), k - 1, plo, phi, wprev);
          if (pp + 1 < g.p1) expv_accumulate(cur.y, gidx(pp + 1, mc), k - 1, plo, phi, wprev);
        }
        if (jump) {
          if (KIND == MJP_TWOSTATE) {
            if constexpr (kComp) {
              float2 l = *lp;
              float2 t = v_fma(c_l, left, l);
              t = v_fma(c_r, right, t);
              t = v_fma(c_sw, v_make(cur.y, cur.x), t);
              t = v_fma(c_dg, cur, t);  // c_dg holds -e (compensated chain)
              y = comp_finish(cur, t, l);
              *lp = l;
            } else {
              const T2 t1 = v_fma(c_l, left, v_mul(c_dg, cur));
              const T2 t2 = v_fma(c_sw, v_make(cur.y, cur.x), v_mul(c_r, right));
              y = v_add(t1, t2);
            }
          } else if (KIND == MJP_AUTOREG) {
            // Pair = (active, inactive) at protein count q: transcription from
            // m-1 (active only), R decay from m+1, translation from q-1, P
            // decay from q+1, unbinding from (q-1, inactive) into active,
            // binding from (q+1, active) into inactive.
            const int q = pp >> 1;
            const T fq = (T)q;
            const bool qtop = q + 1 >= Pm;
            const T decay = f_add(f_mul(co.d, fq), a_gm);         // gamma_P q + gamma_R m
            const T tr = qtop ? (T)0 : a_tl;                       // beta_P m, if q+1 exists
            const T e0 = f_add(f_add(f_add(decay, a_tx), tr), f_mul(co.f, fq));
            const T e1 = f_add(f_add(decay, tr), qtop ? (T)0 : co.e);
            const T gq = f_mul(co.d, (T)(q + 1));
            if constexpr (kComp) {
              float2 l = *lp;
              float2 t = l;
              t.x = f_fma(co.a, left.x, t.x);
              t = v_fma(c_r, right, t);
              t = v_fma(v_make(a_tl, a_tl), prev, t);
              t = v_fma(v_make(gq, gq), next, t);
              t.x = f_fma(co.e, prev.y, t.x);
              t.y = f_fma(f_mul(co.f, (T)(q + 1)), next.x, t.y);
              t = v_fma(v_make(-e0, -e1), cur, t);
              y = comp_finish(cur, t, l);
              *lp = l;
            } else {
              y.x = f_mul(f_sub(one, e0), cur.x);
              y.y = f_mul(f_sub(one, e1), cur.y);
              y.x = f_fma(co.a, left.x, y.x);
              y = v_fma(c_r, right, y);
              y = v_fma(v_make(a_tl, a_tl), prev, y);
              y = v_fma(v_make(gq, gq), next, y);
              y.x = f_fma(co.e, prev.y, y.x);
              y.y = f_fma(f_mul(co.f, (T)(q + 1)), next.x, y.y);
            }
          } else {
            T2 dg = v_fma(c_ngp, fpp, c_dg);        // 1 - e_{m,p} (FP32: -e_{m,p})
            const T2 cup = v_fma(c_gp, fpp, c_gp);  // gamma_p (p+1) from p+1
            if constexpr (kComp) {
              // In the order of the register-resident kernel: residual, the
              // inflows from the left, right, below and above, the exit, and at
              // row P-1 the protein birth k_p m that does not leave it.
              float2 l = *lp;
              float2 t = v_fma(c_l, left, l);
              t = v_fma(c_r, right, t);
              t.x = f_fma(cd, prev.y, t.x);
              t.y = f_fma(cd, cur.x, t.y);
              t.x = f_fma(cup.x, cur.y, t.x);
              t.y = f_fma(cup.y, next.x, t.y);
              t = v_fma(dg, cur, t);
              if (top) {
                if (pp == P - 1) t.x = f_fma(cd, cur.x, t.x);
                else t.y = f_fma(cd, cur.y, t.y);
              }
              y = comp_finish(cur, t, l);
              if (top && pp + 1 >= P) {  // row P does not exist
                y.y = 0.0f;
                l.y = 0.0f;
              }
              *lp = l;
            } else {
              if (top) {
                if (pp == P - 1) dg.x = f_add(dg.x, cd);
                else dg.y = f_add(dg.y, cd);
              }
              y = v_fma(c_r, right, v_fma(c_l, left, v_mul(dg, cur)));
              y.x = f_fma(cup.x, cur.y, f_fma(cd, prev.y, y.x));  // rows below / above
              y.y = f_fma(cup.y, next.x, f_fma(cd, cur.x, y.y));
              if (top && pp + 1 >= P) y.y = (T)0;     // row P does not exist
            }
            fpp = v_add(fpp, two2);
          }
          if constexpr (kComp) {
            if (dfix) *lp = v_fma(*cbp, y, *lp);
          }
          *dp = y;
        }
        prev = cur;
        cur = next;
        sp += W2;
        dp += W2;
        if constexpr (kComp) {
          lp += W2;
          cbp += W2;
        }
        pp += 2;
      };
      const bool has_top = (KIND == MJP_MRNA_PROT2D) && jb == g.Hp && g.p1 == P;
      const int jend = has_top ? jb - 1 : jb;
#pragma unroll 2
      for (int j = ja; j < jend; ++j) pair_row(false);
      if (has_top) pair_row(true);
      if (jump) {
        if (push_dn[par ^ 1] && ja == 0) reinterpret_cast<T2*>(push_dn[par ^ 1])[mc + 1] = *dfirst;
        if (push_up[par ^ 1] && jb == g.Hp) reinterpret_cast<T2*>(push_up[par ^ 1])[mc + 1] = y;
      }
    }
    if (C > 1) {
      cluster_arrive();
      cluster_wait();
    } else {
      __syncthreads();
    }
    lo = clo;
    hi = chi;
    sprev = scur;
    scur = scur + 1 == kWeightRing ? 0 : scur + 1;
    sfut = sfut + 1 == kWeightRing ? 0 : sfut + 1;
  }

  if (wwarp) cp_async_wait<0>();
  if (LL) {
    // ---- epilogue: sum_g c_g log(a_g), partial sums of all CTAs ------------
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

// Kernel attributes of one chain_kernel instantiation, raised only when
// needed (never lowered), so that launches made during CUDA-graph capture
// issue no attribute calls once a size has been set; the launcher and the
// occupancy query share them.
template <typename T, int KIND, bool LL>
cudaError_t ensure_attrs(int smem, int cluster) {
  static int smem_set = 0;
  static bool nonportable = false;
  auto kern = chain_kernel<T, KIND, LL>;
  cudaError_t e;
  if (smem > smem_set) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    smem_set = smem;
  }
  if (cluster > 8 && !nonportable) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    nonportable = true;
  }
  return cudaSuccess;
}

template <typename T, int KIND, bool LL>
cudaError_t launch_typed(const ChainParams& p, int cluster, int threads, cudaStream_t s) {
  int tile = p.tile_max > 0 ? p.tile_max : tile_elems(KIND, p.M, p.P, (int)p.N, (int)p.slab);
  size_t smem = smem_layout(sizeof(T), tile, p.ntimes, p.G, p.nmem, LL).total;
  auto kern = chain_kernel<T, KIND, LL>;
  cudaError_t e = ensure_attrs<T, KIND, LL>((int)smem, cluster);
  if (e != cudaSuccess) return e;
  if (p.B <= 0) return cudaSuccess;  // attribute preparation only
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
    case MJP_AUTOREG: return launch_typed<T, MJP_AUTOREG, LL>(p, cluster, threads, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int KIND, bool LL>
int max_clusters_typed(int cluster, int threads, size_t smem) {
  auto kern = chain_kernel<T, KIND, LL>;
  if (ensure_attrs<T, KIND, LL>((int)smem, cluster) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
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
    case MJP_AUTOREG: return max_clusters_typed<T, MJP_AUTOREG, LL>(cluster, threads, smem);
    default: return max_clusters_typed<T, MJP_MRNA_PROT2D, LL>(cluster, threads, smem);
  }
}

}  // namespace

int chain_stencil_tile(int kind, int64_t M, int64_t P, int64_t slab) {
  return tile_elems(kind, (int)M, (int)P, (int)(M * P), (int)slab);
}

int64_t chain_stencil_slab(int kind, int64_t M, int64_t P, int cluster) {
  int64_t N = M * P;
  if (kind == MJP_BD1D) return (N + cluster - 1) / cluster;
  int64_t rows = (P + cluster - 1) / cluster;
  rows += rows & 1;  // row pairs never straddle two CTAs
  return rows * M;
}

size_t chain_stencil_smem_tile(int precision, int loglik_mode, int tile, int ntimes, int G, int nmem) {
  return smem_layout(precision == MJP_FP64 ? 8 : 4, tile, ntimes, G, nmem, loglik_mode != 0).total;
}

size_t chain_stencil_smem(int kind, int precision, int loglik_mode, int64_t M, int64_t P, int64_t slab,
                          int ntimes, int G, int nmem) {
  int tile = tile_elems(kind, (int)M, (int)P, (int)(M * P), (int)slab);
  return smem_layout(precision == MJP_FP64 ? 8 : 4, tile, ntimes, G, nmem, loglik_mode != 0).total;
}

cudaError_t launch_chain_stencil(int kind, int precision, int loglik_mode, const ChainParams& p,
                                 int cluster, int threads, cudaStream_t s) {
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
