// stencil_regts.cu -- register-resident jump chain for the two-state
// promoter model (Eq. Gene_def: states (n_R, sigma), sigma = 0 active, 1
// inactive), FP32 compensated, log-likelihood mode: Algorithm 2 with one chain
// shared by all observation times, one small CTA per theta.
//
// The model has few states (2 N_R, N_R a few hundred) but is evaluated for
// many theta at once (one launch per sampler iteration), so what counts is the
// work per jump of a small chain, not bandwidth: the shared-memory kernel
// spends ~150 instructions per state update on its per-jump bookkeeping.
// Here the chain warps of a CTA hold the whole chain in registers and a jump
// is a few dozen packed FP32x2 operations per thread.
//
// Layout.  Thread g (= warp * 32 + lane) holds the columns (mRNA counts)
// [g 2QP, g 2QP + 2QP) of both rows, each row as QP pairs: pair j = (column
// c0 + j, column c0 + QP + j), so the neighbours of pair j in n_R are pairs
// j - 1 and j + 1 component by component (the whole update runs on FP32x2
// pairs) and the two gene states of a column sit in the same slot of the two
// rows.  Only a thread's first and last column need another thread's value:
// shuffles inside a warp, a double-buffered shared-memory slot and a named
// barrier of the chain warps between warps.  The pairs rotate through QP + 1
// register slots (pair j of rho_k is written over pair j - 1 of rho_{k-1},
// its last reader), so an in-place jump copies no register.
//
// Arithmetic per state is the shared-memory kernel's compensated jump
// (stencil.cu; chain_common.cuh) in the same order -- residual, inflow from
// n_R - 1, from n_R + 1, from the other gene state, the exit, then the
// residual step -- and the exit defects are added back every p.renorm jumps,
// so both kernels run bit-identical chains.
//
// Observations (warp specialised).  After every jump the chain threads whose
// columns hold observed states write their states of rho_k into a history in
// shared memory: a row per state, 32 jump columns, two halves of 16 filled in
// turn.  Separate reducer warps take each half when it is full: every
// observation group whose window meets those 16 jumps gets the weighted sum
// over them, sum_k w_{i,k} sum_{s in g} rho_k[s] (two FP32 FMA chains of at
// most 8 terms), added to the group's accumulator with a Kahan step, while
// the chain warps fill the other half.  Two mbarriers per half hand it over
// (full: the chain threads have written it; empty: the reducers have read
// it); every wait on them is bounded (p.wait_limit polls, MJP_OPT_WAIT_LIMIT)
// and reports kStatusTimeout when it runs out.  The reducers also stage the
// weights of Algorithm 2 (FP64 in the planner, rounded to FP32) from the
// planner's arena 32 jumps at a time, one chunk ahead; a window without a
// stored copy runs the recurrence P_k = P_{k-1} x / k from P_L (FP64) while
// its chunk is staged.
#include <algorithm>
#include <type_traits>

#include "chain_common.cuh"
#include "internal.cuh"

namespace mjp {

namespace {

constexpr int kHist = 16;        // jumps per observation chunk (half of the history)
constexpr int kWChunk = 32;      // jumps of weights staged at a time
constexpr int kWRing = 2 * kWChunk;
// Ring row stride: a multiple of 4 (a chunk's 16 weights are read as float4)
// that is not a multiple of 32, so that threads of a warp reading different
// times spread over the shared-memory banks.
constexpr int kWStride = kWRing + 4;
// History row stride (floats): 2 kHist jump columns (the two halves), padded
// so that the chain threads writing one jump's values spread over the banks.
constexpr int kHS = 2 * kHist + 4;
constexpr int kMaxChainWarps = 8;
constexpr int kReduceWarps = 2;

struct TsLayout {
  size_t edge, tx, tPL, ttail, twb, pw, tL, tK, trec, gptr, ring, gloc, gtime, acc_s, acc_c, hist, total;
};

// Floats of the history: a row per state slot (4 per pair slot: X.x, X.y,
// Y.x, Y.y, component-major) and a zero row (an absent second member).
__host__ __device__ inline size_t ts_hist(int nslot) { return (size_t)(4 * nslot + 1) * kHS; }

// Shared memory of one CTA: edge slots [2 parities][Wc + 2][3] (chain warps
// 0..Wc-1 in slots 1..Wc, zero slots 0 and Wc + 1 beyond the first and last),
// window tables, the weight ring [time][kWStride], the groups (member offsets
// in the history, time, Kahan sum and compensation), the history [state
// slot][jump column].
__host__ __device__ inline TsLayout ts_layout(int Wc, int nslot, int nt, int G) {
  TsLayout s;
  size_t o = 0;
  s.edge = o; o += align_up(4 * 2 * 3 * (size_t)(Wc + 2), 16);
  s.tx = o; o += 8 * (size_t)nt;
  s.tPL = o; o += 8 * (size_t)nt;
  s.ttail = o; o += 8 * (size_t)nt;
  s.twb = o; o += 8 * (size_t)nt;
  s.pw = o; o += 8 * (size_t)nt;
  s.tL = o; o += align_up(4 * (size_t)nt, 8);
  s.tK = o; o += align_up(4 * (size_t)nt, 8);
  s.trec = o; o += align_up(4 * (size_t)nt, 8);
  s.gptr = o; o += align_up(4 * (size_t)(nt + 1), 16);
  o = align_up(o, 16);  // the ring is read as float4
  s.ring = o; o += align_up(4 * (size_t)kWStride * nt, 16);
  s.gloc = o; o += 8 * (size_t)G;
  s.gtime = o; o += align_up(4 * (size_t)G, 8);
  s.acc_s = o; o += align_up(4 * (size_t)G, 8);
  s.acc_c = o; o += align_up(4 * (size_t)G, 16);
  o = align_up(o, 16);  // the history rows are read as float4
  s.hist = o; o += 4 * ts_hist(nslot);
  s.total = align_up(o, 16);
  return s;
}

// Calls f(T, a), f(T + 1, a), ..., f(T + N - 1, a) with compile-time T.
template <int T, int N>
struct TsSeq {
  template <class F, class A>
  __device__ __forceinline__ static void run(F& f, A a) {
    f(std::integral_constant<int, T>{}, a);
    TsSeq<T + 1, N - 1>::run(f, a);
  }
};
template <int T>
struct TsSeq<T, 0> {
  template <class F, class A>
  __device__ __forceinline__ static void run(F&, A) {}
};

// Shared-memory mbarriers (CTA scope): arrive releases this thread's prior
// shared-memory writes; a completed wait acquires those of every arriving
// thread.  The wait polls test_wait (non-blocking) with a short sleep and
// gives up after `polls` polls (returns false).
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(b);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(b);
  asm volatile("{ .reg .b64 st; mbarrier.arrive.shared::cta.b64 st, [%0]; }" ::"r"(a) : "memory");
}
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity, long long polls) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(b);
  for (long long i = 0; i < polls; ++i) {
    unsigned ok;
    asm volatile("{ .reg .pred p; mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                 : "=r"(ok) : "r"(a), "r"(parity) : "memory");
    if (ok) return true;
    __nanosleep(64);
  }
  return false;
}
// Named barrier of `count` threads (a multiple of 32), and the same with an
// AND of every thread's predicate.
__device__ __forceinline__ void named_sync(unsigned id, unsigned count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ bool named_and(unsigned id, unsigned count, bool v) {
  unsigned r;
  asm volatile("{ .reg .pred p, q; setp.ne.u32 p, %1, 0; bar.red.and.pred q, %2, %3, p; selp.u32 %0, 1, 0, q; }"
               : "=r"(r) : "r"((unsigned)v), "r"(id), "r"(count) : "memory");
  return r != 0;
}

// tlo: first chain thread whose columns hold an observed state; nslot = QP x
// the chain threads [tlo, tlo + nslot / QP) that write history.  Warps
// 0..Wc-1 run the chain, the others (kReduceWarps) reduce the observations.
template <int QP>
__global__ void __launch_bounds__(32 * (kMaxChainWarps + kReduceWarps))
    chain_regts_kernel(const ChainParams p, const int tlo, const int nslot, const int Wc) {
  constexpr int P1 = QP + 1;  // register rotation period; divides kHist
  static_assert(kHist % P1 == 0 && kHist % 8 == 0 && kWChunk == 2 * kHist, "chunk geometry");
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[kMaxChainWarps + kReduceWarps];
  __shared__ __align__(8) unsigned long long full_bar[2], empty_bar[2];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nthr = blockDim.x, NW = nthr >> 5;
  const int nchain = 32 * Wc, nred = nthr - nchain;
  const bool is_chain = warp < Wc;
  const int rtid = tid - nchain, rwarp = warp - Wc;  // reducer thread / warp index
  const int job = p.job_map ? p.job_map[blockIdx.x] : (int)blockIdx.x;
  const int nt = p.ntimes, M = p.M, G = p.G;
  const TsLayout Ly = ts_layout(Wc, nslot, nt, G);
  float* const edge = reinterpret_cast<float*>(smem + Ly.edge);  // [2][Wc + 2][last X, first X, first Y]
  double* t_x = reinterpret_cast<double*>(smem + Ly.tx);
  double* t_PL = reinterpret_cast<double*>(smem + Ly.tPL);
  double* t_tail = reinterpret_cast<double*>(smem + Ly.ttail);
  const float** t_wb = reinterpret_cast<const float**>(smem + Ly.twb);
  double* pw = reinterpret_cast<double*>(smem + Ly.pw);
  int* t_L = reinterpret_cast<int*>(smem + Ly.tL);
  int* t_K = reinterpret_cast<int*>(smem + Ly.tK);
  int* t_rec = reinterpret_cast<int*>(smem + Ly.trec);
  int* s_gptr = reinterpret_cast<int*>(smem + Ly.gptr);
  float* ring = reinterpret_cast<float*>(smem + Ly.ring);
  int2* gloc = reinterpret_cast<int2*>(smem + Ly.gloc);
  int* gtime = reinterpret_cast<int*>(smem + Ly.gtime);
  float* acc_s = reinterpret_cast<float*>(smem + Ly.acc_s);
  float* acc_c = reinterpret_cast<float*>(smem + Ly.acc_c);
  float* hist = reinterpret_cast<float*>(smem + Ly.hist);
  const float* arena = reinterpret_cast<const float*>(p.arena);

  // ---- prologue (all threads): windows, groups, coefficients, rho0 ----------
  if (tid == 0) {
    mbar_init(&full_bar[0], nchain);
    mbar_init(&full_bar[1], nchain);
    mbar_init(&empty_bar[0], nred);
    mbar_init(&empty_bar[1], nred);
  }
  const int64_t Kmax64 = p.info[job].Kmax;
  const Win* wj = p.win + (int64_t)job * nt;
  for (int i = tid; i < nt; i += nthr) {
    const Win w = wj[i];
    t_x[i] = w.x;
    t_PL[i] = w.PL;
    t_tail[i] = w.tail;
    t_L[i] = (int)w.L;
    t_K[i] = (int)w.K;
    t_rec[i] = (w.woff < 0 || !arena) ? 1 : 0;
    t_wb[i] = (w.woff >= 0 && arena) ? arena + (w.woff - w.L) : nullptr;
    pw[i] = w.PL;
  }
  for (int i = tid; i <= nt; i += nthr) s_gptr[i] = (int)p.gptr[i];
  // The planner caps K (MJP_OPT_K_CAP, default 2^26); the loop counts in 32 bits.
  const int Kmax = Kmax64 < (1LL << 30) ? (int)Kmax64 : 0;
  if (Kmax64 >= (1LL << 30) && tid == 0) set_status(p.status, kStatusKcap);
  for (int q = tid; q < (int)ts_hist(nslot); q += nthr) hist[q] = 0.0f;
  for (int q = tid; q < 2 * 3 * (Wc + 2); q += nthr) edge[q] = 0.0f;
  __syncthreads();  // the window tables and group pointers are read by every thread below
  // Group gq: its members (at most two) as float offsets of history rows,
  // its time, and a zero Kahan accumulator.  A member state s = m + M sigma
  // sits in chain thread g = m / (2 QP), pair j = (m mod 2 QP) mod QP, half
  // h = (m mod 2 QP) / QP: pair slot q = (g - tlo) QP + j, history row
  // (2 sigma + h) nslot + q.
  const int zero_off = 4 * nslot * kHS;
  auto place = [&](int s) -> int {
    const int sg = s >= M ? 1 : 0, m = s - sg * M;
    const int g = m / (2 * QP), r = m - g * 2 * QP, j = r % QP, h = r / QP;
    return ((2 * sg + h) * nslot + (g - tlo) * QP + j) * kHS;
  };
  for (int gq = tid; gq < G; gq += nthr) {
    const int q0 = (int)p.mptr[gq], q1 = (int)p.mptr[gq + 1];
    const int a = q1 > q0 ? place(p.members[q0]) : zero_off;
    const int b = q1 > q0 + 1 ? place(p.members[q0 + 1]) : zero_off;
    gloc[gq] = make_int2(a, b);
    acc_s[gq] = 0.0f;
    acc_c[gq] = 0.0f;
  }
  for (int i = warp; i < nt; i += NW)
    for (int gq = s_gptr[i] + lane; gq < s_gptr[i + 1]; gq += 32) gtime[gq] = i;
  const bool hist_me = is_chain && tid >= tlo && (tid - tlo) * QP < nslot;
  float* const hslot = hist + (hist_me ? (tid - tlo) * QP : 0) * kHS;  // pair 0, component X.x

  // Coefficients of a chain thread's states (rates into the state, scaled by
  // 1/Omega), zero outside the box so that padding states stay zero: birth
  // beta from m - 1 (active row only, m >= 1), death gamma (m + 1) from m + 1
  // (both rows, m + 1 < N_R), the negated exits, activation lambda_act into
  // the active and deactivation lambda_ina into the inactive row (shared),
  // and p.renorm x the exit defects.  Residuals start at zero.
  const Coef<float> co = make_coef<float, MJP_TWOSTATE>(p.theta + (int64_t)job * p.ntheta, p.info[job].omega);
  const float* rho0 = reinterpret_cast<const float*>(p.rho0);
  const int c0 = is_chain ? tid * 2 * QP : M;  // reducer threads hold nothing
  float2 X[P1], Y[P1];
  float2 al[QP], cr[QP], nx[QP], ny[QP], bX[QP], bY[QP], rX[QP], rY[QP];
#pragma unroll
  for (int j = 0; j < QP; ++j) {
    float va[2], vc[2], vx[2], vy[2], vbx[2], vby[2], x0[2], y0[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int m = c0 + h * QP + j;
      const bool in = m < M;
      const float bm = __fmul_rn(co.b, (float)m);
      const float ain = m + 1 < M ? co.a : 0.0f;
      const float ex = __fadd_rn(__fadd_rn(bm, ain), co.d), ey = __fadd_rn(co.c, bm);
      va[h] = (in && m >= 1) ? co.a : 0.0f;
      vc[h] = m + 1 < M ? __fmul_rn(co.b, (float)(m + 1)) : 0.0f;
      vx[h] = in ? -ex : 0.0f;
      vy[h] = in ? -ey : 0.0f;
      vbx[h] = (in && p.renorm > 0) ? (float)p.renorm * ts_defect(co, 0, m, M) : 0.0f;
      vby[h] = (in && p.renorm > 0) ? (float)p.renorm * ts_defect(co, 1, m, M) : 0.0f;
      x0[h] = in ? rho0[m] : 0.0f;
      y0[h] = in ? rho0[m + M] : 0.0f;
    }
    al[j] = make_float2(va[0], va[1]);
    cr[j] = make_float2(vc[0], vc[1]);
    nx[j] = make_float2(vx[0], vx[1]);
    ny[j] = make_float2(vy[0], vy[1]);
    bX[j] = make_float2(vbx[0], vbx[1]);
    bY[j] = make_float2(vby[0], vby[1]);
    X[j] = make_float2(x0[0], x0[1]);
    Y[j] = make_float2(y0[0], y0[1]);
    rX[j] = rY[j] = make_float2(0.0f, 0.0f);
  }
  X[QP] = Y[QP] = make_float2(0.0f, 0.0f);
  const float2 cc = make_float2(co.c, co.c), dd = make_float2(co.d, co.d);
  __syncthreads();  // the history is zero (and the mbarriers set) before any thread writes

  // History column of jump k: (k - 1) mod 2 kHist (rho_0 in the last); the
  // chain warps' edge values of rho_k in parity k mod 2.
  const int cstride = nslot * kHS;  // floats between the components of a pair slot
  auto write_hist = [&](int col, auto OC) {
    constexpr int O = decltype(OC)::value;
    if (hist_me) {
      float* h = hslot + col;
#pragma unroll
      for (int j = 0; j < QP; ++j) {
        const float2 x = X[(j + O) % P1], y = Y[(j + O) % P1];
        h[j * kHS] = x.x;
        h[j * kHS + cstride] = x.y;
        h[j * kHS + 2 * cstride] = y.x;
        h[j * kHS + 3 * cstride] = y.y;
      }
    }
  };
  float* const eown = edge + 3 * (warp + 1);  // a chain warp's slot (parity 0)
  const int epar = 3 * (Wc + 2);               // floats per parity
  auto write_edges = [&](int par, auto OC) {
    constexpr int O = decltype(OC)::value;
    float* e = eown + par * epar;
    if (lane == 31) e[0] = X[(QP - 1 + O) % P1].y;
    if (lane == 0) {
      e[1] = X[O % P1].x;
      e[2] = Y[O % P1].x;
    }
  };
  if (is_chain) {
    write_hist(2 * kHist - 1, std::integral_constant<int, 0>{});
    write_edges(0, std::integral_constant<int, 0>{});
  }

  // Weights into ring slot (k - 1) mod kWRing: chunk c holds jumps
  // [32 c + 1, 32 c + 32] (slots [32 c, 32 c + 32) mod 64), jump 0 slot 63.
  // Only the windows that meet the jumps are touched (ordered in L and K, a
  // contiguous range that moves forward); warp w of the lW staging warps
  // copies times w, w + lW, ..., lane l jump ka + l; windows without a stored
  // copy run the recurrence (one thread per time, chunks in jump order).
  int slo = 0, shi = -1;
  auto stage = [&](int ka, int kb, int ltid, int lnthr, int lwarp, int lW) {  // jumps [ka, kb], kb - ka < 32
    kb = min(kb, Kmax);
    if (kb < ka) return;
    while (slo < nt && t_K[slo] < ka) ++slo;
    while (shi + 1 < nt && t_L[shi + 1] <= kb) ++shi;
    const int j = ka + lane;
    for (int i = slo + lwarp; i <= shi; i += lW)
      if (j <= kb && t_wb[i] && j >= t_L[i] && j <= t_K[i])
        cp_async_elem(ring + i * kWStride + ((j - 1) & (kWRing - 1)), t_wb[i] + j);
    cp_async_commit();
    for (int i = slo + ltid; i <= shi; i += lnthr) {
      if (!t_rec[i]) continue;
      const int a = max(ka, t_L[i]), b = min(kb, t_K[i]);
      double P = pw[i];
      for (int jj = a; jj <= b; ++jj) {
        P = (jj == t_L[i]) ? t_PL[i] : __dmul_rn(P, __ddiv_rn(t_x[i], (double)jj));
        ring[i * kWStride + ((jj - 1) & (kWRing - 1))] = (float)(P + (jj == t_K[i] ? t_tail[i] : 0.0));
      }
      pw[i] = P;
    }
  };
  stage(0, 0, tid, nthr, warp, NW);
  stage(1, kWChunk, tid, nthr, warp, NW);
  cp_async_wait<0>();
  __syncthreads();

  // rho_0: the groups of the windows that start at jump 0 take their first
  // term (a zero accumulator: no rounding to carry).
  int wlo = 0, whi = -1;
  while (whi + 1 < nt && t_L[whi + 1] <= 0) ++whi;
  if (whi >= 0)
    for (int gq = tid; gq < s_gptr[whi + 1]; gq += nthr) {
      const int2 lq = gloc[gq];
      const float v = __fadd_rn(hist[lq.x + 2 * kHist - 1], hist[lq.y + 2 * kHist - 1]);
      acc_s[gq] = __fmul_rn(ring[gtime[gq] * kWStride + (kWRing - 1)], v);
    }
  whi = -1;
  __syncthreads();
  stage(kWChunk + 1, 2 * kWChunk, tid, nthr, warp, NW);  // chunk 1 (its slot 63 held jump 0's weight)
  cp_async_wait<0>();
  __syncthreads();

  // Observations of jumps [k0, k0 + kHist) (k0 = 1 mod kHist, capped at
  // Kmax), history columns hc + t: every group of a window that meets them
  // adds sum_k w_{i,k} rho_k(g) over its part of the chunk (two FMA chains,
  // even and odd jumps) to its Kahan accumulator.  Ring slot (k0 - 1) mod 64
  // + t holds jump k0 + t; history and weights are read four jumps at a time.
  // Windows of the sorted times are ordered in L and in K, so the groups
  // concerned form one index range.  Reducer threads.
  auto reduce = [&](int k0, int hc) {
    const int k1 = min(k0 + kHist - 1, Kmax);
    while (wlo < nt && t_K[wlo] < k0) ++wlo;
    while (whi + 1 < nt && t_L[whi + 1] <= k1) ++whi;
    if (wlo > whi) return;
    const int ga = s_gptr[wlo], gb = s_gptr[whi + 1];
    const int wbase = (k0 - 1) & (kWRing - 1);
    for (int gq = ga + rtid; gq < gb; gq += nred) {
      const int2 lq = gloc[gq];
      const int i = gtime[gq];
      const int ta = max(k0, t_L[i]) - k0, tb = min(k1, t_K[i]) - k0;  // jumps of the window in the chunk
      const unsigned live = ((2u << tb) - 1u) & ~((1u << ta) - 1u);
      const float4* wr = reinterpret_cast<const float4*>(ring + i * kWStride + wbase);
      const float4* ha = reinterpret_cast<const float4*>(hist + lq.x + hc);
      const float4* hb = reinterpret_cast<const float4*>(hist + lq.y + hc);
      float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
      for (int t4 = 0; t4 < kHist / 4; ++t4) {
        const float4 a = ha[t4], b = hb[t4], w = wr[t4];
        const float va[4] = {a.x, a.y, a.z, a.w}, vb[4] = {b.x, b.y, b.z, b.w}, ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int t = 4 * t4 + u;
          const float v = __fadd_rn(va[u], vb[u]);
          if (live & (1u << t)) {
            if (t & 1) s1 = __fmaf_rn(ww[u], v, s1);
            else s0 = __fmaf_rn(ww[u], v, s0);
          }
        }
      }
      const float s = __fadd_rn(s0, s1);
      const float y = __fsub_rn(s, acc_c[gq]);
      const float a0 = acc_s[gq];
      const float tt = __fadd_rn(a0, y);
      acc_c[gq] = __fsub_rn(__fsub_rn(tt, a0), y);
      acc_s[gq] = tt;
    }
  };

  // ---- the chain warps and the reducer warps ---------------------------------
  const int nq = (Kmax + kHist - 1) / kHist;  // chunks of jumps [kHist q + 1, kHist q + kHist]
  bool ok = true;
  if (is_chain) {
    // Jump t of a chunk (k = kHist q + 1 + t) in place: rho_{k-1} with pair j
    // in slot (j + O) mod P1, O = -t mod P1 -> rho_k with pair j in slot
    // (j + O - 1) mod P1.  Per state, in the shared-memory kernel's order:
    // residual, inflow from n_R - 1 (active row), from n_R + 1, from the
    // other gene state, the exit, then comp_finish.  The values just outside
    // a thread's columns come from the neighbour lanes (shuffles) and, across
    // warps, from the edge slots of rho_{k-1} (parity t mod 2); at the box
    // ends their coefficients are zero.  Terms with such a value are two
    // scalar FMAs (the same roundings as one FP32x2 FMA, without assembling a
    // register pair).  The exit defects are added back after jumps that are
    // multiples of p.renorm (a multiple of 8, so t = 7 or 15); rho_k goes to
    // history column hc + t.  CHECK: the last chunk, whose jumps may pass Kmax.
    auto chain_sync = [&]() {
      if (Wc > 1) named_sync(1, nchain);
      else __syncwarp();
    };
    auto chain_all = [&](bool v) -> bool { return Wc > 1 ? named_and(1, nchain, v) : __all_sync(kFull, v) != 0; };
    int k = 1, hc = 0;
    int d8 = p.renorm > 0 ? p.renorm / 8 : 0x7fffffff;  // 8-jump blocks to the next defect correction
    auto jump = [&](auto TC, auto CHECKC) {
      constexpr int t = decltype(TC)::value;
      constexpr bool CHECK = decltype(CHECKC)::value;
      constexpr int O = (P1 - t % P1) % P1;
      constexpr int ON = (O + P1 - 1) % P1;
      if (CHECK && k > Kmax) return;
      const float* e = eown + (t & 1) * epar;  // a warp's own slot is never read
      const float eL = e[-3], eRX = e[4], eRY = e[5];
      const float lastXy = X[(QP - 1 + O) % P1].y, lastXx = X[(QP - 1 + O) % P1].x;
      const float fXx = X[O % P1].x, fXy = X[O % P1].y, fYx = Y[O % P1].x, fYy = Y[O % P1].y;
      float lin = __shfl_up_sync(kFull, lastXy, 1);
      float rinX = __shfl_down_sync(kFull, fXx, 1);
      float rinY = __shfl_down_sync(kFull, fYx, 1);
      lin = lane == 0 ? eL : lin;
      rinX = lane == 31 ? eRX : rinX;
      rinY = lane == 31 ? eRY : rinY;
#pragma unroll
      for (int j = 0; j < QP; ++j) {
        const float2 cx = X[(j + O) % P1], cy = Y[(j + O) % P1];
        float2 tx, ty;
        if (j == 0) {  // left of column c0: lin; left of c0 + QP: column c0 + QP - 1
          tx.x = __fmaf_rn(al[j].x, lin, rX[j].x);
          tx.y = __fmaf_rn(al[j].y, lastXx, rX[j].y);
        } else {
          tx = v_fma(al[j], X[(j - 1 + O) % P1], rX[j]);
        }
        if (j + 1 == QP) {  // right of column c0 + QP - 1: c0 + QP; of c0 + 2 QP - 1: rin
          tx.x = __fmaf_rn(cr[j].x, fXy, tx.x);
          tx.y = __fmaf_rn(cr[j].y, rinX, tx.y);
          ty.x = __fmaf_rn(cr[j].x, fYy, rY[j].x);
          ty.y = __fmaf_rn(cr[j].y, rinY, rY[j].y);
        } else {
          tx = v_fma(cr[j], X[(j + 1 + O) % P1], tx);
          ty = v_fma(cr[j], Y[(j + 1 + O) % P1], rY[j]);
        }
        tx = v_fma(cc, cy, tx);
        tx = v_fma(nx[j], cx, tx);
        const float2 yx = comp_finish(cx, tx, rX[j]);
        ty = v_fma(dd, cx, ty);
        ty = v_fma(ny[j], cy, ty);
        const float2 yy = comp_finish(cy, ty, rY[j]);
        const int d = j == 0 ? (O + QP) % P1 : (j - 1 + O) % P1;
        X[d] = yx;
        Y[d] = yy;
      }
      if ((t & 7) == 7 && --d8 == 0) {
        d8 = p.renorm / 8;
#pragma unroll
        for (int j = 0; j < QP; ++j) {
          rX[j] = v_fma(bX[j], X[(j + ON) % P1], rX[j]);
          rY[j] = v_fma(bY[j], Y[(j + ON) % P1], rY[j]);
        }
      }
      write_hist(hc + t, std::integral_constant<int, ON>{});
      write_edges((t + 1) & 1, std::integral_constant<int, ON>{});
      chain_sync();
      ++k;
    };
    // Chunk q fills history half q mod 2 once the reducers have emptied it
    // (chunk q - 2), then hands it over; at the end, wait until the reducers
    // have read the last two chunks.
    for (int q = 0; q < nq && ok; ++q) {
      if (q >= 2) ok = chain_all(mbar_wait(&empty_bar[q & 1], ((q >> 1) - 1) & 1, p.wait_limit));
      if (!ok) break;
      hc = kHist * (q & 1);
      if (kHist * q + kHist <= Kmax) TsSeq<0, kHist>::run(jump, std::false_type{});
      else TsSeq<0, kHist>::run(jump, std::true_type{});
      mbar_arrive(&full_bar[q & 1]);
    }
    for (int q = nq; q < nq + 2 && ok; ++q)
      if (q >= 2) ok = chain_all(mbar_wait(&empty_bar[q & 1], ((q >> 1) - 1) & 1, p.wait_limit));
    if (!ok && tid == 0) set_status(p.status, kStatusTimeout);
  } else {
    auto red_sync = [&]() { named_sync(2, nred); };
    for (int q = 0; q < nq && ok; ++q) {
      ok = named_and(2, nred, mbar_wait(&full_bar[q & 1], (q >> 1) & 1, p.wait_limit));
      if (!ok) break;
      cp_async_wait<0>();
      red_sync();  // the weights every reducer staged for this chunk have landed
      reduce(kHist * q + 1, kHist * (q & 1));
      mbar_arrive(&empty_bar[q & 1]);
      red_sync();  // every reducer is done with the slots of a finished weight chunk
      if (q & 1) {
        const int c = (q + 3) / 2;
        stage(kWChunk * c + 1, kWChunk * c + kWChunk, rtid, nred, rwarp, NW - Wc);
      }
    }
    cp_async_wait<0>();
    if (!ok && rtid == 0) set_status(p.status, kStatusTimeout);
  }
  __syncthreads();

  // ---- epilogue: sum_g c_g log(a_g) ------------------------------------------
  double ll = 0.0;
  bool bad = false;
  for (int gq = tid; gq < G; gq += nthr) {
    const double a = (double)acc_s[gq] - (double)acc_c[gq];
    const double c = p.counts[gq];
    if (c == 0.0) continue;
    if (a > 0.0) ll += c * log(a);
    else if (a > -1e-30) ll = -INFINITY;
    else bad = true;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ll += __shfl_xor_sync(kFull, ll, o);
  if (lane == 0) red[warp] = ll;
  __syncthreads();
  if (tid == 0) {
    double tot = 0.0;
    for (int w = 0; w < NW; ++w) tot += red[w];
    if (isnan(tot)) set_status(p.status, kStatusNumeric);
    p.ll[job] = tot;
  }
  if (bad) set_status(p.status, kStatusNumeric);
}

}  // namespace

// Chain warps, state pairs per thread and row (QP; the rotation period
// QP + 1 divides the history chunk) and the history slots for a two-state
// box of N_R = M columns whose observed states lie in columns [col_lo,
// col_hi] (col_lo < 0: no observations), or false when the kernel does not
// apply (then the shared-memory kernel runs): groups of more than two
// members, or a box or group table too large for one CTA.  A CTA is the
// chain warps plus kReduceWarps reducer warps.  Automatic: QP = 1 (then 3,
// then 7) with the fewest chain warps; threads = 32 Wc asks for Wc chain
// warps with the smallest QP that covers the box.
bool chain_regts_plan(int64_t M, int ntimes, int G, int maxmem, int col_lo, int col_hi, int threads,
                      RegTsPlan* out) {
  if (M < 2 || ntimes < 1 || G < 0 || maxmem > 2) return false;
  if (threads != 0 && (threads % 32 != 0 || threads < 32 || threads > 32 * kMaxChainWarps)) return false;
  const int qps[3] = {1, 3, 7};
  for (int qi = 0; qi < 3; ++qi) {
    const int qp = qps[qi];
    const int Wc = threads ? threads / 32 : (int)((M + 64 * qp - 1) / (64 * qp));
    if (Wc < 1 || Wc > kMaxChainWarps || (int64_t)64 * Wc * qp < M) continue;
    const int tlo = col_lo >= 0 ? col_lo / (2 * qp) : 0;
    const int thi = col_lo >= 0 ? col_hi / (2 * qp) : -1;
    const int nslot = (thi - tlo + 1) * qp;
    const TsLayout L = ts_layout(Wc, nslot, ntimes, G);
    if (L.total + 1024 > (size_t)227 * 1024) continue;
    // float4 sections on 16 bytes, double and pointer sections on 8.
    if (L.ring % 16 || L.hist % 16 || L.tx % 8 || L.twb % 8 || L.pw % 8 || L.gloc % 8) return false;
    out->threads = 32 * (Wc + kReduceWarps);
    out->chain_warps = Wc;
    out->qp = qp;
    out->tlo = tlo;
    out->nslot = nslot;
    out->smem = L.total;
    return true;
  }
  return false;
}

template <int QP>
cudaError_t launch_regts_typed(const ChainParams& p, const RegTsPlan& rp, cudaStream_t s) {
  static int smem_set = 0;
  auto kern = chain_regts_kernel<QP>;
  if ((int)rp.smem > smem_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rp.smem);
    if (e != cudaSuccess) return e;
    smem_set = (int)rp.smem;
  }
  kern<<<p.B, rp.threads, rp.smem, s>>>(p, rp.tlo, rp.nslot, rp.chain_warps);
  return cudaGetLastError();
}

cudaError_t launch_chain_regts(const ChainParams& p, const RegTsPlan& rp, cudaStream_t s) {
  if (p.B <= 0) return cudaSuccess;
  switch (rp.qp) {
    case 1: return launch_regts_typed<1>(p, rp, s);
    case 3: return launch_regts_typed<3>(p, rp, s);
    case 7: return launch_regts_typed<7>(p, rp, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mjp
