// stencil_reg1d.cu -- register-resident jump chain for birth-death instances
// (Eq. BD_def, reflecting top; expv mode, FP32 and FP64): Algorithm 2 with one
// chain shared by all times of an instance.
//
// Layout.  Thread t of a CTA holds R = 2 QP consecutive states of the CTA's
// segment in registers, as QP pairs: pair j = (state x0 + j, state x0 + QP + j)
// with x0 = t R.  The stencil neighbours of pair j are then pairs j - 1 and
// j + 1 component by component, so the update runs on whole pairs (packed
// FP32x2 instructions) and only the two ends of a thread's run need another
// thread's value.  Those come through shared memory (the first and last state
// of every thread, double-buffered by jump parity, with a zero slot at the
// segment's ends): one CTA barrier per jump.
//
// Clusters with temporal blocking.  An instance too large for one CTA's
// registers, or long enough to set a batch's makespan, runs on a cluster of C
// CTAs.  CTA r owns states [r S, r S + S) and also carries a halo of h states
// on each side.  It advances h jumps without hearing from its neighbours: after
// j jumps only the states within distance j of the halo's outer edge are
// stale, which never reaches the owned states.  Then the CTAs copy their
// outermost h owned states into each other's halos through distributed shared
// memory and meet at one cluster barrier, so the cluster barrier (~550 cycles
// on GB300) is paid once per h jumps instead of once per jump.
//
// Arithmetic per state is the shared-memory kernel's (stencil.cu) operation
// sequence in the same order, and the weighted accumulation is the same
// Kahan (FP32) or plain (FP64) sum in jump order, with the same weights, so
// both kernels give bit-identical outputs for every cluster shape and halo.
// FP32 chains run the compensated jump of chain_common.cuh (each state carries
// its rounding residual, and every p.renorm jumps the exact defect of its
// exit coefficient is added back); the residuals travel with the values in
// every halo exchange, so halo copies evolve exactly like their owners.
#include <cooperative_groups.h>

#include <algorithm>

#include <type_traits>

#include "chain_common.cuh"
#include "internal.cuh"

namespace cg = cooperative_groups;

namespace mjp {

namespace {

constexpr int kChunk1 = 32;           // jumps of weights staged at a time
constexpr int kStage1 = 2 * kChunk1;  // ring slots per time

struct Reg1dLayout {
  size_t wh, whl, recv, recvl, tx, tPL, ttail, twb, pw, tL, tK, trec, torig, ring, acc_s, acc_c, total;
};

// Shared memory of one CTA: the warps' halo runs [round parity][left, right]
// [warp][pair], the cluster halo receive buffers [exchange parity][left,
// right][h] (FP32: each with a twin for the chain residuals), the windows, the
// weight ring [time][kStage1], the accumulators [time][pair][thread] (pairs of
// T; FP32 adds the Kahan compensations).
__host__ __device__ inline Reg1dLayout reg1d_layout(size_t elt, int threads, int qp, int halo, int nt) {
  Reg1dLayout s;
  size_t o = 0;
  const bool comp = elt == 4;  // FP32: compensated chain, residuals beside the values
  s.wh = o; o += align_up(elt * 2 * 4 * (size_t)(threads / 32) * qp, 16);
  s.whl = o; if (comp) o += align_up(4 * 2 * 4 * (size_t)(threads / 32) * qp, 16);
  s.recv = o; o += align_up(elt * 4 * (size_t)(halo > 0 ? halo : 1), 16);
  s.recvl = o; if (comp) o += align_up(4 * 4 * (size_t)(halo > 0 ? halo : 1), 16);
  s.tx = o; o += 8 * (size_t)nt;
  s.tPL = o; o += 8 * (size_t)nt;
  s.ttail = o; o += 8 * (size_t)nt;
  s.twb = o; o += 8 * (size_t)nt;
  s.pw = o; o += 16 * (size_t)nt;
  s.tL = o; o += align_up(4 * (size_t)nt, 8);
  s.tK = o; o += align_up(4 * (size_t)nt, 8);
  s.trec = o; o += align_up(4 * (size_t)nt, 8);
  s.torig = o; o += align_up(4 * (size_t)nt, 8);
  o = align_up(o, 16);  // pairs of doubles below are 16-byte accesses
  s.ring = o; o += align_up(elt * kStage1 * (size_t)nt, 16);
  s.acc_s = o; o += align_up(elt * 2 * (size_t)qp * threads * nt, 16);
  s.acc_c = o;
  if (elt == 4) o += align_up(4 * 2 * (size_t)qp * threads * nt, 16);
  s.total = align_up(o, 16);
  return s;
}

// Warps of a CTA for a segment of ext states: one window of 64 qp states, or
// windows that overlap by two lanes' runs (2 x 2 qp states).
__host__ __device__ inline int reg1d_warps(int ext, int qp) {
  const int win = 64 * qp, wo = 60 * qp;
  return ext <= win ? 1 : (ext + wo - 1) / wo;
}

// Calls f(O) for N successive register rotations O, O - 1, ... (mod P1).
template <int P1, int O, int N>
struct RotSeq {
  template <class F>
  __device__ __forceinline__ static void run(F& f) {
    f(std::integral_constant<int, O>{});
    RotSeq<P1, (O + P1 - 1) % P1, N - 1>::run(f);
  }
};
template <int P1, int O>
struct RotSeq<P1, O, 0> {
  template <class F>
  __device__ __forceinline__ static void run(F&) {}
};

template <typename T, int QP, int kMaxT>
__global__ void __launch_bounds__(kMaxT, 1) chain_reg1d_kernel(const ChainParams p, const int halo) {
  using T2 = typename Pair<T>::type;
  constexpr int R = 2 * QP;       // states per lane
  constexpr int P1 = QP + 1;      // register rotation period = jumps per round
  constexpr int WIN = 32 * R;     // states of a warp's window
  static_assert(kChunk1 % P1 == 0 && P1 <= R, "rounds must tile the weight chunks and fit a warp halo");
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int job = p.job_map ? p.job_map[blockIdx.x / C] : (int)(blockIdx.x / C);
  const int tid = threadIdx.x, nthr = blockDim.x, warp = tid >> 5, lane = tid & 31;
  const int nt = p.ntimes;
  const int N = p.jobN ? p.jobN[job] : (int)p.N;
  const int S = (N + C - 1) / C;                     // owned states per CTA
  const int start = rank * S;
  const int own = max(0, min(N, start + S) - start);
  // CTA halo width: at least one round, at most what the last CTA owns (its
  // first h states fill the previous CTA's right halo); the host keeps the
  // last CTA's share >= P1.
  const int h = C > 1 ? min(max(halo, P1), N - (C - 1) * S) : 0;
  const int xb = start - h;                          // state at segment coordinate 0
  const int ext = own + 2 * h;                       // segment: halo, owned, halo
  // Warps: warp w owns segment coordinates [w Wo, (w+1) Wo) and holds its
  // window [w Wo - sw, w Wo - sw + WIN), sw = one lane's run when several
  // warps share the segment; lane l holds window coordinates [l R, l R + R)
  // as pairs (y0 + j, y0 + QP + j).
  const int nwu = reg1d_warps(ext, QP);
  const int sw = nwu > 1 ? R : 0;
  const int Wo = WIN - 2 * sw;
  const bool wact = warp < nwu;
  const int y0 = lane * R;
  const int xw = warp * Wo - sw;                     // segment coordinate of window coordinate 0
  const int64_t out_base = p.job_off ? p.job_off[job] : (int64_t)job * p.out_stride;

  const Reg1dLayout Ly = reg1d_layout(sizeof(T), nthr, QP, h, nt);
  constexpr bool kComp = sizeof(T) == 4;                  // compensated FP32 chain
  T2* const wh = reinterpret_cast<T2*>(smem + Ly.wh);    // [2][2][nthr / 32][QP]
  float2* const whl = reinterpret_cast<float2*>(smem + Ly.whl);  // residuals, same shape (FP32)
  T* const recv = reinterpret_cast<T*>(smem + Ly.recv);  // [2][2][h]
  float* const recvl = reinterpret_cast<float*>(smem + Ly.recvl);  // residuals, same shape (FP32)
  double* t_x = reinterpret_cast<double*>(smem + Ly.tx);
  double* t_PL = reinterpret_cast<double*>(smem + Ly.tPL);
  double* t_tail = reinterpret_cast<double*>(smem + Ly.ttail);
  const T** t_wb = reinterpret_cast<const T**>(smem + Ly.twb);
  double* pw = reinterpret_cast<double*>(smem + Ly.pw);
  int* t_L = reinterpret_cast<int*>(smem + Ly.tL);
  int* t_K = reinterpret_cast<int*>(smem + Ly.tK);
  int* t_rec = reinterpret_cast<int*>(smem + Ly.trec);
  int* t_orig = reinterpret_cast<int*>(smem + Ly.torig);
  T* ring = reinterpret_cast<T*>(smem + Ly.ring);
  T2* acc_s = reinterpret_cast<T2*>(smem + Ly.acc_s);
  float2* acc_c = reinterpret_cast<float2*>(smem + Ly.acc_c);
  const T* arena = reinterpret_cast<const T*>(p.arena);
  const int NW = nthr >> 5;

  // ---- prologue: windows, coefficients, rho0 --------------------------------
  const int64_t Kmax64 = p.info[job].Kmax;
  const Win* wj = p.win + (int64_t)job * nt;
  for (int i = tid; i < nt; i += nthr) {
    const Win w = wj[i];
    t_x[i] = w.x;
    t_PL[i] = w.PL;
    t_tail[i] = w.tail;
    t_L[i] = (int)w.L;
    t_K[i] = (int)w.K;
    t_orig[i] = p.orig ? p.orig[i] : i;
    t_rec[i] = (w.woff < 0 || !arena) ? 1 : 0;
    t_wb[i] = (w.woff >= 0 && arena) ? arena + (w.woff - w.L) : nullptr;
    pw[i] = (w.L == 0) ? w.PL : 0.0;
    if (w.L == 0 && (w.woff < 0 || !arena))  // jump 0 of a window without a stored copy
      ring[i * kStage1] = (T)(w.PL + (w.K == 0 ? w.tail : 0.0));
  }
  const double omega = p.info[job].omega;
  const Coef<T> co = make_coef<T, MJP_BD1D>(p.theta + (int64_t)job * p.ntheta, omega);
  const int Kmax = Kmax64 < (1LL << 30) ? (int)Kmax64 : 0;
  if (Kmax64 >= (1LL << 30) && tid == 0 && rank == 0) set_status(p.status, kStatusKcap);

  // Coefficients of every held state n (rates into n, scaled by 1/Omega): the
  // diagonal 1 - e_n (FP64) or the negated exit -e_n (FP32, compensated jump)
  // and the death rate gamma (n+1) from n+1, both zero outside the segment or
  // the box, and the latter zero at n = N - 1 too (what is held beyond the box
  // is not kept at zero, so it must not be read).  Values entering a lane's run
  // from outside its warp's window are stale by design (halo) except at the
  // segment's left end, where the inflow coefficient of the first state is zero
  // instead (the state left of it is void).  FP32 also keeps, per state, the
  // residual (zero at the start) and p.renorm times the defect of its exit,
  // e_n - (beta + gamma n) with the outflow coefficients as the neighbours
  // apply them (bd_defect).
  const T one = (T)1;
  const T* rho0 = reinterpret_cast<const T*>(p.rho0);
  const int64_t s0 = p.job_s0 ? p.job_s0[job] : -1;
  // r[QP] is a spare pair: the pairs rotate through all QP + 1 slots (below);
  // at a round's end pair j is back in r[j].  res[j] and cb[j] belong to pair
  // j wherever its value sits.
  T2 r[QP + 1], dg[QP], up[QP];
  float2 res[QP], cb[QP];
  r[QP] = v_make((T)0, (T)0);
  // States held outside the segment or the box receive inflow from their left
  // neighbour (the birth coefficient is shared by the run) and hold nothing
  // the chain needs; they are reset to zero at every round end so that they
  // stay finite (0 x inf would otherwise reach the box, and a stale halo
  // state could read an infinity).  Bit 2 j + c: pair j, component c lies
  // outside.
  unsigned outmask = 0;
#pragma unroll
  for (int j = 0; j < QP; ++j) {
    T dv[2], uv[2], rv[2];
    float bv[2];
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const int x = xw + y0 + hh * QP + j;
      const int n = xb + x;
      const bool in = wact && x >= 0 && x < ext && n >= 0 && n < N;
      if (!in) outmask |= 1u << (2 * j + hh);
      const T fm = (T)n;
      const T bn = f_mul(co.b, fm);
      const T ain = n + 1 < N ? co.a : (T)0;
      const T e = f_add(bn, ain);
      dv[hh] = in ? (kComp ? -e : f_sub(one, e)) : (T)0;
      uv[hh] = (in && n + 1 < N) ? f_mul(co.b, f_add(fm, one)) : (T)0;
      rv[hh] = !in ? (T)0 : (s0 >= 0 ? (T)(n == s0 ? 1 : 0) : rho0[n]);
      bv[hh] = (kComp && in && p.renorm > 0) ? (float)p.renorm * bd_defect(co, n, N) : 0.0f;
    }
    dg[j] = v_make(dv[0], dv[1]);
    up[j] = v_make(uv[0], uv[1]);
    r[j] = v_make(rv[0], rv[1]);
    res[j] = make_float2(0.0f, 0.0f);
    cb[j] = make_float2(bv[0], bv[1]);
  }
  const T2 a2 = v_make(co.a, co.a);
  const T2 a2first = v_make(warp == 0 && lane == 0 ? (T)0 : co.a, co.a);  // pair 0's inflow from the left

  // ---- halo exchanges -------------------------------------------------------
  // Cluster: every CTA copies its outermost h owned states into the
  // neighbours' halos (distributed shared memory), by the lanes that own
  // them; recv[ep][side][q], side 0 = left halo (from rank - 1), 1 = right.
  T* rmtL = nullptr;
  T* rmtR = nullptr;
  float* rmtLl = nullptr;
  float* rmtRl = nullptr;
  if (C > 1) {
    if (rank > 0) {
      rmtL = cluster.map_shared_rank(recv, rank - 1);
      if (kComp) rmtLl = cluster.map_shared_rank(recvl, rank - 1);
    }
    if (rank + 1 < C) {
      rmtR = cluster.map_shared_rank(recv, rank + 1);
      if (kComp) rmtRl = cluster.map_shared_rank(recvl, rank + 1);
    }
  }
  const int xo0 = xw + max(sw, y0), xo1 = xw + min(sw + Wo, y0 + R);  // segment range this lane owns
  const bool cl_send = C > 1 && wact && xo0 < xo1 &&
                       ((rank > 0 && xo0 < 2 * h && xo1 > h) || (rank + 1 < C && xo0 < own + h && xo1 > own));
  const bool cl_recv = C > 1 && wact && xo0 < xo1 &&
                       ((rank > 0 && xo0 < h) || (rank + 1 < C && xo0 < own + 2 * h && xo1 > own + h));
  auto owned_y = [&](int y) { return y >= sw && y < sw + Wo; };
  auto cluster_exchange = [&](int ep) {
    if (cl_send) {
#pragma unroll
      for (int j = 0; j < QP; ++j)
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int y = y0 + hh * QP + j, x = xw + y;
          const T v = hh ? r[j].y : r[j].x;
          const float vl = hh ? res[j].y : res[j].x;
          if (!owned_y(y)) continue;
          if (rmtL && x >= h && x < 2 * h) {
            rmtL[(ep * 2 + 1) * h + (x - h)] = v;
            if (kComp) rmtLl[(ep * 2 + 1) * h + (x - h)] = vl;
          }
          if (rmtR && x >= own && x < own + h) {
            rmtR[(ep * 2 + 0) * h + (x - own)] = v;
            if (kComp) rmtRl[(ep * 2 + 0) * h + (x - own)] = vl;
          }
        }
      fence_cluster();
    }
    cluster_arrive_relaxed();
    cluster_wait();
    if (cl_recv) {
#pragma unroll
      for (int j = 0; j < QP; ++j) {
        T v0 = r[j].x, v1 = r[j].y;
        float l0 = res[j].x, l1 = res[j].y;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          const int y = y0 + hh * QP + j, x = xw + y;
          T v = hh ? v1 : v0;
          float l = hh ? l1 : l0;
          if (owned_y(y) && rank > 0 && x < h) {
            v = recv[(ep * 2 + 0) * h + x];
            if (kComp) l = recvl[(ep * 2 + 0) * h + x];
          }
          if (owned_y(y) && rank + 1 < C && x >= own + h && x < own + 2 * h) {
            v = recv[(ep * 2 + 1) * h + (x - own - h)];
            if (kComp) l = recvl[(ep * 2 + 1) * h + (x - own - h)];
          }
          if (hh) {
            v1 = v;
            l1 = l;
          } else {
            v0 = v;
            l0 = l;
          }
        }
        r[j] = v_make(v0, v1);
        res[j] = make_float2(l0, l1);
      }
    }
  };
  // Warps: lane 1's run (the warp's first owned states) becomes lane 31's
  // run (right halo) of the warp to the left, lane 30's run becomes lane 0's
  // run (left halo) of the warp to the right; whole runs, pair by pair,
  // through shared memory and one CTA barrier.  wh[rp][side][w][j], side 0 =
  // left halo of warp w.
  auto warp_exchange = [&](int rp) {
    if (wact && ((lane == 1 && warp > 0) || (lane == 30 && warp + 1 < nwu))) {
      const int off = ((rp * 2 + (lane == 1 ? 1 : 0)) * NW + (lane == 1 ? warp - 1 : warp + 1)) * QP;
#pragma unroll
      for (int j = 0; j < QP; ++j) {
        wh[off + j] = r[j];
        if (kComp) whl[off + j] = res[j];
      }
    }
    __syncthreads();
    if (wact && ((lane == 0 && warp > 0) || (lane == 31 && warp + 1 < nwu))) {
      const int off = ((rp * 2 + (lane == 0 ? 0 : 1)) * NW + warp) * QP;
#pragma unroll
      for (int j = 0; j < QP; ++j) {
        r[j] = wh[off + j];
        if (kComp) res[j] = whl[off + j];
      }
    }
  };

  bool mine_rec = false;
  for (int i = tid; i < nt; i += nthr) mine_rec |= t_rec[i] != 0;
  // Every CTA of the cluster is running (and its tables are set) before any
  // distributed-shared-memory write.
  if (C > 1) cluster.sync();
  const bool any_rec = __syncthreads_or(mine_rec) != 0;

  int lo = 0, hi = -1;
  auto advance = [&](int k, int& l, int& hgh) {
    while (l < nt && t_K[l] < k) ++l;
    while (hgh + 1 < nt && t_L[hgh + 1] <= k) ++hgh;
  };
  advance(0, lo, hi);
  // Stored weights of jumps [k0, k0 + kChunk1) of every window into the ring
  // (slot j % kStage1), spread over all threads.
  auto stage_chunk = [&](int k0) {
    const int k1 = min(k0 + kChunk1, Kmax + 1);
    for (int e = tid; e < nt * kChunk1; e += nthr) {
      const int i = e / kChunk1, j = k0 + (e - i * kChunk1);
      if (j < k1 && t_wb[i] && j >= t_L[i] && j <= t_K[i])
        cp_async_elem(ring + i * kStage1 + (j & (kStage1 - 1)), t_wb[i] + j);
    }
    cp_async_commit();
  };
  // Weights of jump kn for windows without a stored copy (Algorithm 2's
  // recurrence P_kn = P_{kn-1} x / kn from P_L, tail added at K); warp 0.
  int rlo = lo, rhi = hi;
  auto rec_step = [&](int kn) {
    advance(kn, rlo, rhi);
    const double* rprev = pw + ((kn - 1) & 1) * nt;
    double* rcur = pw + (kn & 1) * nt;
    for (int i = rlo + lane; i <= rhi; i += 32) {
      if (!t_rec[i]) continue;
      const double Pk = (kn == t_L[i]) ? t_PL[i] : __dmul_rn(rprev[i], __ddiv_rn(t_x[i], (double)kn));
      rcur[i] = Pk;
      ring[i * kStage1 + (kn & (kStage1 - 1))] = (T)(Pk + (kn == t_K[i] ? t_tail[i] : 0.0));
    }
  };
  auto rec_round = [&](int k1, int k2) {  // jumps [k1, k2]
    if (warp == 0 && any_rec)
      for (int kn = k1; kn <= k2; ++kn) {
        rec_step(kn);
        __syncwarp();
      }
  };

  // rho*_i += w_{i,k} rho_k for the active times [l, hgh] of jump k (Kahan in
  // FP32), the result written out at k = K_i for the states this lane owns;
  // rho_k's pairs at rotation O.
  // Bit 2 j (2 j + 1): state y0 + j (y0 + QP + j) of this lane is owned by
  // it and lies in this CTA's segment, so its outputs are its to write.
  unsigned omask = 0;
#pragma unroll
  for (int j = 0; j < QP; ++j) {
    const int ya = y0 + j, yc = y0 + QP + j;
    if (owned_y(ya) && xw + ya >= h && xw + ya < h + own) omask |= 1u << (2 * j);
    if (owned_y(yc) && xw + yc >= h && xw + yc < h + own) omask |= 2u << (2 * j);
  }
  auto accumulate = [&](int k, int l, int hgh, auto OC) {
    constexpr int O = decltype(OC)::value;
    for (int i = l; i <= hgh; ++i) {
      const T w = ring[i * kStage1 + (k & (kStage1 - 1))];
      const bool first = k == t_L[i], last = k == t_K[i];
      T* const o = reinterpret_cast<T*>(p.out) + out_base + (int64_t)t_orig[i] * N + xb + xw;
#pragma unroll
      for (int j = 0; j < QP; ++j) {
        const int slot = (i * QP + j) * nthr + tid;
        const T2 v = r[(j + O) % P1];
        const int ya = y0 + j, yc = y0 + QP + j;
        const bool oa = (omask >> (2 * j)) & 1u, oc = (omask >> (2 * j + 1)) & 1u;
        if (sizeof(T) == 4) {
          // Kahan step of both states as FP32x2 operations, each lane rounded
          // as the scalar step: y = w v - c, t = s + y, c = (t - s) - y.
          const float2 w2 = make_float2((float)w, (float)w), m1 = make_float2(-1.0f, -1.0f);
          const float2 vf = make_float2((float)v.x, (float)v.y);
          float2 s, cc;
          if (first) {
            s = __fmul2_rn(w2, vf);
            cc = make_float2(0.0f, 0.0f);
          } else {
            const T2 s0v = acc_s[slot];
            s = make_float2((float)s0v.x, (float)s0v.y);
            cc = acc_c[slot];
            const float2 y = __ffma2_rn(cc, m1, __fmul2_rn(w2, vf));
            const float2 t = __fadd2_rn(s, y);
            cc = __ffma2_rn(y, m1, __ffma2_rn(s, m1, t));
            s = t;
          }
          if (last) {
            if (oa) o[ya] = (T)__fsub_rn(s.x, cc.x);
            if (oc) o[yc] = (T)__fsub_rn(s.y, cc.y);
          } else {
            acc_s[slot] = v_make((T)s.x, (T)s.y);
            acc_c[slot] = cc;
          }
        } else {
          T2 s;
          if (first) s = v_make(f_mul(w, v.x), f_mul(w, v.y));
          else {
            const T2 s0v = acc_s[slot];
            s = v_make(f_fma(w, v.x, s0v.x), f_fma(w, v.y, s0v.y));
          }
          if (last) {
            if (oa) o[ya] = s.x;
            if (oc) o[yc] = s.y;
          } else {
            acc_s[slot] = s;
          }
        }
      }
    }
  };

  // One jump in place: rho_{k-1} -> rho_k with the pairs at rotation O (pair
  // j in slot (j + O) % P1); pair j of rho_k is written over pair j-1 of
  // rho_{k-1} (its last reader) and pair 0 into the free slot, so the new
  // rotation is O - 1 (mod P1) and no register is copied.  The values just
  // outside the lane's run come from the neighbour lanes (shuffles); at the
  // window's ends they are the lane's own values, which only halo states or
  // zero coefficients see.
  int k = 1;
  auto jump = [&](auto OC) {
    constexpr int O = decltype(OC)::value;
    const T lin = __shfl_up_sync(kFull, r[(QP - 1 + O) % P1].y, 1);
    const T rin = __shfl_down_sync(kFull, r[O % P1].x, 1);
    const T first_y = r[O % P1].y;
    const T2 left0 = v_make(lin, r[(QP - 1 + O) % P1].x);
#pragma unroll
    for (int j = 0; j < QP; ++j) {
      const T2 cur = r[(j + O) % P1];
      const T2 left = j == 0 ? left0 : r[(j - 1 + O) % P1];
      const T2 right = (j + 1 < QP) ? r[(j + 1 + O) % P1] : v_make(first_y, rin);
      const T2 al = j == 0 ? a2first : a2;
      T2 y;
      if constexpr (kComp) {
        y = comp_jump(cur, res[j], al, left, up[j], right, dg[j]);
      } else {
        y = v_fma(up[j], right, v_fma(al, left, v_mul(dg[j], cur)));
      }
      r[j == 0 ? (O + QP) % P1 : (j - 1 + O) % P1] = y;
    }
  };
  // Reset of the states beyond the box (pairs at home).
  auto scrub = [&]() {
    if (outmask) {
#pragma unroll
      for (int j = 0; j < QP; ++j) {
        if (outmask & (1u << (2 * j))) {
          r[j].x = (T)0;
          res[j].x = 0.0f;
        }
        if (outmask & (2u << (2 * j))) {
          r[j].y = (T)0;
          res[j].y = 0.0f;
        }
      }
    }
  };
  // Defect correction of the compensated chain after every p.renorm jumps,
  // i.e. at the end of every (p.renorm / P1)-th round (pairs at home; the
  // period is a multiple of the round length).  rleft counts the rounds left
  // (never reaching zero when the correction is off: K < 2^30).
  int rleft = (kComp && p.renorm > 0) ? p.renorm / P1 : 0x7fffffff;
  auto defect = [&]() {
    if constexpr (kComp) {
      if (--rleft == 0) {
        rleft = p.renorm / P1;
#pragma unroll
        for (int j = 0; j < QP; ++j) res[j] = __ffma2_rn(cb[j], r[j], res[j]);
      }
    }
  };
  auto jump_plain = [&](auto OC) {
    jump(OC);
    ++k;
  };
  // With weights and accumulation; the round may end early at Kmax.
  auto jump_acc = [&](auto OC) {
    constexpr int O = decltype(OC)::value;
    if (k > Kmax) return;
    if (wact) jump(OC);
    advance(k, lo, hi);
    if (wact) accumulate(k, lo, hi, std::integral_constant<int, (O + QP) % P1>{});
    ++k;
  };

  // ---- the jump chain -------------------------------------------------------
  // Warps run rounds of P1 jumps without meeting: a warp window's halo (one
  // lane's run, R >= P1 states) goes stale from its outer edge at one state
  // per jump; at a round's end the pairs are back home, the warps refresh
  // each other's halos (one CTA barrier) and, at most every h jumps, the CTAs
  // refresh theirs.
  int since = 0;  // jumps since the last cluster exchange
  int cep = 0, wrp = 0;
  auto round_end = [&](int k_e) {
    since += P1;
    if (C > 1 && since + P1 > h) {
      cep ^= 1;
      if (k_e < Kmax) cluster_exchange(cep);
      since = 0;
    }
    if (nwu > 1) {
      wrp ^= 1;
      warp_exchange(wrp);
    }
  };

  // Part 1: jumps before the earliest window start carry no bookkeeping.
  int minL = Kmax;
  for (int i = 0; i < nt; ++i) minL = min(minL, t_L[i]);
  const int ngroups = max(0, minL - 1) / P1;
  const int kE = ngroups * P1;  // last jump of part 1
  for (int g = 0; g < ngroups; ++g) {
    if (wact) RotSeq<P1, 0, P1>::run(jump_plain);
    else k += P1;
    defect();
    scrub();
    round_end(k - 1);
  }

  // Part 2: the same rounds with weights and accumulation.  Chunk c of the
  // weights (jumps [c kChunk1, (c+1) kChunk1)) is staged after the barrier
  // at jump (c-1) kChunk1 (no later round reads the slots it reuses) and
  // waited for before the barrier that precedes the round holding jump
  // c kChunk1; on entry (after jump kE) the chunks of kE and the next one.
  stage_chunk(kChunk1 * (kE / kChunk1));
  if (kChunk1 * (kE / kChunk1 + 1) <= Kmax) stage_chunk(kChunk1 * (kE / kChunk1 + 1));
  cp_async_wait<0>();
  rec_round(kE + 1, min(Kmax, kE + P1));
  __syncthreads();
  advance(kE, lo, hi);
  if (wact) accumulate(kE, lo, hi, std::integral_constant<int, 0>{});
  while (k <= Kmax) {
    RotSeq<P1, 0, P1>::run(jump_acc);
    const int k_e = k - 1;
    if (k_e >= Kmax) break;
    defect();
    scrub();
    if ((k_e + P1) % kChunk1 == 0) cp_async_wait<0>();
    rec_round(k_e + 1, min(Kmax, k_e + P1));
    round_end(k_e);
    if (nwu <= 1) __syncthreads();
    if (k_e % kChunk1 == 0 && k_e + kChunk1 <= Kmax) stage_chunk(k_e + kChunk1);
  }
  cp_async_wait<0>();
}

template <typename T, int QP, int kMaxT>
cudaError_t launch_reg1d_typed(const ChainParams& p, const Reg1dPlan& rp, cudaStream_t s) {
  static int smem_set = 0;
  static bool nonportable = false;
  auto kern = chain_reg1d_kernel<T, QP, kMaxT>;
  cudaError_t e;
  if ((int)rp.smem > smem_set) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rp.smem);
    if (e != cudaSuccess) return e;
    smem_set = (int)rp.smem;
  }
  if (rp.cluster > 8 && !nonportable) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    nonportable = true;
  }
  if (p.B <= 0) return cudaSuccess;  // attribute preparation only
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(p.B * rp.cluster));
  cfg.blockDim = dim3((unsigned)rp.threads);
  cfg.dynamicSmemBytes = rp.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)rp.cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, p, rp.halo);
}

// State pairs per lane (QP, QP + 1 = 8 jumps per round) and the largest CTA
// of each precision: the registers hold per pair of states the values, the
// exit and death coefficients and, in FP32, the residuals and defects (70
// registers at FP32, 84 at FP64); 384 threads leave 170 registers per thread
// (FP32), 256 threads 255 (FP64, whose slow FP64 pipe needs few warps but many
// independent operations).
constexpr int kQP32 = 7, kMaxT32 = 384;
constexpr int kQP64 = 7, kMaxT64 = 256;
// One pair per thread spreads a small chain over more warps: the latency of a
// single solve drops (GB300's FP64 pipe issues a warp's FP64 instruction over
// many cycles, so a chain held by one warp is limited by one sub-partition).
constexpr int kQPSmall = 1, kMaxTSmall = 512;

}  // namespace

bool chain_reg1d_plan(int precision, int64_t Nmax, int ntimes, int cluster, int halo, Reg1dPlan* out,
                      bool small) {
  if (Nmax < 1 || ntimes < 1 || cluster < 1 || cluster > 16) return false;
  const bool f64 = precision == MJP_FP64;
  int qp = f64 ? kQP64 : kQP32, maxt = f64 ? kMaxT64 : kMaxT32;
  const int64_t S = (Nmax + cluster - 1) / cluster;
  if (S + 2 * (int64_t)halo + 64 > (int64_t)1 << 24) return false;
  if (small && 32 * reg1d_warps((int)(S + (cluster > 1 ? 2 * std::max(halo, kQPSmall + 1) : 0)), kQPSmall) <= kMaxTSmall) {
    qp = kQPSmall;
    maxt = kMaxTSmall;
  }
  // The halo covers at least one round (qp + 1 jumps) and the last CTA owns
  // at least that many states.
  const int h = cluster > 1 ? std::max(halo, qp + 1) : 0;
  if (cluster > 1 && Nmax - (int64_t)(cluster - 1) * S < qp + 1) return false;
  const int64_t ext = S + 2 * (int64_t)h;
  const int threads = 32 * reg1d_warps((int)ext, qp);
  if (threads > maxt) return false;
  const Reg1dLayout L = reg1d_layout(f64 ? 8 : 4, threads, qp, h, ntimes);
  if (L.total + 1024 > (size_t)227 * 1024) return false;
  out->cluster = cluster;
  out->threads = threads;
  out->qp = qp;
  out->halo = h;
  out->smem = L.total;
  return true;
}

int64_t chain_reg1d_max_states(int precision) {
  const int qp = precision == MJP_FP64 ? kQP64 : kQP32, maxt = precision == MJP_FP64 ? kMaxT64 : kMaxT32;
  return (int64_t)(maxt / 32) * (60 * qp);  // warp windows overlap by two lanes' runs
}

cudaError_t launch_chain_reg1d(int precision, const ChainParams& p, const Reg1dPlan& rp, cudaStream_t s) {
  if (rp.qp == kQPSmall)
    return precision == MJP_FP64 ? launch_reg1d_typed<double, kQPSmall, kMaxTSmall>(p, rp, s)
                                 : launch_reg1d_typed<float, kQPSmall, kMaxTSmall>(p, rp, s);
  if (precision == MJP_FP64) return launch_reg1d_typed<double, kQP64, kMaxT64>(p, rp, s);
  return launch_reg1d_typed<float, kQP32, kMaxT32>(p, rp, s);
}

}  // namespace mjp
