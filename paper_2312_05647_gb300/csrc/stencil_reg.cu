// stencil_reg.cu -- register-resident jump chain for the mRNA/protein stencil
// (FP32, log-likelihood mode), Algorithm 2 with one chain shared by all times.
//
// Each thread keeps a 4-column x 8- or 10-row block of rho (32 or 40 states,
// as row pairs) in registers for all K jumps; shared memory carries only the
// block edges (its left and right columns, first and last rows),
// double-buffered by jump parity, and the observation accumulators.  Per jump
// a thread reads its four neighbours' edges, updates its states in place (row
// pair by row pair, keeping the old values the next ones still need), writes
// its own edges and meets the rest of its CTA at one barrier; the rows that
// cross to a neighbouring CTA of the cluster go there by st.async, counted on
// that CTA's hand-over mbarriers (no cluster barrier per jump).  Work that
// only some threads have (the observations of rho_k, read from a per-thread
// local array by slot) follows the barrier, so it overlaps the others' next
// jump instead of holding every warp at it.
// Compared with a shared-memory ping-pong of the whole slab (every state read
// three times and written once per jump), shared-memory traffic drops from
// 16 B to ~1.5 B per state and the FP32 pipe becomes the limit.
//
// Arithmetic per state is the same operation sequence, in the same order, as
// the shared-memory kernel in stencil.cu (the compensated jump of
// chain_common.cuh: delta form of rho B with the coefficients built from
// theta, each state's rounding residual carried into the next jump, the exit
// defects added back every p.renorm jumps), so both kernels produce
// bit-identical chains; observations with one member per group give
// bit-identical log-likelihoods.  A cluster of C CTAs splits the rows; block
// edges that cross a CTA boundary are written into the neighbour CTA's halo
// slots through distributed shared memory.
//
// The residuals and the row coefficients live in tensor memory (TMEM, 256 KB
// per SM, otherwise idle in this kernel): the registers of a 512-thread CTA
// hold the 40 values of a block and the column coefficients, not 40 residuals
// as well, and the coefficients that depend on the row (the exit of each
// column pair and the inflow from the row above), formed once in the
// prologue exactly as the update formed them every jump before, are loaded
// instead of recomputed.  Each warp owns its 32 TMEM lanes (the quadrant
// warp % 4 may address) and 12 columns per row of its blocks (two of them
// spare; in rows 0 and 1 they hold the column defects of the exit-defect
// correction, so no FP64 arithmetic runs in the jump loop); a row's residuals
// and coefficients are read with two tcgen05.ld (issued while the previous
// row is computed) and its residuals written back with one tcgen05.st.  The CTA holds one allocation from start to end, sized so that
// all CTAs the register file admits on one SM fit its TMEM (no allocation
// ever waits).
//
// Every neighbour read and edge write uses a per-thread base plus a
// compile-time offset (the edge arrays have fixed strides), and the jump
// counter is 32-bit, so the jump loop carries almost no integer work besides
// the arithmetic of the states.
#include <cooperative_groups.h>

#include <algorithm>
#include <type_traits>

#include "chain_common.cuh"
#include "internal.cuh"

namespace cg = cooperative_groups;

namespace mjp {

namespace {

constexpr int kQC = 4;            // columns per thread block of states
// Threads per CTA at most, T = 512 (one CTA per SM) or 256 (two CTAs of
// different instances per SM, so that one computes while the other waits at
// its barrier); <= 128 registers per thread either way, so the register file
// itself admits one (T = 512) or two (T = 256) CTAs per SM.
constexpr int kMaxNQ = 512;       // column quads (M <= 2048)
// TMEM columns per CTA: T / 128 warps share each lane quadrant, kRowCols
// columns per row of their blocks (<= 10 rows): 480 -> 512 columns at T = 512,
// 240 -> 256 at T = 256, so the CTAs an SM can hold never exceed its 512
// columns and an allocation never waits.
template <int T>
constexpr unsigned tmem_cols() {
  return T == 512 ? 512u : 256u;
}
// Tensor-memory columns per block row: 4 residuals, the exit coefficients of
// the two column pairs, the inflow coefficient from above (twice) and 2 spare.
constexpr unsigned kRowCols = 12;
// Fixed strides of the edge arrays (per parity):
//  - columns [2 sides][QR][T + 1] float2: the left (side 0) and right (side 1)
//    column of block t, row pair r; entry T (kZero) is a zero slot;
//  - rows [2][2 T + 1] float4: the first (0) and last (1) row of block t (its
//    4 columns); entries kZero + 1 + q hold the row just outside the CTA for
//    column quad q (the next CTA's first row in array 0, the previous CTA's
//    last row in array 1), written by those CTAs; entry kZero is zero.
// Every neighbour read goes through a fixed per-thread slot, so threads at
// the box edge read a zero slot instead of branching.
// Poisson weights are staged per time in a ring of kStage jumps, filled
// kChunk jumps at a time, one chunk ahead, by every thread of the CTA.
constexpr int kChunk = 32;
constexpr int kStage = 2 * kChunk;

template <int QR, int T>
struct EdgeGeo {
  static constexpr int kZero = T;
  static constexpr int kCStr = T + 1;
  static constexpr int kRStr = 2 * T + 1;  // column quads <= blocks <= T
  static constexpr size_t col_bytes = ((size_t)8 * 2 * QR * kCStr + 15) / 16 * 16;
  static constexpr size_t par_bytes = col_bytes + (size_t)16 * 2 * kRStr;
  static constexpr size_t col(int side, int r) { return (size_t)8 * (side * QR + r) * kCStr; }
  static constexpr size_t row(int which) { return col_bytes + (size_t)16 * which * kRStr; }
};

struct RegLayout {
  size_t edge, tx, tPL, ttail, twb, pw, tL, tK, trec, ring, gptr, ent, acc_s, acc_c, total;
};

__host__ __device__ inline RegLayout reg_layout(size_t edge_bytes, int nt, int nmem) {
  RegLayout s;
  size_t o = 0;
  s.edge = o; o += edge_bytes;
  s.tx = o; o += 8 * (size_t)nt;
  s.tPL = o; o += 8 * (size_t)nt;
  s.ttail = o; o += 8 * (size_t)nt;
  s.twb = o; o += 8 * (size_t)nt;
  s.pw = o; o += 16 * (size_t)nt;
  s.tL = o; o += align_up(4 * (size_t)nt, 8);
  s.tK = o; o += align_up(4 * (size_t)nt, 8);
  s.trec = o; o += align_up(4 * (size_t)nt, 8);
  s.ring = o; o += align_up(4 * kStage * (size_t)nt, 16);
  s.gptr = o; o += align_up(4 * (size_t)(nt + 1), 8);
  s.ent = o; o += 8 * (size_t)nmem;
  s.acc_s = o; o += align_up(4 * (size_t)nmem, 8);
  s.acc_c = o; o += align_up(4 * (size_t)nmem, 16);
  s.total = align_up(o, 16);
  return s;
}

// Register slot of row r of a block at rotation ROT: 0 = home (row r in slot
// r), 1 = shifted (row r in slot r - 1, row 0 in the spare slot NR).
template <int NR>
__host__ __device__ constexpr int rslot(int r, int rot) {
  return rot == 0 ? r : (r == 0 ? NR : r - 1);
}

// The value of v, hidden from the optimiser: quantities derived from it inside
// the jump loop are recomputed each jump instead of being hoisted out of the
// loop and held in registers for all states.
__device__ __forceinline__ int opaque(int v) {
  asm volatile("" : "+r"(v));
  return v;
}

// Tensor-memory access (tcgen05, sm_100 family): allocation by one warp,
// 32-lane x 4-column loads and stores of 32-bit values, and the waits that
// order them.  Addresses are (lane << 16) | column.
__device__ __forceinline__ void tmem_alloc(unsigned* slot, unsigned ncols) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(slot);
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(a), "r"(ncols) : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// Four residuals of one row: (c0, c2) and (c1, c3), the layout of the state pairs.
__device__ __forceinline__ void tmem_ld4(unsigned taddr, float2& a, float2& b) {
  unsigned r0, r1, r2, r3;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3) : "r"(taddr) : "memory");
  // The loaded registers are defined only after the wait: tie them to it.
  asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r0), "+r"(r1), "+r"(r2), "+r"(r3) :: "memory");
  a = make_float2(__uint_as_float(r0), __uint_as_float(r1));
  b = make_float2(__uint_as_float(r2), __uint_as_float(r3));
}
// Registers of a 4-column load in flight.
struct Tmem4 {
  unsigned r0, r1, r2, r3;
};
// Row r's residuals, exit coefficients and inflow-from-above coefficient
// (an 8-column and a 2-column load, waited for together).
struct Tmem2 {
  unsigned r0, r1;
};
struct Tmem12 {
  Tmem4 r, d;
  Tmem2 c;
};
__device__ __forceinline__ void tmem_ld12_issue(unsigned taddr, Tmem12& v) {
  // Columns 0-7 (residuals, exit coefficients) in one load, 8-9 in another.
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(v.r.r0), "=r"(v.r.r1), "=r"(v.r.r2), "=r"(v.r.r3), "=r"(v.d.r0), "=r"(v.d.r1), "=r"(v.d.r2),
                 "=r"(v.d.r3)
               : "r"(taddr)
               : "memory");
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];"
               : "=r"(v.c.r0), "=r"(v.c.r1) : "r"(taddr + 8u) : "memory");
}
__device__ __forceinline__ void tmem_ld12_wait(Tmem12& v, float2& rA, float2& rB, float2& dA, float2& dB,
                                               float2& cup) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(v.r.r0), "+r"(v.r.r1), "+r"(v.r.r2), "+r"(v.r.r3), "+r"(v.d.r0), "+r"(v.d.r1),
                 "+r"(v.d.r2), "+r"(v.d.r3), "+r"(v.c.r0), "+r"(v.c.r1)::"memory");
  rA = make_float2(__uint_as_float(v.r.r0), __uint_as_float(v.r.r1));
  rB = make_float2(__uint_as_float(v.r.r2), __uint_as_float(v.r.r3));
  dA = make_float2(__uint_as_float(v.d.r0), __uint_as_float(v.d.r1));
  dB = make_float2(__uint_as_float(v.d.r2), __uint_as_float(v.d.r3));
  cup = make_float2(__uint_as_float(v.c.r0), __uint_as_float(v.c.r1));
}
__device__ __forceinline__ void tmem_st4(unsigned taddr, float2 a, float2 b) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr),
               "r"(__float_as_uint(a.x)), "r"(__float_as_uint(a.y)), "r"(__float_as_uint(b.x)),
               "r"(__float_as_uint(b.y))
               : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Hand-over of the block rows that cross a CTA boundary.  A sending thread
// writes its 16 bytes into the neighbour CTA's row array with st.async, which
// counts them on that CTA's hand-over mbarrier (one per direction and jump
// parity); the receiving threads wait for the phase of the jump they need,
// and the first of them re-arms the barrier with the bytes it expects two
// jumps later.  Addresses are 32-bit shared-memory addresses (mapa gives the
// neighbour's copy of a variable).
__device__ __forceinline__ unsigned cluster_addr(unsigned local, int rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
__device__ __forceinline__ void hbar_init(unsigned a) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
}
__device__ __forceinline__ void hbar_arm(unsigned a, unsigned bytes) {
  asm volatile("{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(a), "r"(bytes)
               : "memory");
}
// At most `polls` tests of the phase of parity ph (none when polls is 0):
// false when the phase has not completed by then.  The test acquires at
// cluster scope: the bytes it orders were written by another CTA.
__device__ __forceinline__ bool hbar_wait(unsigned a, unsigned ph, long long polls) {
  for (long long i = 0; i < polls; ++i) {
    unsigned ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok) : "r"(a), "r"(ph) : "memory");
    if (ok) return true;
    if (i >= 16) __nanosleep(32);
  }
  return false;
}
__device__ __forceinline__ void st_async16(unsigned raddr, float2 a, float2 b, unsigned rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(
                   raddr),
               "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "r"(rbar)
               : "memory");
}
// Plain store into a neighbour CTA (ordered by a later cluster barrier).
__device__ __forceinline__ void st_cluster16(unsigned raddr, float2 a, float2 b) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(raddr), "f"(a.x), "f"(a.y), "f"(b.x),
               "f"(b.y)
               : "memory");
}

// Exclusive prefix sum of v over the block (blockDim <= 1024).
__device__ int block_exclusive_scan(int v, int* wsum) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  int off = 0;
  for (int w = 0; w < warp; ++w) off += wsum[w];
  __syncthreads();
  return off + x - v;
}

template <int kQR, int kT>
__global__ void __launch_bounds__(kT, 512 / kT) chain_reg2d_kernel(const ChainParams p, const int NQ, const int RS) {
  using G = EdgeGeo<kQR, kT>;
  constexpr int kZero = G::kZero;
  constexpr int kRows = 2 * kQR;  // rows of a thread's block
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int wsum[32];
  __shared__ unsigned tmem_base;
  // Hand-over barriers [direction][jump parity]: 0 counts the row from the
  // CTA below (rank - 1), 1 the row from the CTA above (rank + 1).
  __shared__ __align__(8) unsigned long long hbar[2][2];
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int job = p.job_map ? p.job_map[blockIdx.x / C] : (int)(blockIdx.x / C);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int nt = p.ntimes;
  const int M = p.M, P = p.P;
  const int p0 = rank * RS;
  const int p1 = min(P, p0 + RS);
  const int nrb = p1 > p0 ? (p1 - p0 + kRows - 1) / kRows : 0;  // row blocks of this CTA
  const bool wwarp = warp == 0;  // runs the weight recurrence of windows without a stored copy
  const int qx = tid % NQ, rb = tid / NQ;
  const bool owner = rb < nrb;   // this thread holds a block of states
  const int m0 = kQC * qx, pb = p0 + kRows * rb;  // first column and first row of the block
  const int nmem = (int)p.mptr[p.G];

  const RegLayout L = reg_layout(2 * G::par_bytes, nt, nmem);
  double* t_x = reinterpret_cast<double*>(smem + L.tx);
  double* t_PL = reinterpret_cast<double*>(smem + L.tPL);
  double* t_tail = reinterpret_cast<double*>(smem + L.ttail);
  int* t_L = reinterpret_cast<int*>(smem + L.tL);
  int* t_K = reinterpret_cast<int*>(smem + L.tK);
  int* t_rec = reinterpret_cast<int*>(smem + L.trec);  // 1: no stored copy, run the recurrence
  const float** t_wb = reinterpret_cast<const float**>(smem + L.twb);
  double* pw = reinterpret_cast<double*>(smem + L.pw);
  float* ring = reinterpret_cast<float*>(smem + L.ring);
  int* s_gptr = reinterpret_cast<int*>(smem + L.gptr);
  int2* ent = reinterpret_cast<int2*>(smem + L.ent);
  float* acc_s = reinterpret_cast<float*>(smem + L.acc_s);
  float* acc_c = reinterpret_cast<float*>(smem + L.acc_c);
  const float* arena = reinterpret_cast<const float*>(p.arena);

  // ---- prologue: windows, weights, observations ---------------------------
  const int64_t Kmax64 = p.info[job].Kmax;
  const Win* wj = p.win + (int64_t)job * nt;
  for (int i = tid; i < nt; i += blockDim.x) {
    const Win w = wj[i];
    t_x[i] = w.x;
    t_PL[i] = w.PL;
    t_tail[i] = w.tail;
    t_L[i] = (int)w.L;
    t_K[i] = (int)w.K;
    t_rec[i] = (w.woff < 0 || !arena) ? 1 : 0;
    t_wb[i] = (w.woff >= 0 && arena) ? arena + (w.woff - w.L) : nullptr;
    pw[i] = (w.L == 0) ? w.PL : 0.0;
    if (w.L == 0 && (w.woff < 0 || !arena))  // jump 0 of a window without a stored copy
      ring[i * kStage] = (float)(w.PL + (w.K == 0 ? w.tail : 0.0));
  }
  for (int i = tid; i <= nt; i += blockDim.x) s_gptr[i] = (int)p.gptr[i];
  const double omega = p.info[job].omega;
  const Coef<float> co = make_coef<float, MJP_MRNA_PROT2D>(p.theta + (int64_t)job * p.ntheta, omega);
  // The planner caps K (MJP_OPT_K_CAP, default 2^26); the loop counts in 32 bits.
  const int Kmax = Kmax64 < (1LL << 30) ? (int)Kmax64 : 0;
  if (Kmax64 >= (1LL << 30) && tid == 0 && rank == 0) set_status(p.status, kStatusKcap);
  if (warp == 0) tmem_alloc(&tmem_base, tmem_cols<kT>());
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  // This thread's residuals: lane 32 (warp % 4) + lane, columns
  // (warp / 4) 4 NR + 4 r .. + 3 for row r of its block.
  const unsigned tres = tmem_base + ((32u * (unsigned)(warp & 3)) << 16) + (unsigned)(warp >> 2) * kRowCols * 2u * kQR;

  // Observation entries: (member q, register slot, time) of the states this
  // thread holds, in member order (= time order).  Two passes: count, then
  // fill after a block-wide prefix sum.
  auto owns = [&](int s, int& slot) -> bool {
    const int ps = s / M, ms = s - ps * M;
    if (!owner || ps < pb || ps >= pb + kRows || ms < m0 || ms >= m0 + kQC) return false;
    slot = (ps - pb) * kQC + (ms - m0);
    return true;
  };
  auto scan_members = [&](bool fill, int base) -> int {
    int n = 0, i = 0;
    for (int g = 0; g < p.G; ++g) {
      while (i < nt && g >= s_gptr[i + 1]) ++i;
      const int q0 = (int)p.mptr[g], q1 = (int)p.mptr[g + 1];
      for (int q = q0; q < q1; ++q) {
        int slot;
        if (owns(p.members[q], slot)) {
          if (fill) ent[base + n] = make_int2(q, slot | (i << 6));
          ++n;
        }
      }
    }
    return n;
  };
  const int ecount = owner ? scan_members(false, 0) : 0;
  const int ebeg = block_exclusive_scan(ecount, wsum);
  if (owner) scan_members(true, ebeg);
  const int eend = ebeg + ecount;
  for (int q = tid; q < nmem; q += blockDim.x) {
    acc_s[q] = 0.0f;
    acc_c[q] = 0.0f;
  }
  {
    float4* e = reinterpret_cast<float4*>(smem + L.edge);
    for (int q = tid; q < (int)(2 * G::par_bytes / 16); q += blockDim.x) e[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  // The hand-over barriers of this CTA, armed for their first phase (jump 1
  // for parity 1, jump 2 for parity 0; the rows of rho_0 cross by plain
  // stores and a cluster barrier).  Every CTA holds at least one row block,
  // so the neighbour's boundary row block sends one 16-byte row per column
  // quad, NQ in all, every jump.
  const unsigned hb = (unsigned)__cvta_generic_to_shared(&hbar[0][0]);
  const unsigned hbytes = 16u * (unsigned)NQ;
  if (C > 1 && tid == 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) hbar_init(hb + 8u * i);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (rank > 0) {
      hbar_arm(hb, hbytes);
      hbar_arm(hb + 8u, hbytes);
    }
    if (rank + 1 < C) {
      hbar_arm(hb + 16u, hbytes);
      hbar_arm(hb + 24u, hbytes);
    }
  }
  // Every CTA's edge arrays are zeroed and its barriers set up before any
  // neighbour writes into them.
  if (C > 1) cluster.sync();
  else __syncthreads();

  // Column coefficients (rates into column m, scaled by 1/Omega): gamma_m
  // (m+1) from m+1, k_p m from p-1, and the negated exit -e0 without the
  // gamma_p p part, as pairs of the columns (c0, c2) and (c1, c3) that share a
  // register pair.  Threads without a block run the same instructions (the
  // tensor-memory accesses are warp-wide) with every coefficient zero, so
  // their values stay zero.
  // The column defects eps (formed in FP64, the only FP64 arithmetic of the
  // defect correction) are kept in tensor memory for it.
  float crc[kQC], cdc[kQC], d0c[kQC], epc[kQC];
  int colmask = 0;  // bit c: column m0 + c lies in the box
  const float own = owner ? 1.0f : 0.0f;
#pragma unroll
  for (int c = 0; c < kQC; ++c) {
    const int m = m0 + c;
    if (m < M) colmask |= 1 << c;
    const float fm = (float)m;
    crc[c] = owner ? f_mul(co.b, (float)(m + 1)) : 0.0f;
    cdc[c] = owner ? f_mul(co.c, fm) : 0.0f;
    const MrnaCol mc = mrna_col(co, m, M);
    d0c[c] = owner ? -mc.e0 : 0.0f;
    epc[c] = owner ? mc.eps : 0.0f;
  }
  const float2 d0A = v_make(d0c[0], d0c[2]), d0B = v_make(d0c[1], d0c[3]);
  const float2 crA = v_make(crc[0], crc[2]), crB = v_make(crc[1], crc[3]);
  const float2 cdA = v_make(cdc[0], cdc[2]), cdB = v_make(cdc[1], cdc[3]);
  const float c_l = own * co.a, c_d = own * co.d;
  const float2 c_l2 = v_make(c_l, c_l), c_gp = v_make(c_d, c_d), c_ngp = v_make(-c_d, -c_d);
  const bool padcols = colmask != (1 << kQC) - 1;
  // Row of this block that holds row P-1 (-1 if none).
  const int rtop = (P - 1 >= pb && P - 1 < pb + kRows) ? P - 1 - pb : -1;

  // Fixed neighbour slots: left block's right column, right block's left
  // column, the row below (a last row) and the row above (a first row).
  const int iL = qx > 0 ? tid - 1 : kZero;
  const int iR = qx + 1 < NQ ? tid + 1 : kZero;
  const int iB = rb > 0 ? tid - NQ : (rank > 0 ? kZero + 1 + qx : kZero);
  const int iA = rb + 1 < nrb ? tid + NQ : (rank + 1 < C ? kZero + 1 + qx : kZero);
  const unsigned oL = 8u * iL, oR = 8u * iR, oB = 16u * iB, oA = 16u * iA, oT8 = 8u * tid, oT16 = 16u * tid;
  unsigned char* const E0 = smem + L.edge;

  // rho0 into registers, its edges into parity 0.  Row r of the block is
  // S[r][0] = (c0, c2), S[r][1] = (c1, c3); S[kRows] is a spare row: a jump
  // writes row r's new values over row r-1's old ones (ascending) or row r+1's
  // (descending), so the rows shift by one slot and back every two jumps and
  // no register is copied.
  constexpr int NR = kRows;
  float2 S[NR + 1][2];
  const float* rho0 = reinterpret_cast<const float*>(p.rho0);
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    float v[kQC];
#pragma unroll
    for (int c = 0; c < kQC; ++c) {
      const int m = m0 + c, pa = pb + r;
      v[c] = (owner && m < M && pa < p1) ? rho0[(int64_t)pa * M + m] : 0.0f;
    }
    S[r][0] = v_make(v[0], v[2]);
    S[r][1] = v_make(v[1], v[3]);
  }
  S[NR][0] = S[NR][1] = v_make(0.0f, 0.0f);
  // Residuals start at zero.  (Tensor-memory instructions are warp-wide: the
  // warp is converged before each group of them that follows lane-dependent
  // code.)
  __syncwarp();
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    // Row r's coefficients, as the update formed them every jump before.
    const float fr = (float)(pb + r);
    const float2 fp2 = v_make(fr, fr);
    tmem_st4(tres + kRowCols * r, v_make(0.0f, 0.0f), v_make(0.0f, 0.0f));
    tmem_st4(tres + kRowCols * r + 4u, v_fma(c_ngp, fp2, d0A), v_fma(c_ngp, fp2, d0B));  // -e_{m,p}
    const float2 cu = v_fma(c_gp, fp2, c_gp);  // gamma_p (p+1) from p+1
    // Spare columns: the column defects of (c0, c2) in row 0, of (c1, c3) in row 1.
    const float2 sp = r == 0 ? v_make(epc[0], epc[2]) : r == 1 ? v_make(epc[1], epc[3]) : v_make(0.0f, 0.0f);
    tmem_st4(tres + kRowCols * r + 8u, cu, sp);
  }
  // The row arrays of the neighbouring CTAs: our first row is the row above
  // CTA rank-1 (its array 0, counted by its barrier from above), our last row
  // the row below CTA rank+1 (array 1, its barrier from below).  The threads
  // that send a row are the ones that receive the neighbour's.
  const bool rx_dn = C > 1 && rank > 0 && rb == 0;
  const bool rx_up = C > 1 && rank + 1 < C && rb == nrb - 1;
  unsigned nb_dn = 0, nb_up = 0, nbar_dn = 0, nbar_up = 0;
  {
    const unsigned e0 = (unsigned)__cvta_generic_to_shared(E0);
    if (rx_dn) {
      nb_dn = cluster_addr(e0 + (unsigned)G::row(0) + 16u * (kZero + 1 + qx), rank - 1);
      nbar_dn = cluster_addr(hb + 16u, rank - 1);
    }
    if (rx_up) {
      nb_up = cluster_addr(e0 + (unsigned)G::row(1) + 16u * (kZero + 1 + qx), rank + 1);
      nbar_up = cluster_addr(hb, rank + 1);
    }
  }
  // False once one of this thread's hand-over waits has run out: from then on
  // it neither waits, re-arms nor sends rows to the neighbouring CTAs (so no
  // barrier sees an arrival or bytes outside the phase it is armed for), and
  // the chain runs on to its end with the status set.
  bool hok = true;
  // Edges of the block: the left (c0) and right (c3) columns per row pair,
  // the first and last rows as (c0, c2, c1, c3).  The rows for the
  // neighbouring CTAs go by st.async (counted on their hand-over barrier of
  // this parity), those of rho_0 (INIT) by plain stores.
  auto publish = [&](int par, auto ROTC, auto INITC) {
    constexpr int ROT = decltype(ROTC)::value;
    constexpr bool INIT = decltype(INITC)::value;
    unsigned char* Ep = E0 + (par ? G::par_bytes : 0);
#pragma unroll
    for (int r = 0; r < kQR; ++r) {
      const int s0 = rslot<NR>(2 * r, ROT), s1 = rslot<NR>(2 * r + 1, ROT);
      // One 8-byte store per column and row pair (the slots are 8-byte aligned).
      *reinterpret_cast<float2*>(Ep + G::col(0, r) + oT8) = make_float2(S[s0][0].x, S[s1][0].x);
      *reinterpret_cast<float2*>(Ep + G::col(1, r) + oT8) = make_float2(S[s0][1].y, S[s1][1].y);
    }
    const int sf = rslot<NR>(0, ROT), sl = rslot<NR>(NR - 1, ROT);
    float2* fr = reinterpret_cast<float2*>(Ep + G::row(0) + oT16);
    float2* lr = reinterpret_cast<float2*>(Ep + G::row(1) + oT16);
    fr[0] = S[sf][0];
    fr[1] = S[sf][1];
    lr[0] = S[sl][0];
    lr[1] = S[sl][1];
    const unsigned po = par ? (unsigned)G::par_bytes : 0u;
    if (rx_dn) {
      if (INIT) st_cluster16(nb_dn + po, S[sf][0], S[sf][1]);
      else if (hok) st_async16(nb_dn + po, S[sf][0], S[sf][1], nbar_dn + 8u * (unsigned)par);
    }
    if (rx_up) {
      if (INIT) st_cluster16(nb_up + po, S[sl][0], S[sl][1]);
      else if (hok) st_async16(nb_up + po, S[sl][0], S[sl][1], nbar_up + 8u * (unsigned)par);
    }
    // Only some lanes send: the warp is converged again before its next
    // warp-wide tensor-memory instruction (the defect correction).
    __syncwarp();
  };
  publish(0, std::integral_constant<int, 0>{}, std::true_type{});
  if (C > 1) cluster.sync();
  else __syncthreads();

  bool mine_rec = false;
  for (int i = tid; i < nt; i += blockDim.x) mine_rec |= t_rec[i] != 0;
  const bool any_rec = __syncthreads_or(mine_rec) != 0;

  int lo = 0, hi = -1;
  auto advance = [&](int k, int& l, int& h) {
    while (l < nt && t_K[l] < k) ++l;
    while (h + 1 < nt && t_L[h + 1] <= k) ++h;
  };
  advance(0, lo, hi);
  // First jump at which the active range [lo, hi] changes (a window ends or
  // the next one starts); the per-jump check is one comparison.
  auto next_change = [&](int l, int h) -> int {
    int kn = 0x7fffffff;
    if (l < nt) kn = min(kn, t_K[l] + 1);
    if (h + 1 < nt) kn = min(kn, t_L[h + 1]);
    return kn;
  };
  int knext = next_change(lo, hi);
  // Stage the stored weights of jumps [k0, k0 + kChunk) of every window into
  // the ring (slot j % kStage), spread over all threads.
  auto stage_chunk = [&](int k0) {
    const int k1 = min(k0 + kChunk, Kmax + 1);
    for (int e = tid; e < nt * kChunk; e += blockDim.x) {
      const int i = e / kChunk, j = k0 + (e - i * kChunk);
      if (j < k1 && t_wb[i] && j >= t_L[i] && j <= t_K[i])
        cp_async_elem(ring + i * kStage + (j & (kStage - 1)), t_wb[i] + j);
    }
    cp_async_commit();
  };
  stage_chunk(0);
  stage_chunk(kChunk);
  cp_async_wait<1>();  // chunk 0 has landed

  // Observations of rho_k for the active times [l, h] of jump k (Kahan, FP32).
  int ecur = ebeg;
  auto accumulate = [&](int k, int l, int h, auto ROTC) {
    constexpr int ROT = decltype(ROTC)::value;
    if (!owner || l > h) return;
    const int sk = k & (kStage - 1);
    while (ecur < eend && (ent[ecur].y >> 6) < l) ++ecur;
    if (ecur >= eend || (ent[ecur].y >> 6) > h) return;
    // Some of this thread's states are observed at this jump: its values go
    // to a per-thread local array once (slot 4 r + c: row r, column c), and
    // each observed one is read back by its slot.
    float loc[NR * kQC];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const float2 a = S[rslot<NR>(r, ROT)][0], b = S[rslot<NR>(r, ROT)][1];
      loc[kQC * r + 0] = a.x;
      loc[kQC * r + 1] = b.x;
      loc[kQC * r + 2] = a.y;
      loc[kQC * r + 3] = b.y;
    }
    for (int e = ecur; e < eend; ++e) {
      const int2 en = ent[e];
      const int ti = en.y >> 6;
      if (ti > h) break;
      const float v = loc[en.y & 63];
      const float w = ring[ti * kStage + sk];
      const float y = __fsub_rn(__fmul_rn(w, v), acc_c[en.x]);
      const float s0 = acc_s[en.x];
      const float t = __fadd_rn(s0, y);
      acc_c[en.x] = __fsub_rn(__fsub_rn(t, s0), y);
      acc_s[en.x] = t;
    }
  };
  // Weights of jump kn for windows without a stored copy (Algorithm 2's
  // recurrence P_kn = P_{kn-1} x / kn from P_L, tail added at K), one jump
  // ahead of their use; warp 0.
  int rlo = lo, rhi = hi;
  auto rec_step = [&](int kn) {
    advance(kn, rlo, rhi);
    const double* rprev = pw + ((kn - 1) & 1) * nt;
    double* rcur = pw + (kn & 1) * nt;
    for (int i = rlo + lane; i <= rhi; i += 32) {
      if (!t_rec[i]) continue;
      const double Pk = (kn == t_L[i]) ? t_PL[i] : __dmul_rn(rprev[i], __ddiv_rn(t_x[i], (double)kn));
      rcur[i] = Pk;
      ring[i * kStage + (kn & (kStage - 1))] = (float)(Pk + (kn == t_K[i] ? t_tail[i] : 0.0));
    }
  };
  if (wwarp && any_rec && Kmax >= 1) rec_step(1);
  __syncthreads();
  accumulate(0, lo, hi, std::integral_constant<int, 0>{});  // rho_0 with the weights of jump 0

  // One jump of the block: rho_{k-1} at rotation DIR (0: home, rows
  // ascending; 1: shifted, rows descending) -> rho_k at rotation 1 - DIR.
  // Per state, in the shared-memory kernel's order: (1 - e) rho + k_m rho(m-1)
  // + gamma_m (m+1) rho(m+1) + k_p m rho(p-1) + gamma_p (p+1) rho(p+1); the row
  // holding P-1 adds k_p m back to 1 - e (no protein birth out of it), rows
  // beyond it and padding columns stay zero.
  // Row P-1 (no protein birth out of it: 1 - e gains k_p m back) is handled
  // without branches when it is a block's last row: every thread adds topA /
  // topB to the diagonal of its last row, k_p m (both columns of the pair) in
  // the block holding P-1 and zero elsewhere (adding +0 changes no value); the
  // row above it is the zero slot.  Warps with a thread whose block holds P-1
  // elsewhere, rows beyond the box or padding columns run the EDGE update with
  // explicit checks (warp-uniform, so no warp runs both).
  const bool edge_t = padcols || (rtop >= 0 && rtop != NR - 1);
  const bool edge_w = __any_sync(kFull, edge_t);
  const float2 topA = rtop == NR - 1 ? cdA : v_make(0.0f, 0.0f);
  const float2 topB = rtop == NR - 1 ? cdB : v_make(0.0f, 0.0f);
  auto update = [&](int par, auto DIRC, auto EDGEC) {
    constexpr int DIR = decltype(DIRC)::value;
    constexpr bool EDGE = decltype(EDGEC)::value;
    const unsigned char* Ep = E0 + (par ? G::par_bytes : 0);
    const int rtk = EDGE ? opaque(rtop) : -1;
    tmem_wait_st();  // the last jump's residual stores are complete
    // The residuals of the next row in this jump's order are loaded while the
    // current row is computed.
    Tmem12 pre;
    tmem_ld12_issue(tres + kRowCols * (DIR == 0 ? 0 : NR - 1), pre);
#pragma unroll
    for (int i = 0; i < NR; ++i) {
      const int r = DIR == 0 ? i : NR - 1 - i;
      const int so = rslot<NR>(r, DIR);                                  // old row r
      const int sn = DIR == 0 ? (r == 0 ? NR : r - 1) : r;               // its new value
      // The left block's c3 and the right block's c0 of this row pair, read at
      // its first row in this jump's order.
      float2 lp, rp;
      if ((i & 1) == 0) {
        lp = *reinterpret_cast<const float2*>(Ep + G::col(1, r >> 1) + oL);
        rp = *reinterpret_cast<const float2*>(Ep + G::col(0, r >> 1) + oR);
      }
      const float2 A = S[so][0], B = S[so][1];
      float2 bA, bB, aA, aB;  // rows p-1 and p+1: registers, or the row below / above the block
      if (r == 0) {
        const float2* e = reinterpret_cast<const float2*>(Ep + G::row(1) + oB);
        bA = e[0];
        bB = e[1];
      } else {
        bA = S[rslot<NR>(r - 1, DIR)][0];
        bB = S[rslot<NR>(r - 1, DIR)][1];
      }
      if (r + 1 == NR) {
        const float2* e = reinterpret_cast<const float2*>(Ep + G::row(0) + oA);
        aA = e[0];
        aB = e[1];
      } else {
        aA = S[rslot<NR>(r + 1, DIR)][0];
        aB = S[rslot<NR>(r + 1, DIR)][1];
      }
      const float lin = (r & 1) ? lp.y : lp.x;
      const float rin = (r & 1) ? rp.y : rp.x;
      float2 rA, rB;  // residuals of row r
      float2 dA, dB, cup;  // -e_{m,p} of the two column pairs; gamma_p (p+1) from p+1
      tmem_ld12_wait(pre, rA, rB, dA, dB, cup);
      if (i + 1 < NR) tmem_ld12_issue(tres + kRowCols * (DIR == 0 ? r + 1 : r - 1), pre);
      // t = residual + inflows from the left, right, below and above + exit,
      // and in row P-1 the protein birth k_p m that does not leave it.
      float2 tA = rA;
      tA.x = f_fma(c_l, lin, tA.x);   // from m - 1: the left block's c3
      tA.y = f_fma(c_l, B.x, tA.y);   // c1
      tA = v_fma(crA, B, tA);         // from m + 1: (c1, c3)
      tA = v_fma(cdA, bA, tA);
      tA = v_fma(cup, aA, tA);
      tA = v_fma(dA, A, tA);
      float2 tB = v_fma(c_l2, A, rB);
      tB.x = f_fma(crB.x, A.y, tB.x); // from m + 1: c2
      tB.y = f_fma(crB.y, rin, tB.y); // the right block's c0
      tB = v_fma(cdB, bB, tB);
      tB = v_fma(cup, aB, tB);
      tB = v_fma(dB, B, tB);
      // (Selections, not branches: the warp stays converged for the
      // tensor-memory store below.)
      const float2 z2 = v_make(0.0f, 0.0f);
      if (EDGE) {
        tA = v_fma(r == rtk ? cdA : z2, A, tA);
        tB = v_fma(r == rtk ? cdB : z2, B, tB);
      } else if (r == NR - 1) {
        tA = v_fma(topA, A, tA);
        tB = v_fma(topB, B, tB);
      }
      float2 yA = comp_finish(A, tA, rA);
      float2 yB = comp_finish(B, tB, rB);
      if (EDGE) {
        const bool beyond = rtk >= 0 && r > rtk;  // rows beyond the box
        yA = beyond ? z2 : yA;
        yB = beyond ? z2 : yB;
        rA = beyond ? z2 : rA;
        rB = beyond ? z2 : rB;
        // Padding columns of the last quad: c1 (bit 1), c2 (bit 2), c3 (bit 3).
        const bool p1c = !(colmask & 2), p2c = !(colmask & 4), p3c = !(colmask & 8);
        yB.x = p1c ? 0.0f : yB.x;
        rB.x = p1c ? 0.0f : rB.x;
        yA.y = p2c ? 0.0f : yA.y;
        rA.y = p2c ? 0.0f : rA.y;
        yB.y = p3c ? 0.0f : yB.y;
        rB.y = p3c ? 0.0f : rB.y;
      }
      tmem_st4(tres + kRowCols * r, rA, rB);
      S[sn][0] = yA;
      S[sn][1] = yB;
    }
  };

  // Exit-defect correction of rho_k (rotation ROT): every state adds p.renorm
  // x its defect x its value to its residual (zero coefficients and values
  // outside the box keep those residuals zero).
  const float period = (float)p.renorm;
  auto defect_fix = [&](auto ROTC) {
    constexpr int ROT = decltype(ROTC)::value;
    tmem_wait_st();
    // Column parts: e0 in FP32 as mrna_col forms it, eps from tensor memory.
    MrnaCol mcol[kQC];
    {
      float2 eA, eB, dummy;
      tmem_ld4(tres + 8u, dummy, eA);
      tmem_ld4(tres + kRowCols + 8u, dummy, eB);
      const float ep[kQC] = {eA.x, eB.x, eA.y, eB.y};
#pragma unroll
      for (int c = 0; c < kQC; ++c) {
        mcol[c].e0 = mrna_col(co, m0 + c, M).e0;
        mcol[c].eps = ep[c];
      }
    }
    // The rows of rho_k, by row index, in a per-thread local array (the row
    // loop is not unrolled, and registers cannot be indexed at run time).
    float4 rows[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const float2 a = S[rslot<NR>(r, ROT)][0], b = S[rslot<NR>(r, ROT)][1];
      rows[r] = make_float4(a.x, a.y, b.x, b.y);
    }
#pragma unroll 1
    for (int r = 0; r < NR; ++r) {
      const int pr = pb + r;
      float2 rA, rB;
      tmem_ld4(tres + kRowCols * r, rA, rB);
      float b[kQC];
#pragma unroll
      for (int c = 0; c < kQC; ++c) b[c] = own * __fmul_rn(period, mrna_defect(mcol[c], co.d, pr));
      const float4 y4 = rows[r];
      const float2 ya = make_float2(y4.x, y4.y), yb = make_float2(y4.z, y4.w);
      rA = v_fma(v_make(b[0], b[2]), ya, rA);
      rB = v_fma(v_make(b[1], b[3]), yb, rB);
      tmem_st4(tres + kRowCols * r, rA, rB);
    }
  };

  // ---- the jump chain -------------------------------------------------------
  int k = 1;
  // Next defect correction (never reached when off: K < 2^30).
  int kdef = p.renorm > 0 ? p.renorm : 0x7fffffff;
  // Jumps with work besides the update, the edges and the observations (a
  // chunk of weights lands (jump = 31 mod kChunk) or is staged (1 mod
  // kChunk), the defect correction, a change of the active window range) are
  // "events"; every other jump tests one counter.  act: this thread has
  // observations to accumulate in the active range.
  auto next_event = [&](int kk) -> int {
    int e = min(kdef, knext);
    e = min(e, (kk + 1) | (kChunk - 1));
    e = min(e, ((kk + kChunk - 1) & ~(kChunk - 1)) + 1);
    return e;
  };
  bool act = owner && lo <= hi;
  const bool do_rec = wwarp && any_rec;
  int kev = min(min(kdef, max(knext, 1)), kChunk - 1);
  // Hand-over waits: bit q of hph is the parity of the next phase of the
  // parity-q barriers.  A completed phase is re-armed (by the column-quad-0
  // thread) for the jump two ahead, before this thread's next row goes out,
  // so the neighbour's bytes of that jump always find it armed.  After a wait
  // that gave up (status kStatusTimeout) the thread stops waiting, arming and
  // sending; a neighbour thread waiting for its rows then gives up too, after
  // at most one more limit, and the chain runs on to its end.
  unsigned hph = 0;
  const bool arm_dn = rx_dn && qx == 0, arm_up = rx_up && qx == 0;
  auto handover = [&](int q) {
    const unsigned ph = (hph >> q) & 1u;
    if (hok) {
      bool ok = !rx_dn || hbar_wait(hb + 8u * (unsigned)q, ph, p.wait_limit);
      if (ok && rx_up) ok = hbar_wait(hb + 16u + 8u * (unsigned)q, ph, p.wait_limit);
      if (ok) {
        if (arm_dn) hbar_arm(hb + 8u * (unsigned)q, hbytes);
        if (arm_up) hbar_arm(hb + 16u + 8u * (unsigned)q, hbytes);
      } else {
        hok = false;
        set_status(p.status, kStatusTimeout);
      }
    }
    hph ^= 1u << q;
  };
  auto step = [&](auto DIRC) {
    constexpr int DIR = decltype(DIRC)::value;
    constexpr int ROT = 1 - DIR;  // rotation of rho_k
    const int par = (k - 1) & 1;
    if (edge_w) update(par, DIRC, std::true_type{});
    else update(par, DIRC, std::false_type{});
    publish(par ^ 1, std::integral_constant<int, ROT>{}, std::false_type{});
    // Chunk c (jumps [c kChunk, (c+1) kChunk)) is staged at jump (c-1) kChunk + 1,
    // after the last read of the slots it reuses (chunk c-2's, read up to jump
    // (c-1) kChunk - 1), and waited for at jump c kChunk - 1, before the barrier
    // that precedes its first read.
    // The exit-defect correction, the window range and the next chunk of
    // weights (whose slots are not the ones read at this jump) at events;
    // the observations of rho_k; the recurrence one jump ahead.
    if (k == kev) {
      if ((k & (kChunk - 1)) == kChunk - 1) cp_async_wait<0>();
      if (k == kdef) {
        kdef += p.renorm;
        defect_fix(std::integral_constant<int, ROT>{});
      }
      if (k >= knext) {
        advance(k, lo, hi);
        knext = next_change(lo, hi);
        act = owner && lo <= hi;
      }
      if ((k & (kChunk - 1)) == 1 && k > 1 && k - 1 + kChunk <= Kmax) stage_chunk(k - 1 + kChunk);
      kev = next_event(k);
    }
    if (do_rec && k + 1 <= Kmax) rec_step(k + 1);
    // The edges of this CTA's blocks (and its weights) are ordered by the CTA
    // barrier; only the threads next to a CTA boundary also wait for the
    // neighbour's row of rho_k.  The observations of rho_k come after the
    // barrier (they read this thread's registers and ring slots that no one
    // rewrites before the next barrier), so the warps that hold observed
    // states sum them while the others start the next jump.
    __syncthreads();
    if (act) accumulate(k, lo, hi, std::integral_constant<int, ROT>{});
    if (rx_dn || rx_up) handover(k & 1);
    __syncwarp();
    ++k;
  };
  while (k + 1 <= Kmax) {
    step(std::integral_constant<int, 0>{});
    step(std::integral_constant<int, 1>{});
  }
  if (k <= Kmax) step(std::integral_constant<int, 0>{});
  // rho_Kmax may be left at rotation 1; only the accumulators are read below.
  cp_async_wait<0>();

  // ---- epilogue: sum_g c_g log(a_g) over the cluster's accumulators ---------
  if (C > 1) cluster.sync();
  else __syncthreads();
  if (rank == 0) {
    double ll = 0.0;
    bool bad = false;
    for (int g = tid; g < p.G; g += blockDim.x) {
      double a = 0.0;
      const int q0 = (int)p.mptr[g], q1 = (int)p.mptr[g + 1];
      for (int q = q0; q < q1; ++q)
        for (int r = 0; r < C; ++r) {
          const float* rs = (C == 1) ? acc_s : cluster.map_shared_rank(acc_s, r);
          const float* rc = (C == 1) ? acc_c : cluster.map_shared_rank(acc_c, r);
          double v = (double)rs[q];
          v -= (double)rc[q];
          a += v;
        }
      const double c = p.counts[g];
      if (c == 0.0) continue;
      if (a > 0.0) ll += c * log(a);
      else if (a > -1e-30) ll = -INFINITY;
      else bad = true;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ll += __shfl_xor_sync(kFull, ll, o);
    double* red = reinterpret_cast<double*>(smem + L.edge);  // the edge arrays are no longer needed
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
  // Keep every CTA's accumulators alive until rank 0 is done, and every
  // residual store complete before the tensor memory is released.
  __syncwarp();
  tmem_wait_st();
  tmem_fence_before();
  if (C > 1) cluster.sync();
  else __syncthreads();
  tmem_fence_after();
  if (warp == 0) tmem_dealloc(tmem_base, tmem_cols<kT>());
}

}  // namespace

// Cluster size, rows per CTA and threads for an M x P box, or false when the
// box does not fit this kernel (then the shared-memory kernel runs).
bool chain_reg2d_plan(int64_t M, int64_t P, int ntimes, int nmem, int max_cluster, int threads, RegPlan* out) {
  if (M < 1 || P < 1 || ntimes < 1) return false;
  if (threads != 0 && threads != 256) return false;
  const int NQ = (int)((M + kQC - 1) / kQC);
  if (NQ > kMaxNQ) return false;
  // Fewest CTAs per instance first; for each, 8 rows per thread before 10.
  // threads = 256 asks for two CTAs per SM (then the edge arrays are half as
  // large and a CTA must fit half the shared memory).
  const int T = threads == 256 ? 256 : 512;
  const size_t smem_cap = T == 256 ? 113 * 1024 : 227 * 1024;
  for (int C = 1; C <= max_cluster; ++C)
    for (int QR = 4; QR <= 5; ++QR) {
      const int rows_blk = 2 * QR;
      const int64_t rows = (P + C - 1) / C;
      const int RS = (int)((rows + rows_blk - 1) / rows_blk) * rows_blk;
      if ((int64_t)(C - 1) * RS >= P) continue;  // the last CTA would be empty
      const int Tc = NQ * (RS / rows_blk);
      if (Tc > T) continue;
      size_t edge;
      if (T == 256) edge = 2 * (QR == 5 ? EdgeGeo<5, 256>::par_bytes : EdgeGeo<4, 256>::par_bytes);
      else edge = 2 * (QR == 5 ? EdgeGeo<5, 512>::par_bytes : EdgeGeo<4, 512>::par_bytes);
      const RegLayout L = reg_layout(edge, ntimes, nmem);
      if (L.total + 1024 > smem_cap) continue;  // leave room for static shared memory
      out->cluster = C;
      out->rows = RS;
      out->nq = NQ;
      out->qr = QR;
      out->tmax = T;
      out->threads = ((Tc + 31) / 32) * 32;
      out->smem = L.total;
      return true;
    }
  return false;
}

template <int QR, int T>
cudaError_t launch_reg(const ChainParams& p, const RegPlan& rp, cudaStream_t s) {
  static int smem_set = 0;
  static bool nonportable = false;
  auto kern = chain_reg2d_kernel<QR, T>;
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
  return cudaLaunchKernelEx(&cfg, kern, p, rp.nq, rp.rows);
}

cudaError_t launch_chain_reg2d(const ChainParams& p, const RegPlan& rp, cudaStream_t s) {
  if (p.B <= 0) return cudaSuccess;
  if (rp.tmax == 256) return rp.qr == 5 ? launch_reg<5, 256>(p, rp, s) : launch_reg<4, 256>(p, rp, s);
  return rp.qr == 5 ? launch_reg<5, 512>(p, rp, s) : launch_reg<4, 512>(p, rp, s);
}

}  // namespace mjp
