// plan.cu -- the FP64 planner: Omega, truncation index K and Poisson weight
// window of every (instance, time) pair (Eq. B_def, Algorithm 2).
//
// One CTA per instance.  Omega = 1.1 max_n e_n is a block max-reduction over
// the matrix-free exit rates (stencil models) or taken from the model (CSR).
// Each warp then plans one time: K = floor(x + 6 sqrt x) + 1 with x = Omega t
// computed with exactly the roundings of Algorithm 2 (no fused multiply-add),
// and the Poisson weights around the mode m = floor(x) as ratios to w_m = 1,
// formed by warp-shuffle inclusive product scans of x/k (upwards) and
// (k+1)/x (downwards).  No exp(-x) is ever formed, so nothing underflows; the
// window sum W normalises the weights, and the tail mass beyond K is summed
// explicitly (equal to 1 - sum_{k<=K} P_k, Algorithm 2's last line).
#include "internal.cuh"

namespace mjp {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ double warp_incl_prod(double v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    double t = __shfl_up_sync(kFull, v, o);
    if (lane >= o) v = __dmul_rn(v, t);
  }
  return v;
}

__device__ __forceinline__ double warp_incl_sum(double v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    double t = __shfl_up_sync(kFull, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

struct Kahan {
  double s = 0.0, c = 0.0;
  __device__ void add(double v) {
    double y = v - c;
    double t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

// Exit rate e_n = sum_m lambda_nm of a stencil model, summed in ascending
// target order (the column order of the rate matrix row) so that Omega is
// bit-identical to a row sum over a CSR with sorted columns.
__device__ double exit_rate(int kind, int64_t M, int64_t P, int64_t n, const double* th) {
  double e = 0.0;
  if (kind == MJP_BD1D) {  // Eq. BD_def
    if (n >= 1) e = __dadd_rn(e, __dmul_rn(th[1], (double)n));
    if (n + 1 < M) e = __dadd_rn(e, th[0]);
  } else if (kind == MJP_TWOSTATE) {  // Eq. Gene_def, sigma = 0 active
    int64_t sg = n / M, nr = n - sg * M;
    if (sg == 0) {
      if (nr >= 1) e = __dadd_rn(e, __dmul_rn(th[1], (double)nr));
      if (nr + 1 < M) e = __dadd_rn(e, th[0]);
      e = __dadd_rn(e, th[3]);
    } else {
      e = __dadd_rn(e, th[2]);
      if (nr >= 1) e = __dadd_rn(e, __dmul_rn(th[1], (double)nr));
    }
  } else if (kind == MJP_AUTOREG) {  // model index n_R + N_R n_P + N_R N_P sigma; P = 2 N_P tile rows
    const int64_t Pm = P / 2, sg = n / (M * Pm), rem = n - sg * M * Pm, q = rem / M, m = rem - q * M;
    // th = {beta_R, beta_P, gamma_R, gamma_P, lambda_act, lambda_ina}, targets ascending
    if (sg == 1 && q + 1 < Pm) e = __dadd_rn(e, th[4]);
    if (q >= 1) e = __dadd_rn(e, __dmul_rn(th[3], (double)q));
    if (m >= 1) e = __dadd_rn(e, __dmul_rn(th[2], (double)m));
    if (sg == 0 && m + 1 < M) e = __dadd_rn(e, th[0]);
    if (q + 1 < Pm && m >= 1) e = __dadd_rn(e, __dmul_rn(th[1], (double)m));
    if (sg == 0 && q >= 1) e = __dadd_rn(e, __dmul_rn(th[5], (double)q));
  } else {  // MRNA_PROT2D: targets n-M, n-1, n+1, n+M
    int64_t p = n / M, m = n - p * M;
    if (p >= 1) e = __dadd_rn(e, __dmul_rn(th[3], (double)p));
    if (m >= 1) e = __dadd_rn(e, __dmul_rn(th[1], (double)m));
    if (m + 1 < M) e = __dadd_rn(e, th[0]);
    if (p + 1 < P && m >= 1) e = __dadd_rn(e, __dmul_rn(th[2], (double)m));
  }
  return e;
}

__device__ void set_status(int* st, int code) {
  if (st) atomicCAS(st, 0, code);
}

// Window [L, K] of x = Omega t under the paper's rule: Algorithm 2's last k
// and the first k whose left Poisson tail is not negligible; false when
// there is no chain (x = 0) or K exceeds the cap.
__device__ bool window_bounds(const PlanParams& p, double x, int64_t& L, int64_t& K) {
  if (x == 0.0) return false;
  const double s = __dsqrt_rn(x);
  const double kstar = __dadd_rn(x, __dmul_rn(6.0, s));  // Omega t + 6 sqrt(Omega t)
  if (!(kstar + 1.0 <= (double)p.kcap)) return false;
  K = (int64_t)floor(kstar) + 1;
  const double lo = __dsub_rn(x, __dmul_rn(10.0, s));  // Poisson left tail below x - 10 sqrt x is < e^-50
  L = lo > 0.0 ? (int64_t)floor(lo) : 0;
  return true;
}

// Float-float numbers (hi + lo, |lo| <= ulp(hi) / 2: ~48 significant bits)
// on the FP32 pipe, which GB300 runs 64 times faster than its FP64 pipe.
// Error-free transformations: TwoSum (Knuth), FastTwoSum (Dekker, |a| >= |b|)
// and TwoProd with a fused multiply-add; every operation explicitly rounded.
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF ff_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return FF{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ FF ff_from(double d) {
  const float hi = __double2float_rn(d);
  return FF{hi, __double2float_rn(d - (double)hi)};
}
__device__ __forceinline__ double ff_to(FF a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff_fast_two_sum(p, e);
}
// a times an integer-valued float c (exact in FP32).
__device__ __forceinline__ FF ff_mul_int(FF a, float c) {
  const float p = __fmul_rn(a.hi, c);
  float e = __fmaf_rn(a.hi, c, -p);
  e = __fmaf_rn(a.lo, c, e);
  return ff_fast_two_sum(p, e);
}
// 1 / c for an integer-valued float c: r0 rounded, plus r0 times the exact
// residual 1 - c r0.
__device__ __forceinline__ FF ff_rcp_int(float c) {
  const float r0 = __frcp_rn(c);
  const float e = __fmaf_rn(-c, r0, 1.0f);
  return ff_fast_two_sum(r0, __fmul_rn(r0, e));
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float v = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return ff_fast_two_sum(s, e);
}
__device__ __forceinline__ FF ff_shfl_up(FF a, int d) {
  return FF{__shfl_up_sync(kFull, a.hi, d), __shfl_up_sync(kFull, a.lo, d)};
}

// Weights of the paper's rule, ratios to w_m = 1 at the mode m = floor(x):
// upward w_k = w_{k-1} x / k over (m, R], downward w_k = w_{k+1} (k+1) / x
// over [L, m).  Each lane forms the running product of a run of kRun
// consecutive terms, one warp-wide product scan joins the runs.  The
// products run in float-float (relative error ~1e-14 over a window of ~10^4
// terms: far below the FP32 weights the chains read and the 1e-12 of the FP64
// chains are served by paper_weights64), and so do the per-lane sums.  Returns the window sum W over [L, R],
// the tail sum over (K, R] and w_L; the unnormalised weights of [L, K] go to
// `put` when `store`.
constexpr int kRun = 8;
__device__ __forceinline__ FF ff_warp_incl_prod(FF v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const FF t = ff_shfl_up(v, o);
    if (lane >= o) v = ff_mul(v, t);
  }
  return v;
}
template <class Put>
__device__ void paper_weights(double x, int64_t L, int64_t K, int64_t m, int64_t R, int lane, bool store,
                              Put& put, double& W, double& tailsum, double& wL) {
  FF sw{lane == 0 ? 1.0f : 0.0f, 0.0f}, st{0.0f, 0.0f}, wl{0.0f, 0.0f};
  if (store && lane == 0) put(m, FF{1.0f, 0.0f});
  const FF xf = ff_from(x), invx = ff_from(1.0 / x);
  FF carry{1.0f, 0.0f};
  for (int64_t base = m + 1; base <= R; base += 32 * kRun) {
    const int64_t k0 = base + (int64_t)lane * kRun;
    FF loc[kRun], pr{1.0f, 0.0f};
#pragma unroll
    for (int b = 0; b < kRun; ++b) {
      const int64_t k = k0 + b;
      const FF term = k <= R ? ff_mul(xf, ff_rcp_int((float)k)) : FF{1.0f, 0.0f};
      pr = ff_mul(pr, term);
      loc[b] = pr;
    }
    const FF incl = ff_warp_incl_prod(pr, lane);
    FF excl = ff_shfl_up(incl, 1);
    if (lane == 0) excl = FF{1.0f, 0.0f};
    const FF pre = ff_mul(carry, excl);
#pragma unroll
    for (int b = 0; b < kRun; ++b) {
      const int64_t k = k0 + b;
      if (k <= R) {
        const FF w = ff_mul(pre, loc[b]);
        sw = ff_add(sw, w);
        if (k > K) st = ff_add(st, w);
        else if (store) put(k, w);
      }
    }
    const FF last = ff_mul(pre, pr);
    carry = FF{__shfl_sync(kFull, last.hi, 31), __shfl_sync(kFull, last.lo, 31)};
  }
  carry = FF{1.0f, 0.0f};
  for (int64_t base = m - 1; base >= L; base -= 32 * kRun) {
    const int64_t k0 = base - (int64_t)lane * kRun;
    FF loc[kRun], pr{1.0f, 0.0f};
#pragma unroll
    for (int b = 0; b < kRun; ++b) {
      const int64_t k = k0 - b;
      const FF term = k >= L ? ff_mul_int(invx, (float)(k + 1)) : FF{1.0f, 0.0f};
      pr = ff_mul(pr, term);
      loc[b] = pr;
    }
    const FF incl = ff_warp_incl_prod(pr, lane);
    FF excl = ff_shfl_up(incl, 1);
    if (lane == 0) excl = FF{1.0f, 0.0f};
    const FF pre = ff_mul(carry, excl);
#pragma unroll
    for (int b = 0; b < kRun; ++b) {
      const int64_t k = k0 - b;
      if (k >= L) {
        const FF w = ff_mul(pre, loc[b]);
        sw = ff_add(sw, w);
        if (store) put(k, w);
        if (k == L) wl = w;
      }
    }
    const FF last = ff_mul(pre, pr);
    carry = FF{__shfl_sync(kFull, last.hi, 31), __shfl_sync(kFull, last.lo, 31)};
  }
  W = warp_sum(ff_to(sw));
  tailsum = warp_sum(ff_to(st));
  wL = (L == m) ? 1.0 : warp_sum(ff_to(wl));  // w_L sits in exactly one lane
}

// The same in FP64 (x / k as x times the reciprocal of k), for the FP64
// chains, whose 1e-12 agreement with the oracle needs weights (and P_L, the
// start of the recurrence of a window without a stored copy) to FP64
// precision.
template <class Put>
__device__ void paper_weights64(double x, int64_t L, int64_t K, int64_t m, int64_t R, int lane, bool store,
                              Put& put, double& W, double& tailsum, double& wL) {
  double sw = lane == 0 ? 1.0 : 0.0, st = 0.0, wl = 0.0;
  if (store && lane == 0) put(m, 1.0);
  double carry = 1.0;
  for (int64_t base = m + 1; base <= R; base += 32 * kRun) {
    const int64_t k0 = base + (int64_t)lane * kRun;
    double loc[kRun], pr = 1.0;
#pragma unroll
    for (int b = 0; b < kRun; ++b) {
      const int64_t k = k0 + b;
      const double term = k <= R ? __dmul_rn(x, __drcp_rn((double)k)) : 1.0;
      pr = __dmul_rn(pr, term);
      loc[b] = pr;
    }
    const double incl = warp_incl_prod(pr, lane);
    double excl = __shfl_up_sync(kFull, incl, 1);
    if (lane == 0) excl = 1.0;
    const double pre = __dmul_rn(carry, excl);
#pragma unroll
    for (int b = 0; b < kRun; ++b) {
      const int64_t k = k0 + b;
      if (k <= R) {
        const double w = __dmul_rn(pre, loc[b]);
        sw += w;
        if (k > K) st += w;
        else if (store) put(k, w);
      }
    }
    carry = __shfl_sync(kFull, __dmul_rn(pre, pr), 31);
  }
  const double invx = __drcp_rn(x);
  carry = 1.0;
  for (int64_t base = m - 1; base >= L; base -= 32 * kRun) {
    const int64_t k0 = base - (int64_t)lane * kRun;
    double loc[kRun], pr = 1.0;
#pragma unroll
    for (int b = 0; b < kRun; ++b) {
      const int64_t k = k0 - b;
      const double term = k >= L ? __dmul_rn((double)(k + 1), invx) : 1.0;
      pr = __dmul_rn(pr, term);
      loc[b] = pr;
    }
    const double incl = warp_incl_prod(pr, lane);
    double excl = __shfl_up_sync(kFull, incl, 1);
    if (lane == 0) excl = 1.0;
    const double pre = __dmul_rn(carry, excl);
#pragma unroll
    for (int b = 0; b < kRun; ++b) {
      const int64_t k = k0 - b;
      if (k >= L) {
        const double w = __dmul_rn(pre, loc[b]);
        sw += w;
        if (store) put(k, w);
        if (k == L) wl = w;
      }
    }
    carry = __shfl_sync(kFull, __dmul_rn(pre, pr), 31);
  }
  W = warp_sum(sw);
  tailsum = warp_sum(st);
  wL = (L == m) ? 1.0 : warp_sum(wl);  // w_L sits in exactly one lane
}

// Plan one time on one warp.  doff: the arena offset reserved for this
// window's weights (paper's rule), or -1.
__device__ void plan_time(const PlanParams& p, double omega, double t, Win* dst, int lane, long long doff_in) {
  Win r;
  double x = __dmul_rn(omega, t);
  r.x = x;
  if (x == 0.0) {  // t = 0 or no transitions: rho*(t) = rho0
    r.L = 0;
    r.K = (p.trunc_mode == MJP_TRUNC_PAPER) ? 1 : 0;
    r.PL = 1.0;
    r.tail = 0.0;
    r.woff = -1;
    if (lane == 0) *dst = r;
    return;
  }
  double s = __dsqrt_rn(x);
  double kstar = __dadd_rn(x, __dmul_rn(6.0, s));  // Omega t + 6 sqrt(Omega t)
  if (!(kstar + 1.0 <= (double)p.kcap)) {  // also catches inf/NaN; nothing loops
    if (lane == 0) {
      set_status(p.status, kStatusKcap);
      // A NaN weight makes this time's result (and a log-likelihood using it)
      // NaN, so a caller that keeps going (a sampler) rejects the parameters.
      r.L = 0; r.K = 0; r.PL = __longlong_as_double(0x7ff8000000000000LL); r.tail = 0.0; r.woff = -1;
      *dst = r;
    }
    return;
  }
  int64_t K = 0, L = 0;
  window_bounds(p, x, L, K);
  int64_t m = (int64_t)floor(x);
  int64_t R = (int64_t)floor(x + 10.0 * s) + 10;

  // Under the paper's rule K is known before the scans: the window [L, K]
  // of the weight arena was reserved by the CTA and receives the
  // unnormalised weights as the scans form them (scaled by 1 / W below), so
  // no second pair of scans is needed.
  const bool direct = p.arena && p.trunc_mode == MJP_TRUNC_PAPER;
  const int64_t dsize = K - L + 1;
  const unsigned long long doff = doff_in >= 0 ? (unsigned long long)doff_in : 0ull;
  const bool dstore = direct && doff_in >= 0;
  // Raw weights: float-float for FP32 chains, FP64 for FP64 chains (whose
  // arena holds doubles).
  auto put_raw = [&](int64_t k, FF w) { reinterpret_cast<float*>(p.arena)[doff + (k - L)] = w.hi; };
  auto put_raw64 = [&](int64_t k, double w) {
    if (p.arena_fp64) reinterpret_cast<double*>(p.arena)[doff + (k - L)] = w;
    else reinterpret_cast<float*>(p.arena)[doff + (k - L)] = (float)w;
  };
  if (p.trunc_mode == MJP_TRUNC_PAPER) {
    double W, ts, wL;
    if (p.fp64_weights || p.arena_fp64) paper_weights64(x, L, K, m, R, lane, dstore, put_raw64, W, ts, wL);
    else paper_weights(x, L, K, m, R, lane, dstore, put_raw, W, ts, wL);
    r.L = L;
    r.K = K;
    r.PL = wL / W;
    r.tail = ts / W;
    r.woff = -1;
    if (dstore) {
      r.woff = (int64_t)doff;
      __syncwarp();  // every lane's raw weights are visible to the lane that scales them
      const double invW = __ddiv_rn(1.0, W);
      if (p.arena_fp64) {
        double* a = reinterpret_cast<double*>(p.arena) + doff;
        for (int64_t j = lane; j < dsize; j += 32) {
          double v = __dmul_rn(a[j], invW);
          if (L + j == K) v = v + r.tail;
          a[j] = v;
        }
      } else {  // FP32 weights scaled in float-float on the FP32 pipe
        float* a = reinterpret_cast<float*>(p.arena) + doff;
        const FF invWf = ff_from(invW);
        for (int64_t j = lane; j < dsize; j += 32) {
          FF v = ff_mul(FF{a[j], 0.0f}, invWf);
          if (L + j == K) v = ff_add(v, ff_from(r.tail));
          a[j] = __fadd_rn(v.hi, v.lo);
        }
      }
    }
    if (lane == 0) *dst = r;
    return;
  }

  // Tolerance rule.  Upward from the mode: w_k = w_{k-1} x / k, w_m = 1.
  Kahan sum;
  if (lane == 0) sum.add(1.0);
  double carry = 1.0;
  for (int64_t base = m + 1; base <= R; base += 32) {
    int64_t k = base + lane;
    double term = (k <= R) ? __ddiv_rn(x, (double)k) : 1.0;
    double w = __dmul_rn(warp_incl_prod(term, lane), carry);
    carry = __shfl_sync(kFull, w, 31);
    if (k <= R) sum.add(w);
  }
  double wR = carry;
  // Downward from the mode: w_k = w_{k+1} (k+1) / x.
  double wL = (L == m) ? 1.0 : 0.0;
  carry = 1.0;
  for (int64_t base = m - 1; base >= L; base -= 32) {
    int64_t k = base - lane;
    double term = (k >= L) ? __ddiv_rn((double)(k + 1), x) : 1.0;
    double w = __dmul_rn(warp_incl_prod(term, lane), carry);
    carry = __shfl_sync(kFull, w, 31);
    if (k >= L) sum.add(w);
    if (k == L) wL = w;
  }
  double W = warp_sum(sum.s) - warp_sum(sum.c);
  // wL sits in exactly one lane (or lane-uniformly 1.0 when L == m).
  wL = (L == m) ? 1.0 : warp_sum(wL);

  double tail;
  {
    // Smallest K with sum_{j>K} w_j <= tol W: walk down from R with suffix sums.
    double thr = p.tol * W;
    double S = 0.0;   // sum_{j > base}
    double wnext = wR;  // w_{base+1} after the first chunk; starts as w_R for base = R-1
    int64_t Kt = R;
    bool found = false;
    for (int64_t base = R - 1; base >= m && !found; base -= 32) {
      int64_t k = base - lane;
      bool valid = k >= m;
      double term = valid ? __ddiv_rn((double)(k + 1), x) : 1.0;
      double w = __dmul_rn(warp_incl_prod(term, lane), wnext);  // w_k
      // S_k = sum_{j>k} w_j = S + w_{base+1} + ... + w_{k+1}; w_{base+1} = wnext.
      double incl = warp_incl_sum(valid ? w : 0.0, lane);
      double excl = incl - (valid ? w : 0.0);
      double Sk = S + wnext + excl;
      unsigned ok = __ballot_sync(kFull, valid && Sk <= thr);
      unsigned vmask = __ballot_sync(kFull, valid);
      if ((ok & vmask) != vmask) {
        int j = __ffs(~ok) - 1;  // first failing lane: passing lanes form a prefix
        Kt = base - j + 1;
        found = true;
      } else {
        Kt = base - (__popc(vmask) - 1);
      }
      S = S + wnext + __shfl_sync(kFull, incl, 31) - __shfl_sync(kFull, valid ? w : 0.0, 31);
      wnext = __shfl_sync(kFull, w, 31);
    }
    K = Kt;
    // tail = sum_{j > K} w_j / W, recomputed upward from the mode for clarity.
    Kahan ts;
    carry = 1.0;
    for (int64_t base = m + 1; base <= R; base += 32) {
      int64_t k = base + lane;
      double term = (k <= R) ? __ddiv_rn(x, (double)k) : 1.0;
      double w = __dmul_rn(warp_incl_prod(term, lane), carry);
      carry = __shfl_sync(kFull, w, 31);
      if (k <= R && k > K) ts.add(w);
    }
    tail = (warp_sum(ts.s) - warp_sum(ts.c)) / W;
  }
  r.L = L;
  r.K = K;
  r.PL = wL / W;
  r.tail = tail;
  r.woff = -1;
  // P_L..P_K (the tail folded into P_K) in the arena, so the chain reads the
  // weights instead of running the recurrence (K is known only now: the same
  // product scans run again).
  if (p.arena) {
    const int64_t size = K - L + 1;
    unsigned long long off = 0;
    if (lane == 0) off = atomicAdd(p.arena_used, (unsigned long long)size);
    off = __shfl_sync(kFull, off, 0);
    if ((int64_t)off + size <= p.arena_cap) {
      r.woff = (int64_t)off;
      auto put = [&](int64_t k, double w) {
        double v = __ddiv_rn(w, W);
        if (k == K) v = v + tail;
        if (p.arena_fp64) reinterpret_cast<double*>(p.arena)[off + (k - L)] = v;
        else reinterpret_cast<float*>(p.arena)[off + (k - L)] = (float)v;
      };
      if (lane == 0) put(m, 1.0);
      carry = 1.0;
      for (int64_t base = m + 1; base <= K; base += 32) {
        int64_t k = base + lane;
        double term = (k <= R) ? __ddiv_rn(x, (double)k) : 1.0;
        double w = __dmul_rn(warp_incl_prod(term, lane), carry);
        carry = __shfl_sync(kFull, w, 31);
        if (k <= K) put(k, w);
      }
      carry = 1.0;
      for (int64_t base = m - 1; base >= L; base -= 32) {
        int64_t k = base - lane;
        double term = (k >= L) ? __ddiv_rn((double)(k + 1), x) : 1.0;
        double w = __dmul_rn(warp_incl_prod(term, lane), carry);
        carry = __shfl_sync(kFull, w, 31);
        if (k >= L) put(k, w);
      }
    } else if (lane == 0 && p.arena_over) {
      atomicOr(p.arena_over, 1);
    }
  }
  if (lane == 0) *dst = r;
}

__global__ void __launch_bounds__(256) plan_kernel(PlanParams p) {
  const int job = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ double red[8];
  __shared__ double s_omega;
  double omega;
  if (p.omega_fixed >= 0.0) {
    omega = p.omega_fixed;
  } else {
    const double* th = p.theta + (int64_t)job * p.ntheta;
    const int64_t NJ = p.jobN ? (int64_t)p.jobN[job] : p.N;
    const int64_t MJ = p.jobN ? NJ : p.M;
    double mx = 0.0;
    for (int64_t n = tid; n < NJ; n += blockDim.x) {
      double e = exit_rate(p.kind, MJ, p.P, n, th);
      mx = e > mx ? e : mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double t = __shfl_xor_sync(kFull, mx, o);
      mx = t > mx ? t : mx;
    }
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    if (tid == 0) {
      double v = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = red[w] > v ? red[w] : v;
      s_omega = (v > 0.0) ? __dmul_rn(p.omega_factor, v) : 0.0;
    }
    __syncthreads();
    omega = s_omega;
  }
  Win* wj = p.win + (int64_t)job * p.ntimes;
  const double* tj = p.times + (p.times_per_job ? (int64_t)job * p.ntimes : 0);
  // Paper's rule: the weight windows of all this instance's times are
  // reserved in one piece, in time order (the same layout every call, and an
  // instance's windows either all fit or all run the chain's recurrence).
  __shared__ long long s_off[kMaxTimes];
  const bool direct = p.arena && p.trunc_mode == MJP_TRUNC_PAPER;
  if (direct) {
    for (int i = tid; i < p.ntimes; i += blockDim.x) {
      int64_t L = 0, K = 0;
      s_off[i] = window_bounds(p, __dmul_rn(omega, tj[i]), L, K) ? (long long)(K - L + 1) : 0;
    }
    __syncthreads();
    if (tid == 0) {
      long long tot = 0;
      for (int i = 0; i < p.ntimes; ++i) {
        const long long sz = s_off[i];
        s_off[i] = sz > 0 ? tot : -1;
        tot += sz;
      }
      const unsigned long long base = tot > 0 ? atomicAdd(p.arena_used, (unsigned long long)tot) : 0ull;
      const bool fit = (long long)base + tot <= (long long)p.arena_cap;
      for (int i = 0; i < p.ntimes; ++i) s_off[i] = (fit && s_off[i] >= 0) ? (long long)base + s_off[i] : -1;
      if (!fit && p.arena_over) atomicOr(p.arena_over, 1);
    }
    __syncthreads();
  }
  for (int i = warp; i < p.ntimes; i += blockDim.x >> 5)
    plan_time(p, omega, tj[i], wj + i, lane, direct ? s_off[i] : -1);
  __syncthreads();
  if (tid == 0) {
    int64_t kmax = 0;
    for (int i = 0; i < p.ntimes; ++i) kmax = wj[i].K > kmax ? wj[i].K : kmax;
    p.info[job].omega = omega;
    p.info[job].Kmax = kmax;
  }
}

// Longest chain first: map[r] = the job of rank r by decreasing Kmax (ties
// by index), so clusters that start in later waves carry the short chains.
// Each thread ranks one job against all others (a strict total order, so the
// map is a permutation whatever the keys hold).
__global__ void order_jobs_kernel(const JobInfo* info, int B, int32_t* map) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B; i += gridDim.x * blockDim.x) {
    const int64_t ki = info[i].Kmax;
    int r = 0;
    for (int j = 0; j < B; ++j) {
      const int64_t kj = info[j].Kmax;
      r += (kj > ki || (kj == ki && j < i)) ? 1 : 0;
    }
    map[r] = i;
  }
}

}  // namespace

cudaError_t launch_plan(const PlanParams& p, cudaStream_t s) {
  if (p.B <= 0) return cudaSuccess;
  plan_kernel<<<p.B, 256, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_order_jobs(const JobInfo* info, int B, int32_t* map, cudaStream_t s) {
  if (B <= 0) return cudaSuccess;
  const int blocks = (B + 255) / 256 < 1024 ? (B + 255) / 256 : 1024;
  order_jobs_kernel<<<blocks, 256, 0, s>>>(info, B, map);
  return cudaGetLastError();
}

}  // namespace mjp
