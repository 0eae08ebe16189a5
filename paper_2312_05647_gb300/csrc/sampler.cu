// sampler.cu -- the posterior sampler of include/mjp_surrogate.h:
// Metropolis-Hastings on Psi = log(theta) (SI A.1, Eq. prop, Eq. prior), the
// adaptive covariance of Eq. update_S (SI A.2, SI A.4.3), delayed acceptance
// with the surrogate as first stage (Christen & Fox 2005), and Geyer's
// initial-monotone-sequence effective sample size.
//
// All chain arithmetic runs in kernels: proposals (Philox4x32-10 +
// Box-Muller), acceptance, the surrogate screen, survivor compaction, the
// covariance update with its Cholesky factor, and the ESS.  The exact
// log-likelihood of a round's proposals is one batched loglik() launch
// (planner + persistent chain kernel).  The host only sequences launches and,
// under delayed acceptance, reads the survivor count once per round (the
// batch size of the exact launch).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "host_util.h"
#include "mjp_surrogate.h"
#include "mlp_dev.cuh"
#include "philox.cuh"

using namespace mjp;

namespace mjp {
int model_kind(const mjp_model* m);
int model_take_status(mjp_model* m, cudaStream_t s, int* status);
const float* mlp_params(const mjp_mlp* net);
const void* mlp_norm(const mjp_mlp* net);
}  // namespace mjp

namespace {

constexpr int NP = 4;          // rates per parameter vector
constexpr int NCNT = 5;        // per-chain counters
enum { CNT_ITER = 0, CNT_ACC = 1, CNT_STAGE1 = 2, CNT_EXACT = 3, CNT_FAIL = 4 };
constexpr int NBEST = 1 + NP;  // best log-posterior and its Psi
constexpr double kPriorMu = 1.0, kPriorSigma = 1e5;

// Device view of the sampler state.
struct SD {
  int C;
  int64_t cap, evcap;
  uint32_t k0, k1;
  double* psi;    // [C][4] current Psi
  double* ll;     // [C] exact log-likelihood at psi
  double* scur;   // [C] surrogate at psi
  double* prop;   // [C][4] proposal waiting for (or just given) its exact value
  double* sprop;  // [C] surrogate at prop
  int64_t* it;    // [C] iterations done (the Philox counter)
  int64_t* tgt;   // [C] iteration target of the current run
  int64_t* nrec;  // [C] samples recorded (ring position = nrec % cap)
  int64_t* cnt;   // [C][NCNT]
  double* best;   // [C][NBEST]
  int* pend;      // [C] 1 while a proposal waits for the exact stage
  int* pidx;      // [C] chains of the compacted batch
  double* thb;    // [C][4] theta = exp(Psi') of the batch
  double* llb;    // [C] exact log-likelihood of the batch
  int* ctl;       // [2] survivors, unfinished chains
  double* trace;  // [C][cap][4]
  double* evpsi;  // [evcap][4]
  double* evll;   // [evcap]
  const double* L;  // [16] lower Cholesky factor of Z
};

__device__ __forceinline__ double log_prior(const double* psi) {
  const double c = log(kPriorSigma * sqrt(2.0 * 3.141592653589793));
  double s = 0.0;
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    const double z = (psi[a] - kPriorMu) / kPriorSigma;
    s += -0.5 * z * z - c;
  }
  return s;
}

// min(1, exp(r)), 0 for NaN or a -inf proposal.
__device__ __forceinline__ double accept_prob(double r, double top) {
  if (isnan(r) || top == -INFINITY) return 0.0;
  return r >= 0.0 ? 1.0 : exp(r);
}

__device__ void normals4(uint32_t k0, uint32_t k1, int c, int64_t h, double z[4]) {
  const uint32_t hl = (uint32_t)h, hh = (uint32_t)((uint64_t)h >> 32);
  const uint4 a = philox4x32_10(make_uint4(hl, hh, (uint32_t)c, 0u), k0, k1);
  const uint4 b = philox4x32_10(make_uint4(hl, hh, (uint32_t)c, 1u), k0, k1);
  box_muller(uniform52(a.x, a.y), uniform52(a.z, a.w), z[0], z[1]);
  box_muller(uniform52(b.x, b.y), uniform52(b.z, b.w), z[2], z[3]);
}

__device__ void uniforms2(uint32_t k0, uint32_t k1, int c, int64_t h, double& ua, double& ub) {
  const uint4 w = philox4x32_10(make_uint4((uint32_t)h, (uint32_t)((uint64_t)h >> 32), (uint32_t)c, 2u), k0, k1);
  ua = uniform52(w.x, w.y);
  ub = uniform52(w.z, w.w);
}

// Psi' = Psi + L z (Eq. prop with Z = L L^T).
__device__ void propose(const SD& d, int c, int64_t h, const double* psi, double* out) {
  double z[4];
  normals4(d.k0, d.k1, c, h, z);
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    double s = 0.0;
#pragma unroll
    for (int b = 0; b < NP; ++b) s += d.L[a * 4 + b] * z[b];
    out[a] = psi[a] + s;
  }
}

__device__ void record(const SD& d, int c, const double* psi) {
  const int64_t q = d.nrec[c];
  double* dst = d.trace + ((size_t)c * d.cap + (size_t)(q % d.cap)) * NP;
#pragma unroll
  for (int a = 0; a < NP; ++a) dst[a] = psi[a];
  d.nrec[c] = q + 1;
}

__device__ void note_best(const SD& d, int c, double lpost, const double* psi) {
  double* b = d.best + (size_t)c * NBEST;
  if (lpost > b[0]) {
    b[0] = lpost;
#pragma unroll
    for (int a = 0; a < NP; ++a) b[1 + a] = psi[a];
  }
}

// ---- plain Metropolis-Hastings ------------------------------------------

__global__ void propose_all_kernel(const SD d) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.C) return;
  double psi[4], pr[4];
#pragma unroll
  for (int a = 0; a < NP; ++a) psi[a] = d.psi[c * NP + a];
  propose(d, c, d.it[c], psi, pr);
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    d.prop[c * NP + a] = pr[a];
    d.thb[c * NP + a] = exp(pr[a]);
  }
}

__global__ void mh_accept_kernel(const SD d, int rec, int64_t evbase) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.C) return;
  double psi[4], pr[4];
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    psi[a] = d.psi[c * NP + a];
    pr[a] = d.prop[c * NP + a];
  }
  const int64_t h = d.it[c];
  double ua, ub;
  uniforms2(d.k0, d.k1, c, h, ua, ub);
  const double lnew = d.llb[c];
  const double top = lnew + log_prior(pr);
  const double r = top - (d.ll[c] + log_prior(psi));
  int64_t* cnt = d.cnt + (size_t)c * NCNT;
  if (ua < accept_prob(r, top)) {
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      psi[a] = pr[a];
      d.psi[c * NP + a] = pr[a];
    }
    d.ll[c] = lnew;
    cnt[CNT_ACC] += 1;
    note_best(d, c, top, psi);
  }
  cnt[CNT_ITER] += 1;
  cnt[CNT_EXACT] += 1;
  if (isnan(lnew)) cnt[CNT_FAIL] += 1;
  d.it[c] = h + 1;
  if (rec) record(d, c, psi);
  if (evbase + c < d.evcap) {
#pragma unroll
    for (int a = 0; a < NP; ++a) d.evpsi[(evbase + c) * NP + a] = pr[a];
    d.evll[evbase + c] = lnew;
  }
}

// ---- delayed acceptance -------------------------------------------------

struct Net {
  const float* P;
  const mlp::Norm* nm;
};

// Surrogate s(psi) of one row by the whole 128-thread CTA (same operation
// order as the batched kernels of mlp.cu).  Every thread returns the value.
__device__ double surrogate_row(const mlp::Norm& nm, const double* psi, const float w1[4], float b1, float b2,
                                float w3, float b3, const float* W2s, float* h1, float* red) {
  using namespace mlp;
  const int j = threadIdx.x, lane = j & 31, warp = j >> 5;
  float x[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) x[k] = std_input(nm, psi, k);
  h1[j] = tanhf(layer1(x, w1, b1));
  __syncthreads();
  float a = b2;
  for (int i = 0; i < H; i += 4) {
    const float4 h = *reinterpret_cast<const float4*>(h1 + i);
    a = fmaf(h.x, W2s[i * W2S + j], a);
    a = fmaf(h.y, W2s[(i + 1) * W2S + j], a);
    a = fmaf(h.z, W2s[(i + 2) * W2S + j], a);
    a = fmaf(h.w, W2s[(i + 3) * W2S + j], a);
  }
  a = tanhf(a);
  const float v = warp_sum(a * w3);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  const float f = b3 + red[0] + red[1] + red[2] + red[3];
  __syncthreads();
  return nm.muy + nm.sdy * (double)f;
}

constexpr size_t kScreenSmem = sizeof(float) * ((size_t)mlp::H * mlp::W2S + mlp::H + 4) + sizeof(double) * 8;

// One CTA per chain: screen proposals with the surrogate until one passes
// the first stage, max_inner were screened, or the chain reached its target.
__global__ void __launch_bounds__(128) da_screen_kernel(const SD d, const Net net, int max_inner, int rec,
                                                         int init_s) {
  using namespace mlp;
  extern __shared__ __align__(16) float sm[];
  float* W2s = sm;
  float* h1 = W2s + H * W2S;
  float* red = h1 + H;
  double* bc = reinterpret_cast<double*>(red + 4);  // proposal [4], verdict
  const int c = blockIdx.x, j = threadIdx.x;
  int64_t h = d.it[c];
  const int64_t tg = d.tgt[c];
  if (h >= tg && !init_s) return;
  const Norm nm = *net.nm;
  stage_w2(net.P, W2s);
  float w1[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) w1[k] = net.P[OW1 + k * H + j];
  const float b1 = net.P[OB1 + j], b2 = net.P[OB2 + j], w3 = net.P[OW3 + j], b3 = net.P[OB3];
  double psi[4];
#pragma unroll
  for (int a = 0; a < NP; ++a) psi[a] = d.psi[c * NP + a];
  __syncthreads();
  double scur;
  if (init_s) {
    scur = surrogate_row(nm, psi, w1, b1, b2, w3, b3, W2s, h1, red);
    if (j == 0) d.scur[c] = scur;
  } else {
    scur = d.scur[c];
  }
  int64_t* cnt = d.cnt + (size_t)c * NCNT;
  for (int q = 0; q < max_inner && h < tg; ++q) {
    if (j == 0) {
      double pr[4];
      propose(d, c, h, psi, pr);
#pragma unroll
      for (int a = 0; a < NP; ++a) bc[a] = pr[a];
    }
    __syncthreads();
    double pr[4];
#pragma unroll
    for (int a = 0; a < NP; ++a) pr[a] = bc[a];
    const double sp = surrogate_row(nm, pr, w1, b1, b2, w3, b3, W2s, h1, red);
    if (j == 0) {
      double ua, ub;
      uniforms2(d.k0, d.k1, c, h, ua, ub);
      const double top = sp + log_prior(pr);
      const double r = top - (scur + log_prior(psi));
      bc[4] = (ua < accept_prob(r, 0.0)) ? 1.0 : 0.0;
    }
    __syncthreads();
    const bool pass = bc[4] != 0.0;
    ++h;
    if (pass) {
      if (j == 0) {
#pragma unroll
        for (int a = 0; a < NP; ++a) d.prop[c * NP + a] = pr[a];
        d.sprop[c] = sp;
        d.pend[c] = 1;
        cnt[CNT_STAGE1] += 1;
      }
      break;
    }
    if (j == 0) {
      cnt[CNT_ITER] += 1;
      if (rec) record(d, c, psi);
    }
    __syncthreads();  // bc is rewritten by the next proposal
  }
  if (j == 0) d.it[c] = h;
}

// Survivors in chain order -> pidx, theta batch; counts of survivors and of
// chains still below their target.  One block.
__global__ void __launch_bounds__(1024) compact_kernel(const SD d) {
  __shared__ int wsum[32];
  __shared__ int wact[32];
  __shared__ int carry;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  if (t == 0) carry = 0;
  int active = 0;
  for (int base = 0; base < d.C; base += blockDim.x) {
    const int c = base + t;
    const int f = (c < d.C) ? d.pend[c] : 0;
    if (c < d.C && d.it[c] < d.tgt[c]) ++active;
    int x = f;  // inclusive warp scan
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    int off = carry;
    for (int w = 0; w < warp; ++w) off += wsum[w];
    if (f) {
      const int k = off + x - 1;
      d.pidx[k] = c;
#pragma unroll
      for (int a = 0; a < NP; ++a) d.thb[k * NP + a] = exp(d.prop[c * NP + a]);
    }
    __syncthreads();
    if (t == 0) {
      int s = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += wsum[w];
      carry += s;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) active += __shfl_xor_sync(0xffffffffu, active, o);
  if (lane == 0) wact[warp] = active;
  __syncthreads();
  if (t == 0) {
    int s = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += wact[w];
    d.ctl[0] = carry;
    d.ctl[1] = s;
  }
}

__global__ void da_finish_kernel(const SD d, int rec, int64_t evbase) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d.ctl[0]) return;
  const int c = d.pidx[k];
  const int64_t h = d.it[c] - 1;  // the iteration that waited
  double ua, ub;
  uniforms2(d.k0, d.k1, c, h, ua, ub);
  double psi[4], pr[4];
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    psi[a] = d.psi[c * NP + a];
    pr[a] = d.prop[c * NP + a];
  }
  const double lnew = d.llb[k];
  const double r = (lnew - d.ll[c]) - (d.sprop[c] - d.scur[c]);
  int64_t* cnt = d.cnt + (size_t)c * NCNT;
  if (ub < accept_prob(r, lnew)) {
#pragma unroll
    for (int a = 0; a < NP; ++a) {
      psi[a] = pr[a];
      d.psi[c * NP + a] = pr[a];
    }
    d.ll[c] = lnew;
    d.scur[c] = d.sprop[c];
    cnt[CNT_ACC] += 1;
    note_best(d, c, lnew + log_prior(psi), psi);
  }
  cnt[CNT_ITER] += 1;
  cnt[CNT_EXACT] += 1;
  if (isnan(lnew)) cnt[CNT_FAIL] += 1;
  d.pend[c] = 0;
  if (rec) record(d, c, psi);
  if (evbase + k < d.evcap) {
#pragma unroll
    for (int a = 0; a < NP; ++a) d.evpsi[(evbase + k) * NP + a] = pr[a];
    d.evll[evbase + k] = lnew;
  }
}

// ---- state, covariance ----------------------------------------------------

__global__ void exp_kernel(const double* __restrict__ psi, double* __restrict__ th, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) th[i] = exp(psi[i]);
}

__global__ void set_best_kernel(const SD d) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d.C) return;
  double psi[4];
#pragma unroll
  for (int a = 0; a < NP; ++a) psi[a] = d.psi[c * NP + a];
  double* b = d.best + (size_t)c * NBEST;
  b[0] = d.ll[c] + log_prior(psi);
  if (isnan(b[0])) b[0] = -INFINITY;
#pragma unroll
  for (int a = 0; a < NP; ++a) b[1 + a] = psi[a];
}

__global__ void set_target_kernel(const SD d, int64_t iters) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < d.C) d.tgt[c] = d.it[c] + iters;
}

// Lower Cholesky factor, column by column; ok = 0 if Z is not positive definite.
__device__ bool cholesky4(const double* Z, double* L) {
  for (int i = 0; i < 16; ++i) L[i] = 0.0;
  for (int j = 0; j < 4; ++j) {
    double dsum = Z[j * 4 + j];
    for (int k = 0; k < j; ++k) dsum -= L[j * 4 + k] * L[j * 4 + k];
    if (!(dsum > 0.0)) return false;
    const double ljj = sqrt(dsum);
    L[j * 4 + j] = ljj;
    for (int i = j + 1; i < 4; ++i) {
      double s = Z[i * 4 + j];
      for (int k = 0; k < j; ++k) s -= L[i * 4 + k] * L[j * 4 + k];
      L[i * 4 + j] = s / ljj;
    }
  }
  return true;
}

__global__ void chol_kernel(const double* __restrict__ Z, double* __restrict__ Lout, int* __restrict__ ok) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double l[16];
  const bool good = cholesky4(Z, l);
  *ok = good ? 1 : 0;
  if (good)
    for (int i = 0; i < 16; ++i) Lout[i] = l[i];
}

// Eq. update_S on the newest `window` ring samples of every chain (pooled):
// Z = scale (mean(psi^T psi) - mean(psi)^T mean(psi) + eps I), then its
// Cholesky factor.  One block; sums in a fixed order.
__global__ void __launch_bounds__(256) adapt_cov_kernel(const SD d, int64_t window, double eps, double* Zout,
                                                        double* Lout, int* ok) {
  __shared__ double part[256][14];
  const int t = threadIdx.x;
  double s[14];  // 4 sums, then the 10 entries of the upper triangle of sum psi^T psi
  for (int q = 0; q < 14; ++q) s[q] = 0.0;
  const int64_t total = (int64_t)d.C * window;
  for (int64_t e = t; e < total; e += blockDim.x) {
    const int c = (int)(e / window);
    const int64_t q = d.nrec[c] - window + (e % window);
    const double* x = d.trace + ((size_t)c * d.cap + (size_t)(q % d.cap)) * NP;
    int u = 4;
    for (int a = 0; a < NP; ++a) {
      s[a] += x[a];
      for (int b = a; b < NP; ++b) s[u++] += x[a] * x[b];
    }
  }
  for (int q = 0; q < 14; ++q) part[t][q] = s[q];
  __syncthreads();
  if (t != 0) return;
  double S[14];
  for (int q = 0; q < 14; ++q) {
    double v = 0.0;
    for (int i = 0; i < (int)blockDim.x; ++i) v += part[i][q];
    S[q] = v;
  }
  const double n = (double)total, scale = (2.38 / 4.0) * (2.38 / 4.0);
  double mean[4], Z[16];
  for (int a = 0; a < NP; ++a) mean[a] = S[a] / n;
  int u = 4;
  for (int a = 0; a < NP; ++a)
    for (int b = a; b < NP; ++b) {
      const double cov = S[u++] / n - mean[a] * mean[b];
      const double z = scale * (cov + (a == b ? eps : 0.0));
      Z[a * 4 + b] = z;
      Z[b * 4 + a] = z;
    }
  double l[16];
  const bool good = cholesky4(Z, l);
  *ok = good ? 1 : 0;
  if (good)
    for (int i = 0; i < 16; ++i) {
      Zout[i] = Z[i];
      Lout[i] = l[i];
    }
}

__global__ void gather_trace_kernel(const SD d, int64_t kept, double* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)d.C * kept;
  if (e >= total) return;
  const int c = (int)(e / kept);
  const int64_t q = d.nrec[c] - kept + e % kept;
  const double* src = d.trace + ((size_t)c * d.cap + (size_t)(q % d.cap)) * NP;
#pragma unroll
  for (int a = 0; a < NP; ++a) out[e * NP + a] = src[a];
}

// ---- effective sample size ------------------------------------------------

// Per parameter: pooled mean, variance, and variance of the squared
// deviations (two passes, FP64, fixed order).  Block per parameter.
__global__ void __launch_bounds__(256) pooled_moments_kernel(const double* __restrict__ tr, int64_t C, int64_t S,
                                                             int P, double* __restrict__ mom) {
  __shared__ double red[8];
  const int a = blockIdx.x;
  const int64_t n = C * S;
  auto bsum = [&](double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;
  };
  double s = 0.0;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) s += tr[e * P + a];
  const double mean = bsum(s) / (double)n;
  s = 0.0;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
    const double dd = tr[e * P + a] - mean;
    s += dd * dd;
  }
  const double var = bsum(s) / (double)n;
  s = 0.0;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
    const double dd = tr[e * P + a] - mean;
    const double q = dd * dd - var;
    s += q * q;
  }
  const double var_sq = bsum(s) / (double)n;
  if (threadIdx.x == 0) {
    mom[a * 3] = mean;
    mom[a * 3 + 1] = var;
    mom[a * 3 + 2] = var_sq;
  }
}

// Geyer ESS of one chain's series of one parameter (mode 0: x, mode 1:
// (x - pooled mean)^2).  Block per (chain, parameter); the centred series is
// staged in shared memory when it fits.
__global__ void __launch_bounds__(256) chain_ess_kernel(const double* __restrict__ tr, int64_t S, int P, int mode,
                                                        const double* __restrict__ mom, int staged,
                                                        double* __restrict__ ess) {
  extern __shared__ double xs[];
  __shared__ double red[8];
  const int c = blockIdx.x / P, a = blockIdx.x % P;
  const double* x = tr + (size_t)c * S * P + a;
  const double m = mom[a * 3];
  auto val = [&](int64_t t) {
    const double v = x[t * P];
    return mode ? (v - m) * (v - m) : v;
  };
  auto bsum = [&](double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;
  };
  double s = 0.0;
  for (int64_t t = threadIdx.x; t < S; t += blockDim.x) s += val(t);
  const double cm = bsum(s) / (double)S;
  if (staged) {
    for (int64_t t = threadIdx.x; t < S; t += blockDim.x) xs[t] = val(t) - cm;
    __syncthreads();
  }
  auto dev = [&](int64_t t) { return staged ? xs[t] : val(t) - cm; };
  auto gamma = [&](int64_t k) {
    double g = 0.0;
    for (int64_t t = threadIdx.x; t < S - k; t += blockDim.x) g += dev(t) * dev(t + k);
    return bsum(g) / (double)S;
  };
  double result = (double)S;
  if (S >= 4) {
    const double g0 = gamma(0);
    if (g0 > 0.0) {
      double total = -g0, prev = INFINITY;
      for (int64_t mm = 0; 2 * mm + 1 < S; ++mm) {
        double G = gamma(2 * mm) + gamma(2 * mm + 1);
        if (G <= 0.0) break;
        G = fmin(G, prev);
        total += 2.0 * G;
        prev = G;
      }
      // tau >= 1 / log10(S): the bound S log10 S on the ESS that Vehtari et
      // al. (2021, Bayesian Analysis 16(2)) apply to keep antithetic chains stable.
      result = (double)S / fmax(total / g0, 1.0 / log10((double)S));
    }
  }
  if (threadIdx.x == 0) ess[blockIdx.x] = result;
}

__global__ void ess_final_kernel(const double* __restrict__ chain_ess, const double* __restrict__ chain_ess_sq,
                                 const double* __restrict__ mom, int64_t C, int P, double* __restrict__ res) {
  const int a = threadIdx.x;
  if (a >= P) return;
  double e = 0.0, ev = 0.0;
  for (int64_t c = 0; c < C; ++c) {
    e += chain_ess[c * P + a];
    ev += chain_ess_sq[c * P + a];
  }
  const double var = mom[a * 3 + 1], var_sq = mom[a * 3 + 2];
  res[0 * P + a] = e;
  res[1 * P + a] = mom[a * 3];
  res[2 * P + a] = var;
  res[3 * P + a] = sqrt(var / e);
  res[4 * P + a] = sqrt(var_sq / ev);
}

}  // namespace

// ---- host side ------------------------------------------------------------

struct mjp_sampler {
  mjp_model* m = nullptr;
  const mjp_obs* obs = nullptr;
  int C = 0;
  int64_t cap = 0, evcap = 0;
  uint64_t seed = 0;
  DevBuf psi, ll, scur, prop, sprop, it, tgt, nrec, cnt, best, pend, pidx, thb, llb, ctl, trace, evpsi, evll;
  DevBuf Z, L, Zstage, ok;
  int* h_ctl = nullptr;  // pinned: survivors, unfinished, cholesky verdict
  int64_t evn = 0;
  int64_t rounds = 0;
  int64_t kept_base = 0;  // nrec of every chain at the last clear
  ~mjp_sampler() {
    for (DevBuf* b : {&psi, &ll, &scur, &prop, &sprop, &it, &tgt, &nrec, &cnt, &best, &pend, &pidx, &thb, &llb,
                      &ctl, &trace, &evpsi, &evll, &Z, &L, &Zstage, &ok})
      b->release();
    if (h_ctl) cudaFreeHost(h_ctl);
  }
  SD view() const {
    SD d;
    d.C = C;
    d.cap = cap;
    d.evcap = evcap;
    d.k0 = (uint32_t)seed;
    d.k1 = (uint32_t)(seed >> 32);
    d.psi = psi.as<double>();
    d.ll = ll.as<double>();
    d.scur = scur.as<double>();
    d.prop = prop.as<double>();
    d.sprop = sprop.as<double>();
    d.it = it.as<int64_t>();
    d.tgt = tgt.as<int64_t>();
    d.nrec = nrec.as<int64_t>();
    d.cnt = cnt.as<int64_t>();
    d.best = best.as<double>();
    d.pend = pend.as<int>();
    d.pidx = pidx.as<int>();
    d.thb = thb.as<double>();
    d.llb = llb.as<double>();
    d.ctl = ctl.as<int>();
    d.trace = trace.as<double>();
    d.evpsi = evpsi.as<double>();
    d.evll = evll.as<double>();
    d.L = L.as<double>();
    return d;
  }
};

namespace {

unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Batched exact log-likelihood of thb[0..B) into llb (device, asynchronous).
int exact_batch(mjp_sampler* s, int B, cudaStream_t st) {
  return loglik(s->m, s->obs, s->thb.as<double>(), B, s->llb.as<double>(), MJP_PTR_DEVICE, MJP_TRUNC_PAPER, 0.0,
                st);
}

// Status of the exact evaluations: a flagged K cap or non-finite result is a
// rejected proposal (its log-likelihood is NaN); anything else is an error.
int settle(mjp_sampler* s, cudaStream_t st) {
  int status = 0;
  int rc = model_take_status(s->m, st, &status);
  if (rc) return rc;
  if (status == 0 || status == 1 || status == 2) return MJP_OK;
  return fail(status == 3 ? MJP_ERR_DEVICE_TIMEOUT : MJP_ERR_CUDA, "exact log-likelihood failed on the device");
}

int set_cov_device(mjp_sampler* s, const double* Z, cudaStream_t st) {
  MJP_CUDA(cudaMemcpyAsync(s->Zstage.p, Z, 16 * sizeof(double), cudaMemcpyHostToDevice, st));
  chol_kernel<<<1, 1, 0, st>>>(s->Zstage.as<double>(), s->L.as<double>(), s->ok.as<int>());
  MJP_CUDA(cudaGetLastError());
  MJP_CUDA(cudaMemcpyAsync(s->h_ctl + 2, s->ok.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  MJP_CUDA(cudaStreamSynchronize(st));
  if (!s->h_ctl[2]) return fail(MJP_ERR_ARG, "Z is not symmetric positive definite");
  MJP_CUDA(cudaMemcpyAsync(s->Z.p, s->Zstage.p, 16 * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return MJP_OK;
}

int read_counts(mjp_sampler* s, cudaStream_t st, std::vector<int64_t>& cnt, std::vector<int64_t>* nrec) {
  cnt.resize((size_t)s->C * NCNT);
  MJP_CUDA(cudaMemcpyAsync(cnt.data(), s->cnt.p, cnt.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  if (nrec) {
    nrec->resize(s->C);
    MJP_CUDA(cudaMemcpyAsync(nrec->data(), s->nrec.p, s->C * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  }
  MJP_CUDA(cudaStreamSynchronize(st));
  return MJP_OK;
}

int64_t sum_count(const std::vector<int64_t>& cnt, int which) {
  int64_t v = 0;
  for (size_t c = 0; c * NCNT < cnt.size(); ++c) v += cnt[c * NCNT + which];
  return v;
}

}  // namespace

namespace {

// Checkpoint layout: a header, then the device buffers that carry a
// sampler from one run to the next, in the order ckpt_parts lists them.
// Buffers that live only inside a run (proposals, the compacted batch, its
// theta and log-likelihoods, the control words) are not saved.
constexpr uint64_t kCkptMagic = 0x3154504b434d4a4dULL;  // "MJMCKPT1" read as little-endian bytes
constexpr int32_t kCkptVersion = 1;
struct CkptHeader {
  uint64_t magic;
  int32_t version, chains;
  int64_t cap, evcap;
  uint64_t seed;
  int64_t evn, rounds, kept_base;
  int32_t np, ncnt, nbest, pad;
};
template <class F>
void ckpt_parts(mjp_sampler* s, F&& f) {
  const size_t C = (size_t)s->C;
  const size_t ev = (size_t)std::max<int64_t>(s->evcap, 1);
  f(s->psi, C * NP * 8);
  f(s->ll, C * 8);
  f(s->scur, C * 8);
  f(s->it, C * 8);  // the chains' Philox counters
  f(s->nrec, C * 8);
  f(s->cnt, C * NCNT * 8);
  f(s->best, C * NBEST * 8);
  f(s->trace, C * (size_t)s->cap * NP * 8);
  f(s->evpsi, ev * NP * 8);
  f(s->evll, ev * 8);
  f(s->Z, 16 * 8);
  f(s->L, 16 * 8);
}
size_t ckpt_bytes(mjp_sampler* s) {
  size_t n = sizeof(CkptHeader);
  ckpt_parts(s, [&](DevBuf&, size_t b) { n += b; });
  return n;
}

}  // namespace

extern "C" {

int mjp_sampler_create(mjp_sampler** out, mjp_model* m, const mjp_obs* obs, int chains, int64_t capacity,
                       int64_t eval_capacity, uint64_t seed) try {
  if (!out || !m || !obs) return fail(MJP_ERR_ARG, "NULL argument");
  *out = nullptr;
  if (chains < 1 || chains > 4096) return fail(MJP_ERR_ARG, "chains must be in [1, 4096]");
  if (capacity < 1 || eval_capacity < 0) return fail(MJP_ERR_ARG, "capacity must be >= 1, eval_capacity >= 0");
  const int kind = model_kind(m);
  if (kind != MJP_TWOSTATE && kind != MJP_MRNA_PROT2D)
    return fail(MJP_ERR_UNSUPPORTED, "the sampler handles the 4-rate stencil models");
  mjp_sampler* s = new mjp_sampler();
  s->m = m;
  s->obs = obs;
  s->C = chains;
  s->cap = capacity;
  s->evcap = eval_capacity;
  s->seed = seed;
  const size_t C = (size_t)chains;
  int rc = 0;
  auto grab = [&](DevBuf& b, size_t bytes) {
    if (!rc) rc = b.ensure(bytes);
    if (!rc && cudaMemset(b.p, 0, bytes) != cudaSuccess) rc = fail(MJP_ERR_CUDA, "cudaMemset failed");
  };
  grab(s->psi, C * NP * 8);
  grab(s->ll, C * 8);
  grab(s->scur, C * 8);
  grab(s->prop, C * NP * 8);
  grab(s->sprop, C * 8);
  grab(s->it, C * 8);
  grab(s->tgt, C * 8);
  grab(s->nrec, C * 8);
  grab(s->cnt, C * NCNT * 8);
  grab(s->best, C * NBEST * 8);
  grab(s->pend, C * 4);
  grab(s->pidx, C * 4);
  grab(s->thb, C * NP * 8);
  grab(s->llb, C * 8);
  grab(s->ctl, 16);
  grab(s->trace, C * (size_t)capacity * NP * 8);
  grab(s->evpsi, (size_t)std::max<int64_t>(eval_capacity, 1) * NP * 8);
  grab(s->evll, (size_t)std::max<int64_t>(eval_capacity, 1) * 8);
  grab(s->Z, 16 * 8);
  grab(s->L, 16 * 8);
  grab(s->Zstage, 16 * 8);
  grab(s->ok, 16);
  if (!rc && cudaMallocHost(&s->h_ctl, 4 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    rc = fail(MJP_ERR_ALLOC, "pinned allocation failed");
  }
  if (!rc) {
    double Z[16] = {};
    for (int a = 0; a < NP; ++a) Z[a * 4 + a] = 1e-8;
    rc = set_cov_device(s, Z, nullptr);
  }
  if (rc) {
    delete s;
    return rc;
  }
  *out = s;
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

void mjp_sampler_destroy(mjp_sampler* s) {
  if (!s) return;
  cudaDeviceSynchronize();
  delete s;
}

int mjp_sampler_set_state(mjp_sampler* s, const double* psi, int where, void* stream) try {
  if (!s || !psi) return fail(MJP_ERR_ARG, "NULL argument");
  if (where != MJP_PTR_HOST && where != MJP_PTR_DEVICE) return fail(MJP_ERR_ARG, "bad where");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = (size_t)s->C * NP * sizeof(double);
  std::vector<double> h(NP * (size_t)s->C);
  MJP_CUDA(cudaMemcpyAsync(h.data(), psi, bytes, where == MJP_PTR_HOST ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost,
                           st));
  MJP_CUDA(cudaStreamSynchronize(st));
  for (double v : h)
    if (!std::isfinite(v)) return fail(MJP_ERR_ARG, "psi must be finite");
  // The planner sizes its weight arena from the model's rates: use chain 0's.
  double th[NP];
  for (int a = 0; a < NP; ++a) th[a] = std::exp(h[a]);
  int rc = rate_model_set_theta(s->m, th, NP);
  if (rc) return rc;
  MJP_CUDA(cudaMemcpyAsync(s->psi.p, h.data(), bytes, cudaMemcpyHostToDevice, st));
  exp_kernel<<<blocks_for((int64_t)s->C * NP, 256), 256, 0, st>>>(s->psi.as<double>(), s->thb.as<double>(),
                                                                  s->C * NP);
  MJP_CUDA(cudaGetLastError());
  if ((rc = loglik(s->m, s->obs, s->thb.as<double>(), s->C, s->ll.as<double>(), MJP_PTR_DEVICE, MJP_TRUNC_PAPER,
                   0.0, st)))
    return rc;
  SD d = s->view();
  set_best_kernel<<<blocks_for(s->C, 128), 128, 0, st>>>(d);
  MJP_CUDA(cudaGetLastError());
  return settle(s, st);
} catch (...) {
  return ::mjp::exception_status();
}

int mjp_sampler_get_state(mjp_sampler* s, double* psi, double* ll, int where, void* stream) try {
  if (!s) return fail(MJP_ERR_ARG, "NULL sampler");
  if (where != MJP_PTR_HOST && where != MJP_PTR_DEVICE) return fail(MJP_ERR_ARG, "bad where");
  cudaStream_t st = (cudaStream_t)stream;
  const cudaMemcpyKind k = where == MJP_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (psi) MJP_CUDA(cudaMemcpyAsync(psi, s->psi.p, (size_t)s->C * NP * sizeof(double), k, st));
  if (ll) MJP_CUDA(cudaMemcpyAsync(ll, s->ll.p, (size_t)s->C * sizeof(double), k, st));
  if (where == MJP_PTR_HOST) MJP_CUDA(cudaStreamSynchronize(st));
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

int mjp_sampler_set_cov(mjp_sampler* s, const double* Z, void* stream) try {
  if (!s || !Z) return fail(MJP_ERR_ARG, "NULL argument");
  for (int i = 0; i < 16; ++i)
    if (!std::isfinite(Z[i])) return fail(MJP_ERR_ARG, "Z must be finite");
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < a; ++b)
      if (Z[a * 4 + b] != Z[b * 4 + a]) return fail(MJP_ERR_ARG, "Z must be symmetric");
  return set_cov_device(s, Z, (cudaStream_t)stream);
} catch (...) {
  return ::mjp::exception_status();
}

int mjp_sampler_get_cov(mjp_sampler* s, double* Z, void* stream) try {
  if (!s || !Z) return fail(MJP_ERR_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  MJP_CUDA(cudaMemcpyAsync(Z, s->Z.p, 16 * sizeof(double), cudaMemcpyDeviceToHost, st));
  MJP_CUDA(cudaStreamSynchronize(st));
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

int mjp_sampler_adapt_cov(mjp_sampler* s, int64_t window, double eps, void* stream) try {
  if (!s) return fail(MJP_ERR_ARG, "NULL sampler");
  if (window < 2 || window > s->cap) return fail(MJP_ERR_ARG, "window must be in [2, capacity]");
  if (!(eps >= 0.0) || !std::isfinite(eps)) return fail(MJP_ERR_ARG, "eps must be finite and >= 0");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int64_t> cnt, nrec;
  int rc = read_counts(s, st, cnt, &nrec);
  if (rc) return rc;
  for (int64_t q : nrec)
    if (q - s->kept_base < window) return fail(MJP_ERR_ARG, "fewer than `window` samples are kept");
  SD d = s->view();
  adapt_cov_kernel<<<1, 256, 0, st>>>(d, window, eps, s->Z.as<double>(), s->L.as<double>(), s->ok.as<int>());
  MJP_CUDA(cudaGetLastError());
  MJP_CUDA(cudaMemcpyAsync(s->h_ctl + 2, s->ok.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  MJP_CUDA(cudaStreamSynchronize(st));
  if (!s->h_ctl[2]) return fail(MJP_ERR_NUMERIC, "updated Z is not positive definite (Z kept)");
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

int mjp_sampler_run_plain(mjp_sampler* s, int64_t iters, int rec, void* stream) try {
  if (!s) return fail(MJP_ERR_ARG, "NULL sampler");
  if (iters < 0) return fail(MJP_ERR_ARG, "iters must be >= 0");
  cudaStream_t st = (cudaStream_t)stream;
  SD d = s->view();
  const unsigned nb = blocks_for(s->C, 128);
  for (int64_t q = 0; q < iters; ++q) {
    propose_all_kernel<<<nb, 128, 0, st>>>(d);
    MJP_CUDA(cudaGetLastError());
    int rc = exact_batch(s, s->C, st);
    if (rc) return rc;
    mh_accept_kernel<<<nb, 128, 0, st>>>(d, rec ? 1 : 0, s->evn);
    MJP_CUDA(cudaGetLastError());
    s->evn = std::min(s->evn + s->C, s->evcap);
    s->rounds += 1;
  }
  return settle(s, st);
} catch (...) {
  return ::mjp::exception_status();
}

int mjp_sampler_run_da(mjp_sampler* s, mjp_mlp* net, int64_t iters, int max_inner, int rec, void* stream) try {
  if (!s || !net) return fail(MJP_ERR_ARG, "NULL argument");
  if (iters < 0) return fail(MJP_ERR_ARG, "iters must be >= 0");
  if (max_inner < 1 || max_inner > 1024) return fail(MJP_ERR_ARG, "max_inner must be in [1, 1024]");
  cudaStream_t st = (cudaStream_t)stream;
  SD d = s->view();
  Net nw;
  nw.P = mlp_params(net);
  nw.nm = reinterpret_cast<const mlp::Norm*>(mlp_norm(net));
  MJP_CUDA(cudaFuncSetAttribute(da_screen_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScreenSmem));
  set_target_kernel<<<blocks_for(s->C, 128), 128, 0, st>>>(d, iters);
  MJP_CUDA(cudaGetLastError());
  for (int round = 0;; ++round) {
    da_screen_kernel<<<s->C, 128, kScreenSmem, st>>>(d, nw, max_inner, rec ? 1 : 0, round == 0 ? 1 : 0);
    MJP_CUDA(cudaGetLastError());
    compact_kernel<<<1, 1024, 0, st>>>(d);
    MJP_CUDA(cudaGetLastError());
    MJP_CUDA(cudaMemcpyAsync(s->h_ctl, s->ctl.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    MJP_CUDA(cudaStreamSynchronize(st));
    const int npend = s->h_ctl[0], nactive = s->h_ctl[1];
    if (npend > 0) {
      int rc = exact_batch(s, npend, st);
      if (rc) return rc;
      da_finish_kernel<<<blocks_for(npend, 128), 128, 0, st>>>(d, rec ? 1 : 0, s->evn);
      MJP_CUDA(cudaGetLastError());
      s->evn = std::min(s->evn + npend, s->evcap);
      s->rounds += 1;
    }
    if (nactive == 0) break;
  }
  return settle(s, st);
} catch (...) {
  return ::mjp::exception_status();
}

int mjp_sampler_clear(mjp_sampler* s, int evals, void* stream) try {
  if (!s) return fail(MJP_ERR_ARG, "NULL sampler");
  cudaStream_t st = (cudaStream_t)stream;
  MJP_CUDA(cudaMemsetAsync(s->cnt.p, 0, (size_t)s->C * NCNT * sizeof(int64_t), st));
  std::vector<int64_t> cnt, nrec;
  int rc = read_counts(s, st, cnt, &nrec);
  if (rc) return rc;
  for (size_t c = 1; c < nrec.size(); ++c)
    if (nrec[c] != nrec[0]) return fail(MJP_ERR_ARG, "chains hold different sample counts");
  s->kept_base = nrec.empty() ? 0 : nrec[0];
  if (evals) s->evn = 0;
  s->rounds = 0;
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

int mjp_sampler_stats_get(mjp_sampler* s, mjp_sampler_stats* out, void* stream) try {
  if (!s || !out) return fail(MJP_ERR_ARG, "NULL argument");
  std::vector<int64_t> cnt, nrec;
  int rc = read_counts(s, (cudaStream_t)stream, cnt, &nrec);
  if (rc) return rc;
  out->iterations = sum_count(cnt, CNT_ITER);
  out->accepted = sum_count(cnt, CNT_ACC);
  out->stage1 = sum_count(cnt, CNT_STAGE1);
  out->exact_evals = sum_count(cnt, CNT_EXACT);
  out->rounds = s->rounds;
  int64_t kept = s->cap;
  for (int64_t q : nrec) kept = std::min(kept, q - s->kept_base);
  out->kept = std::max<int64_t>(kept, 0);
  out->evals_kept = s->evn;
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

int mjp_sampler_trace(mjp_sampler* s, double* out, int where, void* stream) try {
  if (!s || !out) return fail(MJP_ERR_ARG, "NULL argument");
  if (where != MJP_PTR_HOST && where != MJP_PTR_DEVICE) return fail(MJP_ERR_ARG, "bad where");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int64_t> cnt, nrec;
  int rc = read_counts(s, st, cnt, &nrec);
  if (rc) return rc;
  for (size_t c = 1; c < nrec.size(); ++c)
    if (nrec[c] != nrec[0]) return fail(MJP_ERR_ARG, "chains hold different sample counts");
  const int64_t kept = std::min(s->cap, nrec[0] - s->kept_base);
  if (kept <= 0) return MJP_OK;
  const size_t bytes = (size_t)s->C * kept * NP * sizeof(double);
  DevBuf tmp;
  double* dst = out;
  if (where == MJP_PTR_HOST) {
    if ((rc = tmp.ensure(bytes))) return rc;
    dst = tmp.as<double>();
  }
  SD d = s->view();
  gather_trace_kernel<<<blocks_for((int64_t)s->C * kept, 256), 256, 0, st>>>(d, kept, dst);
  MJP_CUDA(cudaGetLastError());
  if (where == MJP_PTR_HOST) {
    MJP_CUDA(cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, st));
    MJP_CUDA(cudaStreamSynchronize(st));
    tmp.release();
  }
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

int mjp_sampler_evals(mjp_sampler* s, const double** psi, const double** ll, int64_t* n) try {
  if (!s || !psi || !ll || !n) return fail(MJP_ERR_ARG, "NULL argument");
  *psi = s->evpsi.as<double>();
  *ll = s->evll.as<double>();
  *n = s->evn;
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

int mjp_sampler_checkpoint_size(mjp_sampler* s, size_t* bytes) try {
  if (!s || !bytes) return fail(MJP_ERR_ARG, "NULL argument");
  *bytes = ckpt_bytes(s);
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

int mjp_sampler_save(mjp_sampler* s, void* buf, size_t bytes, void* stream) try {
  if (!s || !buf) return fail(MJP_ERR_ARG, "NULL argument");
  if (bytes < ckpt_bytes(s)) return fail(MJP_ERR_ARG, "checkpoint buffer smaller than mjp_sampler_checkpoint_size");
  cudaStream_t st = (cudaStream_t)stream;
  CkptHeader h = {};
  h.magic = kCkptMagic;
  h.version = kCkptVersion;
  h.chains = s->C;
  h.cap = s->cap;
  h.evcap = s->evcap;
  h.seed = s->seed;
  h.evn = s->evn;
  h.rounds = s->rounds;
  h.kept_base = s->kept_base;
  h.np = NP;
  h.ncnt = NCNT;
  h.nbest = NBEST;
  unsigned char* out = static_cast<unsigned char*>(buf);
  std::memcpy(out, &h, sizeof h);
  size_t off = sizeof h;
  cudaError_t e = cudaSuccess;
  ckpt_parts(s, [&](DevBuf& b, size_t n) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(out + off, b.p, n, cudaMemcpyDeviceToHost, st);
    off += n;
  });
  MJP_CUDA(e);
  MJP_CUDA(cudaStreamSynchronize(st));
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

int mjp_sampler_load(mjp_sampler* s, const void* buf, size_t bytes, void* stream) try {
  if (!s || !buf) return fail(MJP_ERR_ARG, "NULL argument");
  if (bytes < sizeof(CkptHeader)) return fail(MJP_ERR_ARG, "checkpoint too short");
  CkptHeader h;
  std::memcpy(&h, buf, sizeof h);
  if (h.magic != kCkptMagic || h.version != kCkptVersion || h.np != NP || h.ncnt != NCNT || h.nbest != NBEST)
    return fail(MJP_ERR_ARG, "not a sampler checkpoint of this library version");
  if (h.chains != s->C || h.cap != s->cap || h.evcap != s->evcap || h.seed != s->seed)
    return fail(MJP_ERR_ARG, "checkpoint of a sampler with other chains, capacities or seed");
  if (bytes < ckpt_bytes(s)) return fail(MJP_ERR_ARG, "checkpoint truncated");
  if (h.evn < 0 || h.evn > s->evcap || h.rounds < 0 || h.kept_base < 0)
    return fail(MJP_ERR_ARG, "checkpoint counters out of range");
  cudaStream_t st = (cudaStream_t)stream;
  const unsigned char* in = static_cast<const unsigned char*>(buf);
  size_t off = sizeof h;
  cudaError_t e = cudaSuccess;
  ckpt_parts(s, [&](DevBuf& b, size_t n) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.p, in + off, n, cudaMemcpyHostToDevice, st);
    off += n;
  });
  MJP_CUDA(e);
  MJP_CUDA(cudaStreamSynchronize(st));
  s->evn = h.evn;
  s->rounds = h.rounds;
  s->kept_base = h.kept_base;
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

int mjp_sampler_adapt(mjp_sampler* s, const mjp_adapt_cfg* cfg, mjp_adapt_report* rep, void* stream) try {
  if (!s || !cfg) return fail(MJP_ERR_ARG, "NULL argument");
  if (cfg->cycle < 1 || cfg->every < cfg->cycle || cfg->every % cfg->cycle != 0)
    return fail(MJP_ERR_ARG, "every must be a positive multiple of cycle");
  if (cfg->window < 2 || cfg->window > cfg->every || cfg->window > s->cap)
    return fail(MJP_ERR_ARG, "window must be in [2, min(every, capacity)]");
  if (cfg->good_cycles < 1 || cfg->max_iters < cfg->cycle) return fail(MJP_ERR_ARG, "bad cycle counts");
  if (!(cfg->z0 > 0.0) || !(cfg->eps >= 0.0) || !(cfg->acc_lo <= cfg->acc_hi))
    return fail(MJP_ERR_ARG, "bad z0, eps or acceptance range");
  cudaStream_t st = (cudaStream_t)stream;
  mjp_adapt_report r = {};
  r.converged = 1;
  const int phases = cfg->restart_at_best ? 2 : 1;
  for (int ph = 0; ph < phases; ++ph) {
    double Z[16] = {};
    for (int a = 0; a < NP; ++a) Z[a * 4 + a] = cfg->z0;
    int rc = set_cov_device(s, Z, st);
    if (rc) return rc;
    if ((rc = mjp_sampler_clear(s, 0, st))) return rc;
    int64_t iters = 0, good = 0;
    std::vector<int64_t> cnt;
    while (good < cfg->good_cycles && iters < cfg->max_iters) {
      if ((rc = read_counts(s, st, cnt, nullptr))) return rc;
      const int64_t acc0 = sum_count(cnt, CNT_ACC);
      if ((rc = mjp_sampler_run_plain(s, cfg->cycle, 1, st))) return rc;
      if ((rc = read_counts(s, st, cnt, nullptr))) return rc;
      const double acc = (double)(sum_count(cnt, CNT_ACC) - acc0) / ((double)s->C * (double)cfg->cycle);
      r.acc_last = acc;
      if (acc >= cfg->acc_lo && acc <= cfg->acc_hi) ++good;
      iters += cfg->cycle;
      if (iters % cfg->every == 0 && good < cfg->good_cycles) {
        rc = mjp_sampler_adapt_cov(s, cfg->window, cfg->eps, st);
        if (rc && rc != MJP_ERR_NUMERIC) return rc;  // a degenerate window keeps the old Z
      }
    }
    r.iters[ph] = iters;
    r.good[ph] = good;
    if (good < cfg->good_cycles) r.converged = 0;
    if (ph + 1 < phases) {  // restart every chain at the best posterior state seen
      std::vector<double> best((size_t)s->C * NBEST);
      MJP_CUDA(cudaMemcpyAsync(best.data(), s->best.p, best.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
      MJP_CUDA(cudaStreamSynchronize(st));
      int bc = 0;
      for (int c = 1; c < s->C; ++c)
        if (best[(size_t)c * NBEST] > best[(size_t)bc * NBEST]) bc = c;
      std::vector<double> psi0((size_t)s->C * NP);
      for (int c = 0; c < s->C; ++c)
        for (int a = 0; a < NP; ++a) psi0[(size_t)c * NP + a] = best[(size_t)bc * NBEST + 1 + a];
      if ((rc = mjp_sampler_set_state(s, psi0.data(), MJP_PTR_HOST, st))) return rc;
    }
  }
  if (rep) *rep = r;
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

int mjp_ess(const double* trace, int64_t chains, int64_t len, int params, double* ess, double* mean, double* var,
            double* mcse_mean, double* mcse_var, int where, void* stream) try {
  if (!trace) return fail(MJP_ERR_ARG, "NULL trace");
  if (chains < 1 || len < 4 || params < 1 || params > 1024) return fail(MJP_ERR_ARG, "bad trace shape");
  if (chains * (int64_t)params > (int64_t)1 << 30) return fail(MJP_ERR_ARG, "trace too large");
  if (where != MJP_PTR_HOST && where != MJP_PTR_DEVICE) return fail(MJP_ERR_ARG, "bad where");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t n = (size_t)chains * len * params;
  DevBuf dtr, mom, ce, cev, res;
  int rc = 0;
  const double* dt = trace;
  if (where == MJP_PTR_HOST) {
    if ((rc = dtr.ensure(n * sizeof(double)))) return rc;
    MJP_CUDA(cudaMemcpyAsync(dtr.p, trace, n * sizeof(double), cudaMemcpyHostToDevice, st));
    dt = dtr.as<double>();
  }
  if ((rc = mom.ensure(3 * params * sizeof(double))) || (rc = ce.ensure(chains * params * sizeof(double))) ||
      (rc = cev.ensure(chains * params * sizeof(double))) || (rc = res.ensure(5 * params * sizeof(double))))
    return rc;
  pooled_moments_kernel<<<params, 256, 0, st>>>(dt, chains, len, params, mom.as<double>());
  MJP_CUDA(cudaGetLastError());
  const size_t stage = (size_t)len * sizeof(double);
  const int staged = stage <= 200 * 1024 ? 1 : 0;
  const size_t smem = staged ? stage : 0;
  MJP_CUDA(cudaFuncSetAttribute(chain_ess_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const unsigned nblk = (unsigned)(chains * params);
  chain_ess_kernel<<<nblk, 256, smem, st>>>(dt, len, params, 0, mom.as<double>(), staged, ce.as<double>());
  MJP_CUDA(cudaGetLastError());
  chain_ess_kernel<<<nblk, 256, smem, st>>>(dt, len, params, 1, mom.as<double>(), staged, cev.as<double>());
  MJP_CUDA(cudaGetLastError());
  ess_final_kernel<<<1, 1024, 0, st>>>(ce.as<double>(), cev.as<double>(), mom.as<double>(), chains, params,
                                       res.as<double>());
  MJP_CUDA(cudaGetLastError());
  std::vector<double> h(5 * (size_t)params);
  MJP_CUDA(cudaMemcpyAsync(h.data(), res.p, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  MJP_CUDA(cudaStreamSynchronize(st));
  double* outs[5] = {ess, mean, var, mcse_mean, mcse_var};
  for (int q = 0; q < 5; ++q) {
    if (!outs[q]) continue;
    MJP_CUDA(cudaMemcpy(outs[q], h.data() + (size_t)q * params, params * sizeof(double),
                        where == MJP_PTR_HOST ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice));
  }
  dtr.release();
  mom.release();
  ce.release();
  cev.release();
  res.release();
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

}  // extern "C"
