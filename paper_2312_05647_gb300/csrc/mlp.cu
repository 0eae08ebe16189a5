// mlp.cu -- the log-likelihood surrogate of include/mjp_surrogate.h: a
// 4 -> 128 -> 128 -> 1 tanh perceptron evaluated and trained (mean squared
// error, Adam of Kingma & Ba 2015) by hand-written FP32 kernels.
//
// Work split: one CTA of 128 threads takes a tile of R rows; thread j owns
// hidden unit j.  W2 (64 KB) sits in shared memory with a padded stride so
// that both the forward pass (column j) and the backward pass (row i) read
// it without bank conflicts; the hidden activations of the tile are
// broadcast from shared memory as float4.  The backward pass writes one
// gradient partial per CTA; a second kernel sums the partials in CTA order
// (FP64) and applies Adam, so every result is run-to-run identical.  The
// network is tiny (17,281 parameters, 34 kflop per row forward): a step is
// latency-bound, and FP32 FMA on the CUDA cores keeps the gradients exact
// enough to check against FP64 backpropagation.
#include <cmath>
#include <cstring>
#include <vector>

#include "host_util.h"
#include "mjp_surrogate.h"
#include "mlp_dev.cuh"
#include "philox.cuh"

using namespace mjp;
using namespace mjp::mlp;

struct mjp_mlp {
  DevBuf P, m, v, norm;
  DevBuf partial, loss_part, psi, y, out, losses, grad, scalar;
  int64_t t = 0;
};

namespace {

__global__ void init_kernel(float* __restrict__ P, uint32_t k0, uint32_t k1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPAR) return;
  double a = 0.0;
  if (i < OB1) a = sqrt(6.0 / (D + H));
  else if (i >= OW2 && i < OB2) a = sqrt(6.0 / (H + H));
  else if (i >= OW3 && i < OB3) a = sqrt(6.0 / (H + 1));
  float v = 0.f;
  if (a > 0.0) {
    const uint4 w = philox4x32_10(make_uint4((uint32_t)i, 0u, kInitStream, 0u), k0, k1);
    v = (float)((2.0 * uniform52(w.x, w.y) - 1.0) * a);
  }
  P[i] = v;
}

// Deterministic block sum (FP64): butterfly within warps, then warp 0 over
// the warp partials in warp order.  All threads get the result.
__device__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < nw; ++w) s += red[w];
  return s;
}

// Means and population standard deviations of the 4 input columns and y.
__global__ void __launch_bounds__(256) fit_norm_kernel(const double* __restrict__ psi, const double* __restrict__ y,
                                                        int64_t n, Norm* __restrict__ out) {
  __shared__ double red[8];
  double mean[5], sd[5];
  for (int c = 0; c < 5; ++c) {
    double s = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) s += c < 4 ? psi[r * 4 + c] : y[r];
    mean[c] = block_sum(s, red) / (double)n;
  }
  for (int c = 0; c < 5; ++c) {
    double s = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
      const double d = (c < 4 ? psi[r * 4 + c] : y[r]) - mean[c];
      s += d * d;
    }
    const double v = block_sum(s, red) / (double)n;
    sd[c] = v > 0.0 ? sqrt(v) : 1.0;
  }
  if (threadIdx.x == 0) {
    Norm nm;
    for (int c = 0; c < 4; ++c) {
      nm.mux[c] = mean[c];
      nm.sdx[c] = sd[c];
    }
    nm.muy = mean[4];
    nm.sdy = sd[4];
    *out = nm;
  }
}

struct RowsParams {
  const float* P;
  const Norm* nm;
  const double* psi;
  const double* y;
  int64_t n;      // rows of the data set
  int64_t batch;  // rows evaluated (tile rows beyond it are padding)
  int sample;     // 1: row r is a Philox draw from the data set, else row r itself
  uint32_t k0, k1, step;
  float inv_batch;
  double* out;        // forward: s(psi) per row
  float* partial;     // backward: [gridDim.x][NPAR] gradient partials
  double* loss_part;  // backward: sum of squared residuals per CTA
};

template <int R>
constexpr size_t rows_smem(bool grad) {
  return sizeof(float) * ((size_t)H * W2S + (size_t)R * H * (grad ? 2 : 1) + R * 4 + R + 4 * R + R);
}

template <int R, bool GRAD>
__global__ void __launch_bounds__(128) rows_kernel(const RowsParams p) {
  extern __shared__ __align__(16) float sm[];
  float* W2s = sm;
  float* h1s = W2s + H * W2S;
  float* dz2s = h1s + R * H;
  float* xs = dz2s + (GRAD ? R * H : 0);
  float* ts = xs + R * 4;
  float* red = ts + R;
  float* dys = red + 4 * R;
  const int j = threadIdx.x, lane = j & 31, warp = j >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * R;
  const Norm nm = *p.nm;

  stage_w2(p.P, W2s);
  if (j < R) {
    const int64_t g = r0 + j;
    const bool valid = g < p.batch;
    int64_t src = g;
    if (valid && p.sample) {
      const uint4 w = philox4x32_10(make_uint4((uint32_t)g, p.step, kBatchStream, 0u), p.k0, p.k1);
      src = (int64_t)(((uint64_t)w.x * (uint64_t)p.n) >> 32);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) xs[j * 4 + k] = valid ? std_input(nm, p.psi + src * 4, k) : 0.f;
    if (GRAD) ts[j] = valid ? (float)((p.y[src] - nm.muy) / nm.sdy) : 0.f;
  }
  float w1[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) w1[k] = p.P[OW1 + k * H + j];
  const float b1 = p.P[OB1 + j], b2 = p.P[OB2 + j], w3 = p.P[OW3 + j], b3 = p.P[OB3];
  __syncthreads();

  // Layer 1 -> h1 (shared), layer 2 -> a[r] = h2 (registers, unit j).
#pragma unroll 4
  for (int r = 0; r < R; ++r) {
    const float x[4] = {xs[r * 4], xs[r * 4 + 1], xs[r * 4 + 2], xs[r * 4 + 3]};
    h1s[r * H + j] = tanhf(layer1(x, w1, b1));
  }
  __syncthreads();
  float a[R];
#pragma unroll
  for (int r = 0; r < R; ++r) a[r] = b2;
  for (int i = 0; i < H; i += 4) {
    const float wa = W2s[i * W2S + j], wb = W2s[(i + 1) * W2S + j];
    const float wc = W2s[(i + 2) * W2S + j], wd = W2s[(i + 3) * W2S + j];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float4 h = *reinterpret_cast<const float4*>(h1s + r * H + i);
      a[r] = fmaf(h.x, wa, a[r]);
      a[r] = fmaf(h.y, wb, a[r]);
      a[r] = fmaf(h.z, wc, a[r]);
      a[r] = fmaf(h.w, wd, a[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    a[r] = tanhf(a[r]);
    const float v = warp_sum(a[r] * w3);
    if (lane == 0) red[warp * R + r] = v;
  }
  __syncthreads();

  if (!GRAD) {
    if (j < R && r0 + j < p.batch) {
      const float f = b3 + red[j] + red[R + j] + red[2 * R + j] + red[3 * R + j];
      p.out[r0 + j] = nm.muy + nm.sdy * (double)f;
    }
    return;
  }

  // dL/df per row and the tile's squared residuals (warp 0: R <= 32 rows).
  if (warp == 0) {
    double l = 0.0;
    if (lane < R) {
      const bool valid = r0 + lane < p.batch;
      const float f = b3 + red[lane] + red[R + lane] + red[2 * R + lane] + red[3 * R + lane];
      const float res = f - ts[lane];
      dys[lane] = valid ? 2.f * res * p.inv_batch : 0.f;
      l = valid ? (double)res * (double)res : 0.0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if (lane == 0) p.loss_part[blockIdx.x] = l;
  }
  __syncthreads();

  float* out = p.partial + (size_t)blockIdx.x * NPAR;
  float gw3 = 0.f, gb2 = 0.f, gb3 = 0.f;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const float dy = dys[r];
    gw3 = fmaf(dy, a[r], gw3);
    gb3 += dy;
    const float dz = dy * w3 * (1.f - a[r] * a[r]);
    a[r] = dz;  // a[] now holds dL/dz2[r][j]
    gb2 += dz;
    dz2s[r * H + j] = dz;
  }
  out[OW3 + j] = gw3;
  out[OB2 + j] = gb2;
  if (j == 0) out[OB3] = gb3;
  // dL/dW2[i][j] = sum_r h1[r][i] dz2[r][j]
  for (int i = 0; i < H; i += 4) {
    float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float4 h = *reinterpret_cast<const float4*>(h1s + r * H + i);
      g0 = fmaf(h.x, a[r], g0);
      g1 = fmaf(h.y, a[r], g1);
      g2 = fmaf(h.z, a[r], g2);
      g3 = fmaf(h.w, a[r], g3);
    }
    out[OW2 + i * H + j] = g0;
    out[OW2 + (i + 1) * H + j] = g1;
    out[OW2 + (i + 2) * H + j] = g2;
    out[OW2 + (i + 3) * H + j] = g3;
  }
  __syncthreads();
  // dL/dh1[r][i] = sum_c dz2[r][c] W2[i][c] for i = j, then through tanh.
  float d[R];
#pragma unroll
  for (int r = 0; r < R; ++r) d[r] = 0.f;
  for (int c = 0; c < H; c += 4) {
    const float wa = W2s[j * W2S + c], wb = W2s[j * W2S + c + 1];
    const float wc = W2s[j * W2S + c + 2], wd = W2s[j * W2S + c + 3];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float4 z = *reinterpret_cast<const float4*>(dz2s + r * H + c);
      d[r] = fmaf(z.x, wa, d[r]);
      d[r] = fmaf(z.y, wb, d[r]);
      d[r] = fmaf(z.z, wc, d[r]);
      d[r] = fmaf(z.w, wd, d[r]);
    }
  }
  float gb1 = 0.f, gw1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const float h = h1s[r * H + j];
    const float dz1 = d[r] * (1.f - h * h);
    gb1 += dz1;
#pragma unroll
    for (int k = 0; k < 4; ++k) gw1[k] = fmaf(xs[r * 4 + k], dz1, gw1[k]);
  }
  out[OB1 + j] = gb1;
#pragma unroll
  for (int k = 0; k < 4; ++k) out[OW1 + k * H + j] = gw1[k];
}

struct AdamParams {
  const float* partial;
  int nblk;
  const double* loss_part;
  double inv_batch;
  float* P;
  float* m;
  float* v;
  float lr, b1, b2, eps, bc1, bc2;
  int apply;      // 1: Adam update, 0: write the gradient only
  float* grad;    // may be null when apply
  double* loss;   // may be null
};

// Gradient = sum of the CTA partials in CTA order (FP64), then Adam.
__global__ void __launch_bounds__(256) reduce_adam_kernel(const AdamParams q) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < NPAR) {
    double g = 0.0;
    for (int b = 0; b < q.nblk; ++b) g += (double)q.partial[(size_t)b * NPAR + p];
    const float gf = (float)g;
    if (q.grad) q.grad[p] = gf;
    if (q.apply) {
      const float m = q.b1 * q.m[p] + (1.f - q.b1) * gf;
      const float v = q.b2 * q.v[p] + (1.f - q.b2) * gf * gf;
      q.m[p] = m;
      q.v[p] = v;
      q.P[p] -= q.lr * (m / q.bc1) / (sqrtf(v / q.bc2) + q.eps);
    }
  }
  if (p == 0 && q.loss) {
    double L = 0.0;
    for (int b = 0; b < q.nblk; ++b) L += q.loss_part[b];
    *q.loss = L * q.inv_batch;
  }
}

template <int R, bool GRAD>
cudaError_t launch_rows(const RowsParams& p, int64_t rows, cudaStream_t s) {
  const size_t smem = rows_smem<R>(GRAD);
  cudaError_t e = cudaFuncSetAttribute(rows_kernel<R, GRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  rows_kernel<R, GRAD><<<(unsigned)((rows + R - 1) / R), 128, smem, s>>>(p);
  return cudaGetLastError();
}

int rows_per_cta(int64_t rows) { return rows <= 512 ? 8 : (rows <= 4096 ? 16 : 32); }

cudaError_t launch_grad(const RowsParams& p, int64_t rows, cudaStream_t s) {
  switch (rows_per_cta(rows)) {
    case 8: return launch_rows<8, true>(p, rows, s);
    case 16: return launch_rows<16, true>(p, rows, s);
    default: return launch_rows<32, true>(p, rows, s);
  }
}

bool all_finite(const float* v, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return false;
  return true;
}

int check_where(int where) {
  if (where != MJP_PTR_HOST && where != MJP_PTR_DEVICE)
    return fail(MJP_ERR_ARG, "where must be MJP_PTR_HOST or MJP_PTR_DEVICE");
  return MJP_OK;
}

// Device copies of the data set (host inputs are uploaded into net scratch).
int stage_data(mjp_mlp* net, const double* psi, const double* y, int64_t n, int where, cudaStream_t s,
               const double** dpsi, const double** dy) {
  *dpsi = psi;
  *dy = y;
  if (where == MJP_PTR_DEVICE) return MJP_OK;
  int rc;
  if ((rc = net->psi.ensure(sizeof(double) * 4 * (size_t)n))) return rc;
  MJP_CUDA(cudaMemcpyAsync(net->psi.p, psi, sizeof(double) * 4 * (size_t)n, cudaMemcpyHostToDevice, s));
  *dpsi = net->psi.as<double>();
  if (y) {
    if ((rc = net->y.ensure(sizeof(double) * (size_t)n))) return rc;
    MJP_CUDA(cudaMemcpyAsync(net->y.p, y, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, s));
    *dy = net->y.as<double>();
  }
  return MJP_OK;
}

}  // namespace

// Used by the sampler: device parameter vector and standardisation.
namespace mjp {
const float* mlp_params(const mjp_mlp* net) { return net->P.as<float>(); }
const void* mlp_norm(const mjp_mlp* net) { return net->norm.p; }
}  // namespace mjp

extern "C" {

int mjp_mlp_create(mjp_mlp** out, uint64_t seed) try {
  if (!out) return fail(MJP_ERR_ARG, "NULL out");
  *out = nullptr;
  mjp_mlp* net = new mjp_mlp();
  int rc;
  if ((rc = net->P.ensure(sizeof(float) * NPAR)) || (rc = net->m.ensure(sizeof(float) * NPAR)) ||
      (rc = net->v.ensure(sizeof(float) * NPAR)) || (rc = net->norm.ensure(sizeof(Norm)))) {
    mjp_mlp_destroy(net);
    return rc;
  }
  init_kernel<<<(NPAR + 255) / 256, 256>>>(net->P.as<float>(), (uint32_t)seed, (uint32_t)(seed >> 32));
  Norm id;
  for (int k = 0; k < 4; ++k) {
    id.mux[k] = 0.0;
    id.sdx[k] = 1.0;
  }
  id.muy = 0.0;
  id.sdy = 1.0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemset(net->m.p, 0, sizeof(float) * NPAR);
  if (e == cudaSuccess) e = cudaMemset(net->v.p, 0, sizeof(float) * NPAR);
  if (e == cudaSuccess) e = cudaMemcpy(net->norm.p, &id, sizeof(Norm), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaGetLastError();
    mjp_mlp_destroy(net);
    return fail(MJP_ERR_CUDA, std::string("mjp_mlp_create: ") + cudaGetErrorString(e));
  }
  *out = net;
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

void mjp_mlp_destroy(mjp_mlp* net) {
  if (!net) return;
  cudaDeviceSynchronize();
  for (DevBuf* b : {&net->P, &net->m, &net->v, &net->norm, &net->partial, &net->loss_part, &net->psi, &net->y,
                    &net->out, &net->losses, &net->grad, &net->scalar})
    b->release();
  delete net;
}

int mjp_mlp_set_params(mjp_mlp* net, const float* params, const double* norm, int where, void* stream) try {
  if (!net) return fail(MJP_ERR_ARG, "NULL network");
  int rc = check_where(where);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<float> hp;
  Norm nm;
  if (params) {
    hp.resize(NPAR);
    MJP_CUDA(cudaMemcpyAsync(hp.data(), params, sizeof(float) * NPAR,
                             where == MJP_PTR_HOST ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost, s));
  }
  if (norm)
    MJP_CUDA(cudaMemcpyAsync(&nm, norm, sizeof(Norm),
                             where == MJP_PTR_HOST ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost, s));
  MJP_CUDA(cudaStreamSynchronize(s));
  if (params && !all_finite(hp.data(), NPAR)) return fail(MJP_ERR_ARG, "parameters must be finite");
  if (norm) {
    const double* v = reinterpret_cast<const double*>(&nm);
    for (int i = 0; i < MJP_MLP_NNORM; ++i)
      if (!std::isfinite(v[i])) return fail(MJP_ERR_ARG, "standardisation must be finite");
    for (int k = 0; k < 4; ++k)
      if (!(nm.sdx[k] > 0.0)) return fail(MJP_ERR_ARG, "input deviations must be > 0");
    if (!(nm.sdy > 0.0)) return fail(MJP_ERR_ARG, "output deviation must be > 0");
  }
  if (params) MJP_CUDA(cudaMemcpyAsync(net->P.p, hp.data(), sizeof(float) * NPAR, cudaMemcpyHostToDevice, s));
  if (norm) MJP_CUDA(cudaMemcpyAsync(net->norm.p, &nm, sizeof(Norm), cudaMemcpyHostToDevice, s));
  MJP_CUDA(cudaMemsetAsync(net->m.p, 0, sizeof(float) * NPAR, s));
  MJP_CUDA(cudaMemsetAsync(net->v.p, 0, sizeof(float) * NPAR, s));
  net->t = 0;
  MJP_CUDA(cudaStreamSynchronize(s));
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

int mjp_mlp_get_params(mjp_mlp* net, float* params, double* norm, int where, void* stream) try {
  if (!net) return fail(MJP_ERR_ARG, "NULL network");
  int rc = check_where(where);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const cudaMemcpyKind k = where == MJP_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  if (params) MJP_CUDA(cudaMemcpyAsync(params, net->P.p, sizeof(float) * NPAR, k, s));
  if (norm) MJP_CUDA(cudaMemcpyAsync(norm, net->norm.p, sizeof(Norm), k, s));
  if (where == MJP_PTR_HOST) MJP_CUDA(cudaStreamSynchronize(s));
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

int mjp_mlp_fit_norm(mjp_mlp* net, const double* psi, const double* y, int64_t n, int where, void* stream) try {
  if (!net || !psi || !y) return fail(MJP_ERR_ARG, "NULL argument");
  if (n < 1) return fail(MJP_ERR_ARG, "n must be >= 1");
  int rc = check_where(where);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const double *dpsi, *dy;
  if ((rc = stage_data(net, psi, y, n, where, s, &dpsi, &dy))) return rc;
  fit_norm_kernel<<<1, 256, 0, s>>>(dpsi, dy, n, net->norm.as<Norm>());
  MJP_CUDA(cudaGetLastError());
  if (where == MJP_PTR_HOST) MJP_CUDA(cudaStreamSynchronize(s));
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

int mjp_mlp_forward(mjp_mlp* net, const double* psi, int64_t n, double* out, int where, void* stream) try {
  if (!net || !psi || !out) return fail(MJP_ERR_ARG, "NULL argument");
  if (n < 1) return fail(MJP_ERR_ARG, "n must be >= 1");
  int rc = check_where(where);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const double *dpsi, *dy;
  if ((rc = stage_data(net, psi, nullptr, n, where, s, &dpsi, &dy))) return rc;
  double* dout = out;
  if (where == MJP_PTR_HOST) {
    if ((rc = net->out.ensure(sizeof(double) * (size_t)n))) return rc;
    dout = net->out.as<double>();
  }
  RowsParams p = {};
  p.P = net->P.as<float>();
  p.nm = net->norm.as<Norm>();
  p.psi = dpsi;
  p.n = n;
  p.batch = n;
  p.out = dout;
  MJP_CUDA((launch_rows<32, false>(p, n, s)));
  if (where == MJP_PTR_HOST) {
    MJP_CUDA(cudaMemcpyAsync(out, dout, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, s));
    MJP_CUDA(cudaStreamSynchronize(s));
  }
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

int mjp_mlp_loss_grad(mjp_mlp* net, const double* psi, const double* y, int64_t n, double* loss, float* grad,
                      int where, void* stream) try {
  if (!net || !psi || !y) return fail(MJP_ERR_ARG, "NULL argument");
  if (n < 1 || n > 0xFFFFFFFFLL) return fail(MJP_ERR_ARG, "n must be in [1, 2^32)");
  int rc = check_where(where);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const double *dpsi, *dy;
  if ((rc = stage_data(net, psi, y, n, where, s, &dpsi, &dy))) return rc;
  const int R = rows_per_cta(n);
  const int nblk = (int)((n + R - 1) / R);
  if ((rc = net->partial.ensure(sizeof(float) * NPAR * (size_t)nblk))) return rc;
  if ((rc = net->loss_part.ensure(sizeof(double) * (size_t)nblk))) return rc;
  if ((rc = net->grad.ensure(sizeof(float) * NPAR))) return rc;
  if ((rc = net->scalar.ensure(sizeof(double)))) return rc;
  RowsParams p = {};
  p.P = net->P.as<float>();
  p.nm = net->norm.as<Norm>();
  p.psi = dpsi;
  p.y = dy;
  p.n = n;
  p.batch = n;
  p.inv_batch = (float)(1.0 / (double)n);
  p.partial = net->partial.as<float>();
  p.loss_part = net->loss_part.as<double>();
  MJP_CUDA(launch_grad(p, n, s));
  AdamParams q = {};
  q.partial = p.partial;
  q.nblk = nblk;
  q.loss_part = p.loss_part;
  q.inv_batch = 1.0 / (double)n;
  q.apply = 0;
  q.grad = (grad && where == MJP_PTR_DEVICE) ? grad : net->grad.as<float>();
  q.loss = (loss && where == MJP_PTR_DEVICE) ? loss : net->scalar.as<double>();
  reduce_adam_kernel<<<(NPAR + 255) / 256, 256, 0, s>>>(q);
  MJP_CUDA(cudaGetLastError());
  if (where == MJP_PTR_HOST) {
    if (grad) MJP_CUDA(cudaMemcpyAsync(grad, q.grad, sizeof(float) * NPAR, cudaMemcpyDeviceToHost, s));
    if (loss) MJP_CUDA(cudaMemcpyAsync(loss, q.loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    MJP_CUDA(cudaStreamSynchronize(s));
  }
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

int mjp_mlp_train(mjp_mlp* net, const double* psi, const double* y, int64_t n, const mjp_train_cfg* cfg,
                  double* losses, int where, void* stream) try {
  if (!net || !psi || !y || !cfg) return fail(MJP_ERR_ARG, "NULL argument");
  if (n < 1 || n > 0xFFFFFFFFLL) return fail(MJP_ERR_ARG, "n must be in [1, 2^32)");
  if (cfg->steps < 1 || cfg->steps > 0xFFFFFFFFLL) return fail(MJP_ERR_ARG, "steps must be in [1, 2^32)");
  if (cfg->batch < 1) return fail(MJP_ERR_ARG, "batch must be >= 1");
  if (!(cfg->lr > 0.0) || !std::isfinite(cfg->lr)) return fail(MJP_ERR_ARG, "lr must be > 0");
  if (!(cfg->beta1 >= 0.0 && cfg->beta1 < 1.0) || !(cfg->beta2 >= 0.0 && cfg->beta2 < 1.0))
    return fail(MJP_ERR_ARG, "beta1 and beta2 must be in [0, 1)");
  if (!(cfg->eps > 0.0) || !std::isfinite(cfg->eps)) return fail(MJP_ERR_ARG, "eps must be > 0");
  int rc = check_where(where);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const double *dpsi, *dy;
  if ((rc = stage_data(net, psi, y, n, where, s, &dpsi, &dy))) return rc;
  if (cfg->fit_norm) {
    fit_norm_kernel<<<1, 256, 0, s>>>(dpsi, dy, n, net->norm.as<Norm>());
    MJP_CUDA(cudaGetLastError());
  }
  const int64_t rows = cfg->batch < n ? cfg->batch : n;
  const int R = rows_per_cta(rows);
  const int nblk = (int)((rows + R - 1) / R);
  if ((rc = net->partial.ensure(sizeof(float) * NPAR * (size_t)nblk))) return rc;
  if ((rc = net->loss_part.ensure(sizeof(double) * (size_t)nblk))) return rc;
  double* dl = losses;
  if (losses && where == MJP_PTR_HOST) {
    if ((rc = net->losses.ensure(sizeof(double) * (size_t)cfg->steps))) return rc;
    dl = net->losses.as<double>();
  }
  RowsParams p = {};
  p.P = net->P.as<float>();
  p.nm = net->norm.as<Norm>();
  p.psi = dpsi;
  p.y = dy;
  p.n = n;
  p.batch = rows;
  p.sample = cfg->batch < n;
  p.k0 = (uint32_t)cfg->seed;
  p.k1 = (uint32_t)(cfg->seed >> 32);
  p.inv_batch = (float)(1.0 / (double)rows);
  p.partial = net->partial.as<float>();
  p.loss_part = net->loss_part.as<double>();
  AdamParams q = {};
  q.partial = p.partial;
  q.nblk = nblk;
  q.loss_part = p.loss_part;
  q.inv_batch = 1.0 / (double)rows;
  q.P = net->P.as<float>();
  q.m = net->m.as<float>();
  q.v = net->v.as<float>();
  q.lr = (float)cfg->lr;
  q.b1 = (float)cfg->beta1;
  q.b2 = (float)cfg->beta2;
  q.eps = (float)cfg->eps;
  q.apply = 1;
  for (int64_t st = 0; st < cfg->steps; ++st) {
    p.step = (uint32_t)st;
    MJP_CUDA(launch_grad(p, rows, s));
    const int64_t t = ++net->t;
    q.bc1 = (float)(1.0 - std::pow(cfg->beta1, (double)t));
    q.bc2 = (float)(1.0 - std::pow(cfg->beta2, (double)t));
    q.loss = dl ? dl + st : nullptr;
    reduce_adam_kernel<<<(NPAR + 255) / 256, 256, 0, s>>>(q);
    MJP_CUDA(cudaGetLastError());
  }
  if (where == MJP_PTR_HOST) {
    if (losses)
      MJP_CUDA(cudaMemcpyAsync(losses, dl, sizeof(double) * (size_t)cfg->steps, cudaMemcpyDeviceToHost, s));
    MJP_CUDA(cudaStreamSynchronize(s));
  }
  return MJP_OK;
} catch (...) {
  return ::mjp::exception_status();
}

}  // extern "C"
