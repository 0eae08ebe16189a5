// rk4.cu -- fourth-order Runge-Kutta for birth-death and two-state models
// (Method #4 of the paper, Sec. 2.3: Eqs. RKstep and RKintermediate), FP64,
// the comparison method beside R-MJP.
//
// One CTA evolves one distribution; thread t holds R consecutive states in
// registers (rho, the stage input x and the partial sum of the deltas).  A
// stage y = x A (Eq. A_def, matrix-free from theta) reads the neighbours and
// the two-state partner from the stage input staged whole in shared memory
// (double-buffered by stage parity): one CTA barrier per stage, four per step.  The times are visited
// in ascending order; each interval between consecutive times is split into
// the host-computed number of equal steps (h <= 1 / max_n |a_nn|).
//
// The operations per state follow the oracle's order exactly (inflows in
// ascending source order, then minus the exit; the deltas summed as
// ((d1 + 2 d2) + 2 d3) + d4, divided by 6), with explicit unfused roundings,
// so the GPU result equals the oracle's to the bit.
#include "chain_common.cuh"
#include "internal.cuh"

namespace mjp {

namespace {

template <int R, int kMaxT>
__global__ void __launch_bounds__(kMaxT, 1) rk4_kernel(const Rk4Params p) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* const X = reinterpret_cast<double*>(smem);  // [parity][N]: the stage input
  const int tid = threadIdx.x;
  const int N = p.N;
  const double* rho0 = p.rho0;

  // Rates of the held states (states beyond the box hold zero).
  double r[R], x[R], acc[R];
  double dn[R], ex[R];
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int n = tid * R + j;
    rate_row_coef(p.kind, n, N, p.M, p.theta, dn[j], ex[j]);
    r[j] = n < N ? rho0[n] : 0.0;
    x[j] = 0.0;
    acc[j] = 0.0;
  }

  // y = v A for the thread's run; v staged whole at parity par (the
  // two-state partner lies N_R states away).
  auto apply = [&](const double (&v)[R], double (&y)[R], int par) {
    double* const Xp = X + (size_t)par * N;
#pragma unroll
    for (int j = 0; j < R; ++j)
      if (tid * R + j < N) Xp[tid * R + j] = v[j];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int n = tid * R + j;
      y[j] = n < N ? rate_apply_row(p.kind, n, N, p.M, p.theta, dn[j], ex[j], Xp, v[j]) : 0.0;
    }
  };

  int par = 0;
  for (int q = 0; q < p.ntimes; ++q) {
    const int64_t ns = p.steps[q];
    const double h = p.hstep[q];
    for (int64_t k = 0; k < ns; ++k) {
      double y[R];
      apply(r, y, par);
      par ^= 1;
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const double d = __dmul_rn(h, y[j]);
        acc[j] = d;
        x[j] = __dadd_rn(r[j], __ddiv_rn(d, 2.0));
      }
      apply(x, y, par);
      par ^= 1;
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const double d = __dmul_rn(h, y[j]);
        acc[j] = __dadd_rn(acc[j], __dmul_rn(2.0, d));
        x[j] = __dadd_rn(r[j], __ddiv_rn(d, 2.0));
      }
      apply(x, y, par);
      par ^= 1;
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const double d = __dmul_rn(h, y[j]);
        acc[j] = __dadd_rn(acc[j], __dmul_rn(2.0, d));
        x[j] = __dadd_rn(r[j], d);
      }
      apply(x, y, par);
      par ^= 1;
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const double d = __dmul_rn(h, y[j]);
        r[j] = __dadd_rn(r[j], __ddiv_rn(__dadd_rn(acc[j], d), 6.0));
      }
    }
    double* o = p.out + (int64_t)p.orig[q] * N;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int n = tid * R + j;
      if (n < N) o[n] = r[j];
    }
  }
}

template <int R, int kMaxT>
cudaError_t launch_rk4_typed(const Rk4Params& p, cudaStream_t s) {
  const int threads = (int)(((p.N + R - 1) / R + 31) / 32 * 32);
  const size_t smem = sizeof(double) * 2 * (size_t)p.N;
  auto kern = rk4_kernel<R, kMaxT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<1, threads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

int64_t rk4_max_states() { return 8 * 512; }

cudaError_t launch_rk4(const Rk4Params& p, cudaStream_t s) {
  if (p.N < 1 || p.N > rk4_max_states() || (p.kind != MJP_BD1D && p.kind != MJP_TWOSTATE)) return cudaErrorInvalidValue;
  if (p.N <= 1024) return launch_rk4_typed<1, 1024>(p, s);
  return launch_rk4_typed<8, 512>(p, s);
}

}  // namespace mjp
