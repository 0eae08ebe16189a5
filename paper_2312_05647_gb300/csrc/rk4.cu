// rk4.cu -- fourth-order Runge-Kutta for birth-death models (Method #4 of the
// paper, Sec. 2.3: Eqs. RKstep and RKintermediate), FP64, the comparison
// method beside R-MJP.
//
// One CTA evolves one distribution; thread t holds R consecutive states in
// registers (rho, the stage input x and the partial sum of the deltas).  A
// stage y = x A (Eq. A_def, matrix-free from theta) needs the neighbours of
// a thread's run, which travel through shared memory (the first and last
// state of every thread, double-buffered by stage parity, a zero slot at the
// box ends): one CTA barrier per stage, four per step.  The times are visited
// in ascending order; each interval between consecutive times is split into
// the host-computed number of equal steps (h <= 1 / max_n |a_nn|).
//
// The operations per state follow the oracle's order exactly (inflow from
// n-1, then from n+1, then minus the exit; the deltas summed as
// ((d1 + 2 d2) + 2 d3) + d4, divided by 6), with explicit unfused roundings,
// so the GPU result equals the oracle's to the bit.
#include "chain_common.cuh"
#include "internal.cuh"

namespace mjp {

namespace {

template <int R, int kMaxT>
__global__ void __launch_bounds__(kMaxT, 1) rk4_bd1d_kernel(const Rk4Params p) {
  extern __shared__ __align__(16) unsigned char smem[];
  double* const E = reinterpret_cast<double*>(smem);  // [parity][first, last][nthr + 1]
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int ES = nthr + 1;
  const int N = p.N;
  const double beta = p.theta[0], gamma = p.theta[1];
  const double* rho0 = p.rho0;

  // Coefficients of the held states: inflow gamma (n+1) from n+1 and the exit
  // rate e_n summed in the rate matrix's row order (death, then birth);
  // states beyond the box hold zero and have zero coefficients.
  double r[R], x[R], acc[R], dn[R], ex[R];
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int n = tid * R + j;
    const bool in = n < N;
    double e = 0.0;
    if (in && n >= 1) e = __dadd_rn(e, __dmul_rn(gamma, (double)n));
    if (in && n + 1 < N) e = __dadd_rn(e, beta);
    ex[j] = e;
    dn[j] = (in && n + 1 < N) ? __dmul_rn(gamma, (double)(n + 1)) : 0.0;
    r[j] = in ? rho0[n] : 0.0;
    x[j] = 0.0;
    acc[j] = 0.0;
  }
  const double bin = beta;  // inflow from n-1 (x_{-1} is the zero slot)
  if (tid < 4) E[tid * ES + nthr] = 0.0;
  const int iL = tid > 0 ? tid - 1 : nthr;
  const int iR = tid + 1 < nthr ? tid + 1 : nthr;

  // y = v A for the thread's run, v's edges published at parity par.
  auto apply = [&](const double (&v)[R], double (&y)[R], int par) {
    E[(par * 2 + 0) * ES + tid] = v[0];
    E[(par * 2 + 1) * ES + tid] = v[R - 1];
    __syncthreads();
    const double vl = E[(par * 2 + 1) * ES + iL];
    const double vr = E[(par * 2 + 0) * ES + iR];
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const double left = j > 0 ? v[j - 1] : vl;
      const double right = j + 1 < R ? v[j + 1] : vr;
      double t = __dmul_rn(left, bin);
      t = __dadd_rn(t, __dmul_rn(right, dn[j]));
      y[j] = __dsub_rn(t, __dmul_rn(v[j], ex[j]));
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
  const size_t smem = sizeof(double) * 4 * (size_t)(threads + 1);
  rk4_bd1d_kernel<R, kMaxT><<<1, threads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

int64_t rk4_max_states() { return 8 * 512; }

cudaError_t launch_rk4_bd1d(const Rk4Params& p, cudaStream_t s) {
  if (p.N < 1 || p.N > rk4_max_states()) return cudaErrorInvalidValue;
  if (p.N <= 1024) return launch_rk4_typed<1, 1024>(p, s);
  return launch_rk4_typed<8, 512>(p, s);
}

}  // namespace mjp
