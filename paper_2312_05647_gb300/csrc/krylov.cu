// krylov.cu -- Krylov subspace steps for birth-death models (Method #5 of the
// paper, Sec. 2.3: Algorithm 3 with the full projection of Eq.
// Krylov_projection, Eq. Krylov_expansion), FP64, a comparison method beside
// R-MJP.
//
// One CTA evolves one distribution.  Thread t holds R consecutive states of
// rho and of the vector being orthogonalised in registers; the orthonormal
// basis Q (kappa x N) lives in a global scratch buffer (L2-resident), each
// thread reading back only the states it wrote.  Per step: beta = ||rho||,
// q_1 = rho / beta; for i = 1..kappa: w = q_i A (matrix-free, run ends through
// shared memory), modified Gram-Schmidt against q_1..q_i with CTA-wide
// reductions in a fixed order, h_(i+1)i = ||w||, q_(i+1) = w / h_(i+1)i; then
// exp(dt H) by Pade-13 scaling and squaring (Higham 2005) on the CTA, and
// rho = beta Q exp(dt H) e_1.  A subdiagonal entry <= 1e-14 max_n |a_nn| marks
// an invariant space: the step uses the vectors found so far.
#include <math.h>

#include "chain_common.cuh"
#include "internal.cuh"

namespace mjp {

namespace {

constexpr int kKmax = 32;  // largest subspace

// Sum of v over the CTA in a fixed order (warp butterflies, then warp 0 over
// the warp sums); every thread receives the total.  red: 33 doubles.
__device__ __forceinline__ double cta_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(kFull, v, o));
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double t = lane < nw ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = __dadd_rn(t, __shfl_xor_sync(kFull, t, o));
    if (lane == 0) red[32] = t;
  }
  __syncthreads();
  return red[32];
}

// C = A B for m x m row-major matrices in shared memory, one element per
// thread (callers separate the steps with barriers).
__device__ void mat_mul(int m, const double* A, const double* B, double* C) {
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int r = e / m, c = e - r * m;
    double s = 0.0;
    for (int k = 0; k < m; ++k) s = __fma_rn(A[r * m + k], B[k * m + c], s);
    C[e] = s;
  }
}

// E = exp(A) for an m x m matrix in shared memory (m <= kKmax): scaling and
// squaring with the [13/13] Pade approximant (N. J. Higham, SIAM J. Matrix
// Anal. Appl. 26 (2005) 1179; theta_13 from its Table 2.3).  W: 9 m x m work
// matrices.  Returns nonzero if the Pade denominator is singular.
__device__ int cta_expm(int m, const double* A, double* E, double* W, int* flag) {
  const int mm = m * m;
  double *As = W, *A2 = W + mm, *A4 = W + 2 * mm, *A6 = W + 3 * mm, *T1 = W + 4 * mm, *T2 = W + 5 * mm,
         *U = W + 6 * mm, *V = W + 7 * mm, *P = W + 8 * mm;
  __shared__ double b[14];
  __shared__ int s_sc;
  if (threadIdx.x == 0) {
    // b_0 = 1, b_(j+1) = b_j (13 - j) / ((26 - j)(j + 1)): the numerator
    // coefficients (2m-j)! m! / ((2m)! j! (m-j)!) of the [m/m] approximant.
    b[0] = 1.0;
    for (int j = 0; j < 13; ++j) b[j + 1] = b[j] * (double)(13 - j) / ((double)(26 - j) * (double)(j + 1));
    double norm1 = 0.0;
    for (int c = 0; c < m; ++c) {
      double s = 0.0;
      for (int r = 0; r < m; ++r) s += fabs(A[r * m + c]);
      norm1 = fmax(norm1, s);
    }
    const double theta13 = 5.371920351148152;
    s_sc = norm1 > theta13 ? (int)ceil(log2(norm1 / theta13)) : 0;
    *flag = 0;
  }
  __syncthreads();
  const int sc = s_sc;
  const double f = ldexp(1.0, -sc);
  for (int e = threadIdx.x; e < mm; e += blockDim.x) As[e] = A[e] * f;
  __syncthreads();
  mat_mul(m, As, As, A2);
  __syncthreads();
  mat_mul(m, A2, A2, A4);
  __syncthreads();
  mat_mul(m, A4, A2, A6);
  __syncthreads();
  // U = As [A6 (b13 A6 + b11 A4 + b9 A2) + b7 A6 + b5 A4 + b3 A2 + b1 I]
  // V =      A6 (b12 A6 + b10 A4 + b8 A2) + b6 A6 + b4 A4 + b2 A2 + b0 I
  for (int e = threadIdx.x; e < mm; e += blockDim.x) {
    T1[e] = b[13] * A6[e] + b[11] * A4[e] + b[9] * A2[e];
    T2[e] = b[12] * A6[e] + b[10] * A4[e] + b[8] * A2[e];
  }
  __syncthreads();
  mat_mul(m, A6, T1, P);
  mat_mul(m, A6, T2, V);
  __syncthreads();
  for (int e = threadIdx.x; e < mm; e += blockDim.x) {
    const bool diag = (e / m) == (e % m);
    P[e] += b[7] * A6[e] + b[5] * A4[e] + b[3] * A2[e] + (diag ? b[1] : 0.0);
    V[e] += b[6] * A6[e] + b[4] * A4[e] + b[2] * A2[e] + (diag ? b[0] : 0.0);
  }
  __syncthreads();
  mat_mul(m, As, P, U);
  __syncthreads();
  // (V - U) X = (V + U): Gaussian elimination with partial pivoting, the
  // m right-hand sides eliminated alongside.
  double* L = T1;   // V - U
  double* Rh = T2;  // V + U
  for (int e = threadIdx.x; e < mm; e += blockDim.x) {
    L[e] = V[e] - U[e];
    Rh[e] = V[e] + U[e];
  }
  __syncthreads();
  __shared__ int s_piv;
  for (int c = 0; c < m; ++c) {
    if (threadIdx.x == 0) {
      int pv = c;
      for (int r = c + 1; r < m; ++r)
        if (fabs(L[r * m + c]) > fabs(L[pv * m + c])) pv = r;
      s_piv = pv;
      if (L[pv * m + c] == 0.0) *flag = 1;
    }
    __syncthreads();
    const int pv = s_piv;
    if (pv != c)
      for (int j = threadIdx.x; j < m; j += blockDim.x) {
        double t = L[c * m + j];
        L[c * m + j] = L[pv * m + j];
        L[pv * m + j] = t;
        t = Rh[c * m + j];
        Rh[c * m + j] = Rh[pv * m + j];
        Rh[pv * m + j] = t;
      }
    __syncthreads();
    if (*flag) return 1;
    const double d = L[c * m + c];
    // Rows below c: multipliers first (column c is read before it is
    // overwritten), then the updates.
    for (int e = threadIdx.x; e < (m - c - 1) * m; e += blockDim.x) {
      const int r = c + 1 + e / m, j = e % m;
      const double l = L[r * m + c] / d;
      if (j > c) L[r * m + j] -= l * L[c * m + j];
      Rh[r * m + j] -= l * Rh[c * m + j];
    }
    __syncthreads();
    for (int r = c + 1 + threadIdx.x; r < m; r += blockDim.x) L[r * m + c] = 0.0;
    __syncthreads();
  }
  // Back substitution, one right-hand side per thread.
  for (int j = threadIdx.x; j < m; j += blockDim.x)
    for (int r = m - 1; r >= 0; --r) {
      double s = Rh[r * m + j];
      for (int c = r + 1; c < m; ++c) s -= L[r * m + c] * E[c * m + j];
      E[r * m + j] = s / L[r * m + r];
    }
  __syncthreads();
  for (int q = 0; q < sc; ++q) {
    mat_mul(m, E, E, P);
    __syncthreads();
    for (int e = threadIdx.x; e < mm; e += blockDim.x) E[e] = P[e];
    __syncthreads();
  }
  return 0;
}

template <int R, int kMaxT>
__global__ void __launch_bounds__(kMaxT, 1) krylov_kernel(const KrylovParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int N = p.N, K = p.kappa;
  double* X = reinterpret_cast<double*>(smem);        // [parity][N]: the vector being multiplied
  double* red = X + 2 * (size_t)N;                     // 33
  double* H = red + 33;                                // kKmax x kKmax
  double* Hm = H + kKmax * kKmax;                      // m x m
  double* Ex = Hm + kKmax * kKmax;                     // m x m
  double* W = Ex + kKmax * kKmax;                      // 9 m x m
  __shared__ int s_flag;
  const double maxe = p.maxe;

  // Rates of each held state (Eq. A_def, the rate matrix's row order); zero
  // beyond the box.
  double r[R], w[R];
  double dn[R], ex[R];
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int n = tid * R + j;
    rate_row_coef(p.kind, n, N, p.M, p.theta, dn[j], ex[j]);
    r[j] = n < N ? p.rho0[n] : 0.0;
    w[j] = 0.0;
  }
  double* const Qb = p.Q;  // [K][N]
  auto qrow = [&](int i) { return Qb + (int64_t)i * N; };

  int par = 0;
  // y = v A for the thread's run; v staged whole at parity par (the
  // two-state partner lies N_R states away).
  auto apply = [&](const double (&v)[R], double (&y)[R]) {
    double* const Xp = X + (size_t)par * N;
#pragma unroll
    for (int j = 0; j < R; ++j)
      if (tid * R + j < N) Xp[tid * R + j] = v[j];
    __syncthreads();
    par ^= 1;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int n = tid * R + j;
      // States beyond the box stay zero (they enter the norms and products).
      y[j] = n < N ? rate_apply_row(p.kind, n, N, p.M, p.theta, dn[j], ex[j], Xp, v[j]) : 0.0;
    }
  };

  for (int q = 0; q < p.ntimes; ++q) {
    const int64_t ns = p.steps[q];
    const double dt = p.hstep[q];
    for (int64_t step = 0; step < ns; ++step) {
      double part = 0.0;
#pragma unroll
      for (int j = 0; j < R; ++j) part = __fma_rn(r[j], r[j], part);
      const double beta = __dsqrt_rn(cta_sum(part, red));
      if (beta == 0.0) break;
      double qc[R];
#pragma unroll
      for (int j = 0; j < R; ++j) {
        qc[j] = __ddiv_rn(r[j], beta);
        if (tid * R + j < N) qrow(0)[tid * R + j] = qc[j];
      }
      int m = K;
      for (int i = 0; i < K; ++i) {
        apply(qc, w);
        for (int jj = 0; jj <= i; ++jj) {
          const double* qj = qrow(jj);
          double pd = 0.0;
#pragma unroll
          for (int j = 0; j < R; ++j) {
            const double qv = tid * R + j < N ? qj[tid * R + j] : 0.0;
            pd = __fma_rn(qv, w[j], pd);
          }
          const double h = cta_sum(pd, red);
          if (tid == 0) H[jj * kKmax + i] = h;
#pragma unroll
          for (int j = 0; j < R; ++j) {
            const double qv = tid * R + j < N ? qj[tid * R + j] : 0.0;
            w[j] = __fma_rn(-h, qv, w[j]);
          }
        }
        if (i + 1 < K) {
          double pn = 0.0;
#pragma unroll
          for (int j = 0; j < R; ++j) pn = __fma_rn(w[j], w[j], pn);
          const double hn = __dsqrt_rn(cta_sum(pn, red));
          if (hn <= 1e-14 * maxe) {
            m = i + 1;
            break;
          }
          if (tid == 0) H[(i + 1) * kKmax + i] = hn;
#pragma unroll
          for (int j = 0; j < R; ++j) {
            qc[j] = __ddiv_rn(w[j], hn);
            if (tid * R + j < N) qrow(i + 1)[tid * R + j] = qc[j];
          }
        }
      }
      __syncthreads();
      // dt H (upper Hessenberg: entries below the subdiagonal are zero; they
      // were not written this step).
      for (int e = tid; e < m * m; e += nthr) {
        const int a = e / m, c = e - a * m;
        Hm[e] = a <= c + 1 ? __dmul_rn(dt, H[a * kKmax + c]) : 0.0;
      }
      __syncthreads();
      if (cta_expm(m, Hm, Ex, W, &s_flag)) {
        if (tid == 0) set_status(p.status, kStatusNumeric);
        return;
      }
      // rho = beta Q exp(dt H) e_1 (each thread its own states of Q).
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int n = tid * R + j;
        double v = 0.0;
        if (n < N)
          for (int i = 0; i < m; ++i) v = __fma_rn(qrow(i)[n], Ex[i * m], v);
        r[j] = __dmul_rn(beta, v);
      }
      __syncthreads();
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
cudaError_t launch_krylov_typed(const KrylovParams& p, cudaStream_t s) {
  const int threads = (int)(((p.N + R - 1) / R + 31) / 32 * 32);
  const size_t smem = sizeof(double) * (2 * (size_t)p.N + 33 + 12 * (size_t)kKmax * kKmax);
  auto kern = krylov_kernel<R, kMaxT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<1, threads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace

int krylov_max_states() { return 8 * 512; }
int krylov_max_kappa() { return kKmax; }

cudaError_t launch_krylov(const KrylovParams& p, cudaStream_t s) {
  if (p.N < 1 || p.N > krylov_max_states() || p.kappa < 1 || p.kappa > kKmax ||
      (p.kind != MJP_BD1D && p.kind != MJP_TWOSTATE))
    return cudaErrorInvalidValue;
  if (p.N <= 512) return launch_krylov_typed<1, 512>(p, s);
  return launch_krylov_typed<8, 512>(p, s);
}

}  // namespace mjp
