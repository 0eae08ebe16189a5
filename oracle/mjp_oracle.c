/*
 * mjp_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct CPU reference for the R-MJP transient
 * distribution of Pessoa, Schweiger & Presse, "Avoiding matrix exponentials
 * for large transition rate matrices" (arXiv 2312.05647).  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no source, header, table or helper with the CUDA library; the two
 * meet only in the seeded input generators.
 *
 * Arithmetic is IEEE FP64 throughout, except the Poisson weights, which are
 * formed in long double log space (80-bit on x86-64, 128-bit on AArch64)
 * because exp(-x) underflows FP64 for x > 708 (the paper's Algorithm 2 starts
 * its recurrence at exp(-Omega t) and would silently return zeros there).
 * Build with -ffp-contract=off: no multiply-add may be fused, so that the
 * truncation index K is computed with exactly two roundings (Algorithm 2).
 *
 * Parity status: every routine below is pinned by the CPU test suite against
 * closed forms, an independent library routine or brute force; see
 * tests/test_oracle_pins.py.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_ALLOC (-3)

/* Model kinds (the same numbers the public header uses, restated here). */
#define ORC_BD1D 1        /* birth-death, Eq. BD_def (Sec. 3.1.1)            */
#define ORC_TWOSTATE 2    /* two-state birth-death, Eq. Gene_def (Sec. 3.1.2)*/
#define ORC_MRNA_PROT2D 3 /* mRNA/protein birth-death, built from Eq.       */
#define ORC_AUTOREG 5     /* autoregulatory gene network, Eq. STS_chem /
                             Eq. autoReg_def (Sec. 3.1.3)                    */
                          /* STS_chem's R->R+P reaction without switching    */

/* ------------------------------------------------------------------------ */
/* Rate matrices Lambda as CSR, rows = source state n, off-diagonal lambda_nm */
/* (Sec. 2.1: lambda_nn = 0).  Columns of each row are ascending.            */
/* ------------------------------------------------------------------------ */

static int64_t push(int64_t* row_ptr, int32_t* col, double* val, int64_t nnz,
                    int64_t cap, int64_t m, double rate) {
  (void)row_ptr;
  if (col != NULL) {
    if (nnz >= cap) return -1;
    col[nnz] = (int32_t)m;
    val[nnz] = rate;
  }
  return nnz + 1;
}

/*
 * Fill (row_ptr, col, val) for model `kind`; return nnz, or a negative error.
 * With col == NULL only nnz is counted.
 *
 * BD1D (dims = {N}, theta = {beta, gamma}), Eq. BD_def:
 *   lambda_{n,n+1} = beta, lambda_{n,n-1} = gamma*n.  The state space is cut
 *   at N (Sec. 3.1.1); a birth out of n = N-1 is dropped (reflecting top), so
 *   rows of A still sum to zero.
 * TWOSTATE (dims = {N_R}, theta = {beta, gamma, lambda_act, lambda_ina}),
 *   Eq. Gene_def with index n = n_R + sigma*N_R, sigma = 0 active, 1 inactive
 *   (Sec. 3.1.2): active states produce at beta (dropped at n_R = N_R-1),
 *   every state degrades at gamma*n_R, active->inactive at lambda_ina and
 *   inactive->active at lambda_act (the reaction scheme Eq. 2S_chem and the
 *   text of Sec. 3.1.2; the case labels of Eq. Gene_def are read accordingly).
 * MRNA_PROT2D (dims = {M, P}, theta = {k_m, gamma_m, k_p, gamma_p}), index
 *   n = m + M*p as in Sec. 3.1.3: m->m+1 at k_m, m->m-1 at gamma_m*m,
 *   p->p+1 at k_p*m, p->p-1 at gamma_p*p; births out of the box are dropped.
 */
int64_t orc_build_model(int kind, const int64_t* dims, int ndims,
                        const double* theta, int ntheta, int64_t* row_ptr,
                        int32_t* col, double* val, int64_t cap) {
  int64_t nnz = 0;
  if (kind == ORC_BD1D) {
    if (ndims != 1 || ntheta != 2 || dims[0] < 1) return ORC_ERR_ARG;
    int64_t N = dims[0];
    double beta = theta[0], gamma = theta[1];
    for (int64_t n = 0; n < N; ++n) {
      if (row_ptr) row_ptr[n] = nnz;
      if (n >= 1) nnz = push(row_ptr, col, val, nnz, cap, n - 1, gamma * (double)n);
      if (n + 1 < N) nnz = push(row_ptr, col, val, nnz, cap, n + 1, beta);
      if (nnz < 0) return ORC_ERR_ARG;
    }
    if (row_ptr) row_ptr[N] = nnz;
    return nnz;
  }
  if (kind == ORC_TWOSTATE) {
    if (ndims != 1 || ntheta != 4 || dims[0] < 2) return ORC_ERR_ARG;
    int64_t NR = dims[0];
    double beta = theta[0], gamma = theta[1], lact = theta[2], lina = theta[3];
    for (int64_t sg = 0; sg < 2; ++sg) {
      for (int64_t nr = 0; nr < NR; ++nr) {
        int64_t n = nr + sg * NR;
        if (row_ptr) row_ptr[n] = nnz;
        if (sg == 0) {
          if (nr >= 1) nnz = push(row_ptr, col, val, nnz, cap, n - 1, gamma * (double)nr);
          if (nr + 1 < NR) nnz = push(row_ptr, col, val, nnz, cap, n + 1, beta);
          nnz = push(row_ptr, col, val, nnz, cap, n + NR, lina);
        } else {
          nnz = push(row_ptr, col, val, nnz, cap, n - NR, lact);
          if (nr >= 1) nnz = push(row_ptr, col, val, nnz, cap, n - 1, gamma * (double)nr);
        }
        if (nnz < 0) return ORC_ERR_ARG;
      }
    }
    if (row_ptr) row_ptr[2 * NR] = nnz;
    return nnz;
  }
  if (kind == ORC_MRNA_PROT2D) {
    if (ndims != 2 || ntheta != 4 || dims[0] < 2 || dims[1] < 1) return ORC_ERR_ARG;
    int64_t M = dims[0], P = dims[1];
    double km = theta[0], gm = theta[1], kp = theta[2], gp = theta[3];
    for (int64_t p = 0; p < P; ++p) {
      for (int64_t m = 0; m < M; ++m) {
        int64_t n = m + M * p;
        if (row_ptr) row_ptr[n] = nnz;
        if (p >= 1) nnz = push(row_ptr, col, val, nnz, cap, n - M, gp * (double)p);
        if (m >= 1) nnz = push(row_ptr, col, val, nnz, cap, n - 1, gm * (double)m);
        if (m + 1 < M) nnz = push(row_ptr, col, val, nnz, cap, n + 1, km);
        if (p + 1 < P && m >= 1) nnz = push(row_ptr, col, val, nnz, cap, n + M, kp * (double)m);
        if (nnz < 0) return ORC_ERR_ARG;
      }
    }
    if (row_ptr) row_ptr[M * P] = nnz;
    return nnz;
  }
  if (kind == ORC_AUTOREG) {
    /*
     * dims = {N_R, N_P}, theta = {beta_R, beta_P, gamma_R, gamma_P, lambda_act,
     * lambda_ina}; n = n_R + N_R n_P + N_R N_P sigma (sigma 0 active), N =
     * 2 N_R N_P.  The reactions of Eq. STS_chem: transcription beta_R (active
     * only), translation beta_P n_R (either gene state), R decay gamma_R n_R,
     * P decay gamma_P n_P, binding sigma_act + P -> sigma_ina at lambda_ina n_P,
     * unbinding sigma_ina -> sigma_act + P at lambda_act; a transition whose
     * target leaves the box is dropped (reflecting).  Entries in ascending
     * target order.
     */
    if (ndims != 2 || ntheta != 6 || dims[0] < 2 || dims[1] < 2) return ORC_ERR_ARG;
    int64_t M = dims[0], P = dims[1];
    double bR = theta[0], bP = theta[1], gR = theta[2], gP = theta[3], la = theta[4], li = theta[5];
    for (int64_t sg = 0; sg < 2; ++sg)
      for (int64_t p = 0; p < P; ++p)
        for (int64_t m = 0; m < M; ++m) {
          int64_t n = m + M * p + M * P * sg;
          if (row_ptr) row_ptr[n] = nnz;
          if (sg == 1 && p + 1 < P) nnz = push(row_ptr, col, val, nnz, cap, n - M * P + M, la);
          if (p >= 1) nnz = push(row_ptr, col, val, nnz, cap, n - M, gP * (double)p);
          if (m >= 1) nnz = push(row_ptr, col, val, nnz, cap, n - 1, gR * (double)m);
          if (sg == 0 && m + 1 < M) nnz = push(row_ptr, col, val, nnz, cap, n + 1, bR);
          if (p + 1 < P && m >= 1) nnz = push(row_ptr, col, val, nnz, cap, n + M, bP * (double)m);
          if (sg == 0 && p >= 1) nnz = push(row_ptr, col, val, nnz, cap, n + M * P - M, li * (double)p);
          if (nnz < 0) return ORC_ERR_ARG;
        }
    if (row_ptr) row_ptr[2 * M * P] = nnz;
    return nnz;
  }
  return ORC_ERR_ARG;
}

/* Largest exit rate max_n sum_m lambda_nm = max_n |a_nn| (Eq. A_def), each
 * row summed in stored (ascending column) order. */
double orc_max_exit(int64_t n, const int64_t* row_ptr, const double* val) {
  double best = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    double e = 0.0;
    for (int64_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j) e = e + val[j];
    if (e > best) best = e;
  }
  return best;
}

/* ------------------------------------------------------------------------ */
/* Truncation index and Poisson weights (Sec. 2.2.3, Algorithm 2).          */
/* ------------------------------------------------------------------------ */

/* Algorithm 2 loops while k <= x + 6 sqrt(x), incrementing k first, so the
 * last jump index reached is K = floor(x + 6 sqrt(x)) + 1, x = Omega t. */
int64_t orc_K_paper(double x) {
  double s = sqrt(x);
  double six_s = 6.0 * s;
  double y = x + six_s;
  return (int64_t)floor(y) + 1;
}

static long double log_pois(long double x, int64_t k) {
  /* log Poisson(k | x), Eq. ME_uniform, in long double. */
  return -x + (long double)k * logl(x) - lgammal((long double)k + 1.0L);
}

/*
 * P[k] = Poisson(k | x) for k = 0..K (Eq. ME_uniform), and *eps = 1 - sum P
 * = epsilon_{k*} of Eq. R-MJP_expansion.  The sum uses Kahan compensation in
 * long double.  x = 0 gives the point mass at k = 0.
 */
int orc_poisson_weights(double x, int64_t K, double* P, double* eps) {
  if (!(x >= 0.0) || K < 0) return ORC_ERR_ARG;
  long double s = 0.0L, c = 0.0L;
  for (int64_t k = 0; k <= K; ++k) {
    long double p;
    if (x == 0.0) p = (k == 0) ? 1.0L : 0.0L;
    else p = expl(log_pois((long double)x, k));
    P[k] = (double)p;
    long double y = p - c;
    long double t = s + y;
    c = (t - s) - y;
    s = t;
  }
  *eps = (double)(1.0L - s);
  return ORC_OK;
}

/* Smallest K with 1 - sum_{k<=K} Poisson(k|x) <= tol (the "tolerance"
 * truncation used by tight closed-form tests; not the paper's rule). */
int64_t orc_K_tol(double x, double tol) {
  if (!(x >= 0.0) || !(tol > 0.0)) return -1;
  if (x == 0.0) return 0;
  long double s = 0.0L, c = 0.0L;
  for (int64_t k = 0;; ++k) {
    long double p = expl(log_pois((long double)x, k));
    long double y = p - c;
    long double t = s + y;
    c = (t - s) - y;
    s = t;
    if (1.0L - s <= (long double)tol) return k;
    if (k > (int64_t)1e9) return -1;
  }
}

/* ------------------------------------------------------------------------ */
/* R-MJP series (Eq. R-MJP_expansion, Algorithm 2) at several times.        */
/* ------------------------------------------------------------------------ */

/*
 * out[i*n + s] = rho*(t_i)_s for i < ntimes, where
 *   rho*(t) = sum_{k=0}^{K} rho0 B^k P_k + (1 - sum_{k=0}^{K} P_k) rho0 B^K,
 *   B = I + A/Omega (Eq. B_def), Omega = omega_factor * max_n |a_nn|
 *   (the paper takes omega_factor = 1.1), P_k = Poisson(k | Omega t),
 *   K = orc_K_paper(Omega t) (mode 0) or orc_K_tol(Omega t, tol) (mode 1).
 * One chain rho0 B^k serves all times; each time gets exactly Algorithm 2
 * with its own K_i and tail.  rho B is formed row by row (scatter form).
 * If every rate is zero, A = 0 and rho(t) = rho0.
 * omega_out/K_out/eps_out (nullable) receive Omega, K_i and epsilon_i.
 */
int orc_expv(int64_t n, const int64_t* row_ptr, const int32_t* col,
             const double* val, const double* rho0, const double* times,
             int ntimes, int mode, double tol, double omega_factor,
             double* out, double* omega_out, int64_t* K_out, double* eps_out) {
  if (n < 1 || ntimes < 0 || !(omega_factor > 1.0)) return ORC_ERR_ARG;
  for (int i = 0; i < ntimes; ++i)
    if (!(times[i] >= 0.0) || isinf(times[i])) return ORC_ERR_ARG;
  double maxe = orc_max_exit(n, row_ptr, val);
  if (maxe == 0.0) {
    for (int i = 0; i < ntimes; ++i) {
      memcpy(out + (size_t)i * n, rho0, sizeof(double) * (size_t)n);
      if (K_out) K_out[i] = 0;
      if (eps_out) eps_out[i] = 0.0;
    }
    if (omega_out) *omega_out = 0.0;
    return ORC_OK;
  }
  double omega = omega_factor * maxe;
  if (omega_out) *omega_out = omega;

  int64_t* K = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ntimes > 0 ? ntimes : 1));
  double** P = (double**)calloc((size_t)(ntimes > 0 ? ntimes : 1), sizeof(double*));
  double* tail = (double*)malloc(sizeof(double) * (size_t)(ntimes > 0 ? ntimes : 1));
  double* bdiag = (double*)malloc(sizeof(double) * (size_t)n);
  double* boff = (double*)malloc(sizeof(double) * (size_t)(row_ptr[n] > 0 ? row_ptr[n] : 1));
  double* rho = (double*)malloc(sizeof(double) * (size_t)n);
  double* nxt = (double*)malloc(sizeof(double) * (size_t)n);
  int rc = ORC_OK;
  if (!K || !P || !tail || !bdiag || !boff || !rho || !nxt) { rc = ORC_ERR_ALLOC; goto done; }

  /* B = I + A/Omega: b_nn = 1 - e_n/Omega, b_nm = lambda_nm/Omega. */
  for (int64_t s = 0; s < n; ++s) {
    double e = 0.0;
    for (int64_t j = row_ptr[s]; j < row_ptr[s + 1]; ++j) {
      e = e + val[j];
      boff[j] = val[j] / omega;
    }
    bdiag[s] = 1.0 - e / omega;
  }

  int64_t Kmax = 0;
  for (int i = 0; i < ntimes; ++i) {
    double x = omega * times[i];
    K[i] = (mode == 0) ? orc_K_paper(x) : orc_K_tol(x, tol);
    if (K[i] < 0) { rc = ORC_ERR_ARG; goto done; }
    P[i] = (double*)malloc(sizeof(double) * (size_t)(K[i] + 1));
    if (!P[i]) { rc = ORC_ERR_ALLOC; goto done; }
    orc_poisson_weights(x, K[i], P[i], &tail[i]);
    if (K_out) K_out[i] = K[i];
    if (eps_out) eps_out[i] = tail[i];
    if (K[i] > Kmax) Kmax = K[i];
  }

  memcpy(rho, rho0, sizeof(double) * (size_t)n);
  for (int i = 0; i < ntimes; ++i)
    for (int64_t s = 0; s < n; ++s) out[(size_t)i * n + s] = P[i][0] * rho[s];

  for (int64_t k = 1; k <= Kmax; ++k) {
    /* rho <- rho B (Algorithm 2, loop body). */
    for (int64_t s = 0; s < n; ++s) nxt[s] = 0.0;
    for (int64_t s = 0; s < n; ++s) {
      double r = rho[s];
      nxt[s] += r * bdiag[s];
      for (int64_t j = row_ptr[s]; j < row_ptr[s + 1]; ++j) nxt[col[j]] += r * boff[j];
    }
    double* tmp = rho; rho = nxt; nxt = tmp;
    /* rho* += P_k rho for every time whose loop is still running. */
    for (int i = 0; i < ntimes; ++i) {
      if (k > K[i]) continue;
      double w = P[i][k];
      double* o = out + (size_t)i * n;
      if (w != 0.0)
        for (int64_t s = 0; s < n; ++s) o[s] += w * rho[s];
      if (k == K[i]) /* rho* += (1 - P_cumulative) rho, after the loop. */
        for (int64_t s = 0; s < n; ++s) o[s] += tail[i] * rho[s];
    }
  }
  /* A time with K_i = 0 (tolerance mode, t = 0) still needs its tail. */
  for (int i = 0; i < ntimes; ++i) {
    if (K[i] != 0) continue;
    double* o = out + (size_t)i * n;
    for (int64_t s = 0; s < n; ++s) o[s] += tail[i] * rho0[s];
  }

done:
  if (P) for (int i = 0; i < ntimes; ++i) free(P[i]);
  free(P); free(K); free(tail); free(bdiag); free(boff); free(rho); free(nxt);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* J-MJP state probabilities (Method #2, Sec. 2.2.2, Algorithm 1)           */
/* ------------------------------------------------------------------------ */

/*
 * phi[i] = sum_{s in group i} (rho0 B^{k_i})_s for observations i < nobs,
 * with B = I + A / Omega, Omega = omega_factor * max_n |a_nn| (Eq. B_def):
 * one chain rho0 B^k, read at every observation's own jump count k_i
 * (Algorithm 1's loop; a group sums a hidden component out, Sec. 3.1.2).
 * If every rate is zero, B = I.
 */
int orc_jmjp(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
             const double* rho0, int64_t nobs, const int64_t* k, const int64_t* group_ptr,
             const int32_t* members, double omega_factor, double* phi) {
  if (n < 1 || nobs < 0 || !(omega_factor > 1.0)) return ORC_ERR_ARG;
  int64_t kmax = 0;
  for (int64_t i = 0; i < nobs; ++i) {
    if (k[i] < 0) return ORC_ERR_ARG;
    if (k[i] > kmax) kmax = k[i];
  }
  const double maxe = orc_max_exit(n, row_ptr, val);
  const double omega = omega_factor * maxe;
  double* bdiag = (double*)malloc(sizeof(double) * (size_t)n);
  double* boff = (double*)malloc(sizeof(double) * (size_t)(row_ptr[n] > 0 ? row_ptr[n] : 1));
  double* rho = (double*)malloc(sizeof(double) * (size_t)n);
  double* nxt = (double*)malloc(sizeof(double) * (size_t)n);
  int rc = ORC_OK;
  if (!bdiag || !boff || !rho || !nxt) { rc = ORC_ERR_ALLOC; goto done; }
  for (int64_t s = 0; s < n; ++s) {
    double e = 0.0;
    for (int64_t j = row_ptr[s]; j < row_ptr[s + 1]; ++j) {
      e = e + val[j];
      boff[j] = maxe > 0.0 ? val[j] / omega : 0.0;
    }
    bdiag[s] = maxe > 0.0 ? 1.0 - e / omega : 1.0;
  }
  memcpy(rho, rho0, sizeof(double) * (size_t)n);
  for (int64_t kk = 0; kk <= kmax; ++kk) {
    for (int64_t i = 0; i < nobs; ++i) {
      if (k[i] != kk) continue;
      double v = 0.0;
      for (int64_t q = group_ptr[i]; q < group_ptr[i + 1]; ++q) v += rho[members[q]];
      phi[i] = v;
    }
    if (kk == kmax) break;
    for (int64_t s = 0; s < n; ++s) nxt[s] = 0.0;
    for (int64_t s = 0; s < n; ++s) {
      double r = rho[s];
      nxt[s] += r * bdiag[s];
      for (int64_t j = row_ptr[s]; j < row_ptr[s + 1]; ++j) nxt[col[j]] += r * boff[j];
    }
    double* tmp = rho; rho = nxt; nxt = tmp;
  }
done:
  free(bdiag); free(boff); free(rho); free(nxt);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Fourth-order Runge-Kutta (Method #4, Sec. 2.3: Eqs. RKstep, RKintermediate)*/
/* ------------------------------------------------------------------------ */

/* y = x A (Eq. A_def): the off-diagonal inflows scattered row by row (source
 * states ascending, each row in stored order), then the exits subtracted:
 * y_m = (sum_n x_n lambda_nm) - x_m e_m. */
static void rate_apply(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
                       const double* exitr, const double* x, double* y) {
  for (int64_t s = 0; s < n; ++s) y[s] = 0.0;
  for (int64_t s = 0; s < n; ++s)
    for (int64_t j = row_ptr[s]; j < row_ptr[s + 1]; ++j) y[col[j]] += x[s] * val[j];
  for (int64_t s = 0; s < n; ++s) y[s] = y[s] - x[s] * exitr[s];
}

/*
 * out[i*n + s] = rho(t_i)_s by RK4: the times are visited in ascending order
 * and each interval between consecutive times (from 0) is split into
 *   n_i = ceil((t_(i) - t_(i-1)) * max_n |a_nn|)
 * equal steps h, the stability condition h <= 1 / max_n |a_nn| of Sec. 2.3.
 * One step:  d1 = h rho A,  d2 = h (rho + d1/2) A,  d3 = h (rho + d2/2) A,
 *            d4 = h (rho + d3) A,  rho <- rho + (d1 + 2 d2 + 2 d3 + d4) / 6.
 * steps_out (nullable) receives the cumulative number of steps to each time,
 * maxe_out (nullable) max_n |a_nn|.  If every rate is zero, rho(t) = rho0.
 */
int orc_rk4(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
            const double* rho0, const double* times, int ntimes, double* out,
            int64_t* steps_out, double* maxe_out) {
  if (n < 1 || ntimes < 0) return ORC_ERR_ARG;
  for (int i = 0; i < ntimes; ++i)
    if (!(times[i] >= 0.0) || isinf(times[i])) return ORC_ERR_ARG;
  double maxe = orc_max_exit(n, row_ptr, val);
  if (maxe_out) *maxe_out = maxe;
  int* order = (int*)malloc(sizeof(int) * (size_t)(ntimes > 0 ? ntimes : 1));
  double* exitr = (double*)malloc(sizeof(double) * (size_t)n);
  double* rho = (double*)malloc(sizeof(double) * (size_t)n);
  double* x = (double*)malloc(sizeof(double) * (size_t)n);
  double* y = (double*)malloc(sizeof(double) * (size_t)n);
  double* d1 = (double*)malloc(sizeof(double) * (size_t)n);
  double* d2 = (double*)malloc(sizeof(double) * (size_t)n);
  double* d3 = (double*)malloc(sizeof(double) * (size_t)n);
  int rc = ORC_OK;
  if (!order || !exitr || !rho || !x || !y || !d1 || !d2 || !d3) { rc = ORC_ERR_ALLOC; goto done; }
  for (int64_t s = 0; s < n; ++s) {
    double e = 0.0;
    for (int64_t j = row_ptr[s]; j < row_ptr[s + 1]; ++j) e = e + val[j];
    exitr[s] = e;
  }
  /* Stable insertion sort of the time indices. */
  for (int i = 0; i < ntimes; ++i) {
    int j = i;
    while (j > 0 && times[order[j - 1]] > times[i]) { order[j] = order[j - 1]; --j; }
    order[j] = i;
  }
  memcpy(rho, rho0, sizeof(double) * (size_t)n);
  double tprev = 0.0;
  int64_t total = 0;
  for (int q = 0; q < ntimes; ++q) {
    const int i = order[q];
    const double tau = times[i] - tprev;
    const int64_t ns = (maxe > 0.0 && tau > 0.0) ? (int64_t)ceil(tau * maxe) : 0;
    const double h = ns > 0 ? tau / (double)ns : 0.0;
    for (int64_t k = 0; k < ns; ++k) {
      rate_apply(n, row_ptr, col, val, exitr, rho, y);
      for (int64_t s = 0; s < n; ++s) { d1[s] = h * y[s]; x[s] = rho[s] + d1[s] / 2.0; }
      rate_apply(n, row_ptr, col, val, exitr, x, y);
      for (int64_t s = 0; s < n; ++s) { d2[s] = h * y[s]; x[s] = rho[s] + d2[s] / 2.0; }
      rate_apply(n, row_ptr, col, val, exitr, x, y);
      for (int64_t s = 0; s < n; ++s) { d3[s] = h * y[s]; x[s] = rho[s] + d3[s]; }
      rate_apply(n, row_ptr, col, val, exitr, x, y);
      for (int64_t s = 0; s < n; ++s) {
        const double d4 = h * y[s];
        rho[s] = rho[s] + (d1[s] + 2.0 * d2[s] + 2.0 * d3[s] + d4) / 6.0;
      }
    }
    total += ns;
    memcpy(out + (size_t)i * n, rho, sizeof(double) * (size_t)n);
    if (steps_out) steps_out[i] = total;
    tprev = times[i];
  }
done:
  free(order); free(exitr); free(rho); free(x); free(y); free(d1); free(d2); free(d3);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Krylov subspace (Method #5, Sec. 2.3: Algorithm 3, Eqs. Krylov_projection,*/
/* Krylov_expansion)                                                        */
/* ------------------------------------------------------------------------ */

int orc_expm_pade13(int n, const double* A, double* E);

/*
 * out[i*n + s] = rho(t_i)_s by Krylov steps: the times are visited in
 * ascending order and each interval between consecutive times (from 0) is
 * split into n_i = ceil(interval * max_n |a_nn| / (2 kappa)) equal steps dt
 * (the paper's dt = 2 kappa / max_n |a_nn|).  One step from rho:
 *   beta = ||rho||_2,  q_1 = rho / beta;
 *   for i = 1..kappa:  w = q_i A;  for j = 1..i: h_ji = <q_j, w>, w -= h_ji q_j
 *                      (modified Gram-Schmidt, Algorithm 3's inner loop);
 *                      if i < kappa: h_(i+1)i = ||w||_2, q_(i+1) = w / h_(i+1)i;
 *   rho <- beta (Q exp(dt H))[:, 1]   (Eq. Krylov_expansion),
 * i.e. H = Q^T A^T Q of Eq. Krylov_projection with all kappa columns (the
 * printed algorithm stops one product short of the last column).  If
 * h_(i+1)i <= 1e-14 max_n |a_nn| the space is invariant: the step uses the
 * first i vectors.  steps_out / maxe_out as in orc_rk4.
 */
int orc_krylov(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* val,
               const double* rho0, const double* times, int ntimes, int kappa, double* out,
               int64_t* steps_out, double* maxe_out) {
  if (n < 1 || ntimes < 0 || kappa < 1 || kappa > 64) return ORC_ERR_ARG;
  for (int i = 0; i < ntimes; ++i)
    if (!(times[i] >= 0.0) || isinf(times[i])) return ORC_ERR_ARG;
  double maxe = orc_max_exit(n, row_ptr, val);
  if (maxe_out) *maxe_out = maxe;
  const int K = kappa;
  int* order = (int*)malloc(sizeof(int) * (size_t)(ntimes > 0 ? ntimes : 1));
  double* exitr = (double*)malloc(sizeof(double) * (size_t)n);
  double* rho = (double*)malloc(sizeof(double) * (size_t)n);
  double* w = (double*)malloc(sizeof(double) * (size_t)n);
  double* Q = (double*)malloc(sizeof(double) * (size_t)n * K);
  double* H = (double*)malloc(sizeof(double) * K * K);
  double* Hm = (double*)malloc(sizeof(double) * K * K);
  double* E = (double*)malloc(sizeof(double) * K * K);
  int rc = ORC_OK;
  if (!order || !exitr || !rho || !w || !Q || !H || !Hm || !E) { rc = ORC_ERR_ALLOC; goto done; }
  for (int64_t s = 0; s < n; ++s) {
    double e = 0.0;
    for (int64_t j = row_ptr[s]; j < row_ptr[s + 1]; ++j) e = e + val[j];
    exitr[s] = e;
  }
  for (int i = 0; i < ntimes; ++i) {
    int j = i;
    while (j > 0 && times[order[j - 1]] > times[i]) { order[j] = order[j - 1]; --j; }
    order[j] = i;
  }
  memcpy(rho, rho0, sizeof(double) * (size_t)n);
  double tprev = 0.0;
  int64_t total = 0;
  for (int q = 0; q < ntimes; ++q) {
    const int ti = order[q];
    const double tau = times[ti] - tprev;
    const int64_t ns = (maxe > 0.0 && tau > 0.0) ? (int64_t)ceil(tau * maxe / (2.0 * K)) : 0;
    const double dt = ns > 0 ? tau / (double)ns : 0.0;
    for (int64_t step = 0; step < ns; ++step) {
      double b2 = 0.0;
      for (int64_t s = 0; s < n; ++s) b2 += rho[s] * rho[s];
      const double beta = sqrt(b2);
      if (beta == 0.0) break;
      for (int64_t s = 0; s < n; ++s) Q[s] = rho[s] / beta;
      for (int i = 0; i < K * K; ++i) H[i] = 0.0;
      int m = K;
      for (int i = 0; i < K; ++i) {
        rate_apply(n, row_ptr, col, val, exitr, Q + (size_t)i * n, w);
        for (int j = 0; j <= i; ++j) {
          const double* qj = Q + (size_t)j * n;
          double h = 0.0;
          for (int64_t s = 0; s < n; ++s) h += qj[s] * w[s];
          H[j * K + i] = h;
          for (int64_t s = 0; s < n; ++s) w[s] = w[s] - h * qj[s];
        }
        if (i + 1 < K) {
          double h2 = 0.0;
          for (int64_t s = 0; s < n; ++s) h2 += w[s] * w[s];
          const double hn = sqrt(h2);
          if (hn <= 1e-14 * maxe) { m = i + 1; break; }
          H[(i + 1) * K + i] = hn;
          double* qn = Q + (size_t)(i + 1) * n;
          for (int64_t s = 0; s < n; ++s) qn[s] = w[s] / hn;
        }
      }
      for (int a = 0; a < m; ++a)
        for (int c = 0; c < m; ++c) Hm[a * m + c] = dt * H[a * K + c];
      rc = orc_expm_pade13(m, Hm, E);
      if (rc) goto done;
      for (int64_t s = 0; s < n; ++s) {
        double v = 0.0;
        for (int i = 0; i < m; ++i) v += Q[(size_t)i * n + s] * E[i * m + 0];
        rho[s] = beta * v;
      }
    }
    total += ns;
    memcpy(out + (size_t)ti * n, rho, sizeof(double) * (size_t)n);
    if (steps_out) steps_out[ti] = total;
    tprev = times[ti];
  }
done:
  free(order); free(exitr); free(rho); free(w); free(Q); free(H); free(Hm); free(E);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Dense matrix exponential: scaling and squaring with the degree-13 Pade   */
/* approximant (N. J. Higham, SIAM J. Matrix Anal. Appl. 26 (2005) 1179).   */
/* The paper's "conventional" baseline (Sec. 1, Sec. 3.2); used on tiny N.  */
/* ------------------------------------------------------------------------ */

static void matmul(int n, const double* A, const double* B, double* C) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int l = 0; l < n; ++l) s += A[i * n + l] * B[l * n + j];
      C[i * n + j] = s;
    }
}

/* E = exp(A) for a dense row-major n x n matrix. */
int orc_expm_pade13(int n, const double* A, double* E) {
  if (n < 1) return ORC_ERR_ARG;
  const int m = 13;
  /* Pade [13/13] numerator coefficients b_j = (2m-j)! m! / ((2m)! j! (m-j)!). */
  double b[14];
  for (int j = 0; j <= m; ++j) {
    long double v = lgammal(2.0L * m - j + 1) + lgammal((long double)m + 1) -
                    lgammal(2.0L * m + 1) - lgammal((long double)j + 1) -
                    lgammal((long double)(m - j) + 1);
    b[j] = (double)expl(v);
  }
  const double theta13 = 5.371920351148152; /* Higham 2005, Table 2.3 */
  size_t nn = (size_t)n * n;
  double* W = (double*)calloc(nn * 12, sizeof(double));
  int* piv = (int*)malloc(sizeof(int) * (size_t)n);
  if (!W || !piv) { free(W); free(piv); return ORC_ERR_ALLOC; }
  double *As = W, *A2 = W + nn, *A4 = W + 2 * nn, *A6 = W + 3 * nn, *U = W + 4 * nn,
         *V = W + 5 * nn, *T1 = W + 6 * nn, *T2 = W + 7 * nn, *Pm = W + 8 * nn,
         *Qm = W + 9 * nn, *R = W + 10 * nn, *T3 = W + 11 * nn;
  double norm1 = 0.0;
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += fabs(A[i * n + j]);
    if (s > norm1) norm1 = s;
  }
  int sc = 0;
  if (norm1 > theta13) sc = (int)ceil(log2(norm1 / theta13));
  double f = ldexp(1.0, -sc);
  for (size_t i = 0; i < nn; ++i) As[i] = A[i] * f;
  matmul(n, As, As, A2);
  matmul(n, A2, A2, A4);
  matmul(n, A4, A2, A6);
  /* U = A [A6 (b13 A6 + b11 A4 + b9 A2) + b7 A6 + b5 A4 + b3 A2 + b1 I] */
  for (size_t i = 0; i < nn; ++i) T1[i] = b[13] * A6[i] + b[11] * A4[i] + b[9] * A2[i];
  matmul(n, A6, T1, T2);
  for (size_t i = 0; i < nn; ++i) T2[i] += b[7] * A6[i] + b[5] * A4[i] + b[3] * A2[i];
  for (int i = 0; i < n; ++i) T2[i * n + i] += b[1];
  matmul(n, As, T2, U);
  /* V = A6 (b12 A6 + b10 A4 + b8 A2) + b6 A6 + b4 A4 + b2 A2 + b0 I */
  for (size_t i = 0; i < nn; ++i) T1[i] = b[12] * A6[i] + b[10] * A4[i] + b[8] * A2[i];
  matmul(n, A6, T1, V);
  for (size_t i = 0; i < nn; ++i) V[i] += b[6] * A6[i] + b[4] * A4[i] + b[2] * A2[i];
  for (int i = 0; i < n; ++i) V[i * n + i] += b[0];
  /* Solve (V - U) R = (V + U) by LU with partial pivoting. */
  for (size_t i = 0; i < nn; ++i) { Qm[i] = V[i] - U[i]; Pm[i] = V[i] + U[i]; }
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(Qm[r * n + c]) > fabs(Qm[p * n + c])) p = r;
    piv[c] = p;
    if (p != c)
      for (int j = 0; j < n; ++j) {
        double t = Qm[c * n + j]; Qm[c * n + j] = Qm[p * n + j]; Qm[p * n + j] = t;
        t = Pm[c * n + j]; Pm[c * n + j] = Pm[p * n + j]; Pm[p * n + j] = t;
      }
    double d = Qm[c * n + c];
    if (d == 0.0) { free(W); free(piv); return ORC_ERR_ARG; }
    for (int r = c + 1; r < n; ++r) {
      double l = Qm[r * n + c] / d;
      if (l == 0.0) continue;
      for (int j = c; j < n; ++j) Qm[r * n + j] -= l * Qm[c * n + j];
      for (int j = 0; j < n; ++j) Pm[r * n + j] -= l * Pm[c * n + j];
    }
  }
  for (int j = 0; j < n; ++j)
    for (int r = n - 1; r >= 0; --r) {
      double s = Pm[r * n + j];
      for (int c = r + 1; c < n; ++c) s -= Qm[r * n + c] * R[c * n + j];
      R[r * n + j] = s / Qm[r * n + r];
    }
  for (int q = 0; q < sc; ++q) {
    matmul(n, R, R, T3);
    memcpy(R, T3, sizeof(double) * nn);
  }
  memcpy(E, R, sizeof(double) * nn);
  free(W);
  free(piv);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Gillespie's direct method (D. T. Gillespie, J. Phys. Chem. 81 (1977)     */
/* 2340), cited by the paper for simulating MJPs (Sec. 2.1.1).  Random      */
/* numbers: splitmix64 seeding xoshiro256** (Blackman & Vigna, 2018).       */
/* ------------------------------------------------------------------------ */

static uint64_t splitmix64(uint64_t* s) {
  uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static uint64_t xoshiro(uint64_t* s) {
  uint64_t r = rotl(s[1] * 5, 7) * 9;
  uint64_t t = s[1] << 17;
  s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
  s[2] ^= t;
  s[3] = rotl(s[3], 45);
  return r;
}
static double unif_open(uint64_t* s) { /* (0, 1) */
  return ((double)(xoshiro(s) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

/*
 * Simulate nruns independent trajectories from state s0 and record the state
 * occupied at each (ascending) observation time: counts[i*n + s] += 1.
 */
int orc_gillespie(int64_t n, const int64_t* row_ptr, const int32_t* col,
                  const double* val, int64_t s0, const double* times,
                  int ntimes, int64_t nruns, uint64_t seed, int64_t* counts) {
  if (n < 1 || s0 < 0 || s0 >= n || ntimes < 1) return ORC_ERR_ARG;
  for (int i = 1; i < ntimes; ++i)
    if (times[i] < times[i - 1]) return ORC_ERR_ARG;
  uint64_t sm = seed, st[4];
  for (int q = 0; q < 4; ++q) st[q] = splitmix64(&sm);
  for (int64_t r = 0; r < nruns; ++r) {
    int64_t s = s0;
    double tau = 0.0;
    int j = 0;
    while (j < ntimes) {
      double e = 0.0;
      for (int64_t q = row_ptr[s]; q < row_ptr[s + 1]; ++q) e += val[q];
      if (e <= 0.0) {
        for (; j < ntimes; ++j) counts[(size_t)j * n + s] += 1;
        break;
      }
      double dt = -log(unif_open(st)) / e;
      while (j < ntimes && tau + dt > times[j]) {
        counts[(size_t)j * n + s] += 1;
        ++j;
      }
      if (j >= ntimes) break;
      tau += dt;
      double u = unif_open(st) * e, acc = 0.0;
      int64_t nxt = col[row_ptr[s + 1] - 1];
      for (int64_t q = row_ptr[s]; q < row_ptr[s + 1]; ++q) {
        acc += val[q];
        if (u < acc) { nxt = col[q]; break; }
      }
      s = nxt;
    }
  }
  return ORC_OK;
}
