/*
 * mjp_surrogate.h -- C ABI of the log-likelihood surrogate and the posterior
 * sampler of libmjp.so (same conventions as mjp.h: MJP_OK or a negative
 * MJP_ERR_* code, mjp_last_error() for the message, `where` selects host or
 * device buffers, `stream` is a cudaStream_t passed as void*, calls with
 * host data synchronise the stream before returning).
 *
 * Sampler: Metropolis-Hastings on Psi = log(theta) (SI A.1) with the
 * Gaussian random-walk proposal Normal(Psi, Z) of Eq. prop, the adaptive
 * covariance of Eq. update_S (SI A.2, constants of SI A.4.3), the prior of
 * Eq. prior (independent Normal(1, 1e5) on each Psi^a) and the exact
 * log-likelihood of mjp.h's loglik() (Sec. 2.1.2).  Delayed acceptance
 * (Christen & Fox 2005) puts a surrogate in front: a proposal is first
 * accepted with probability min(1, exp(s(Psi') + lp(Psi') - s(Psi) -
 * lp(Psi))) for the surrogate s and the log-prior lp, and only its survivors
 * meet the exact log-likelihood l, accepted with probability min(1,
 * exp(l(Psi') - l(Psi) - s(Psi') + s(Psi))); the chain keeps the exact
 * posterior as its stationary law.
 *
 * Surrogate: a 4 -> 128 -> 128 -> 1 perceptron with tanh hidden layers on
 * standardised inputs, s(Psi) = mu_y + sd_y f((Psi - mu_x) / sd_x), FP32
 * weights and arithmetic, trained by mean squared error with Adam on
 * (Psi, exact log-likelihood) pairs the sampler records.
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = (seed low 32
 * bits, seed high 32 bits).  Chain c at its iteration h draws its proposal
 * normals from blocks (h, 0, c, 0) and (h, 0, c, 1) (two Box-Muller pairs of
 * the uniforms (m + 0.5) 2^-52, m = the top 26 bits of two words), and its
 * accept uniforms from block (h, 0, c, 2): the first for a plain MH step or
 * the first stage, the second for the exact stage.
 */
#ifndef MJP_SURROGATE_H
#define MJP_SURROGATE_H

#include "mjp.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ---- surrogate --------------------------------------------------------- */
#define MJP_MLP_IN 4
#define MJP_MLP_HIDDEN 128
/* Flat FP32 parameter vector, row-major, y = x W + b: W1[4][128] at 0,
 * b1[128] at 512, W2[128][128] at 640, b2[128] at 17024, W3[128] at 17152,
 * b3 at 17280. */
#define MJP_MLP_NPAR 17281
/* FP64 standardisation: mu_x[4], sd_x[4], mu_y, sd_y. */
#define MJP_MLP_NNORM 10

typedef struct mjp_mlp mjp_mlp;

/* Create a network on the current device with Glorot-uniform weights
 * U(-a, a), a = sqrt(6 / (fan_in + fan_out)), and zero biases: weight i is
 * (2u - 1) a for the first uniform of Philox block (i, 0, 0x4D4C5000, 0).
 * Standardisation starts as the identity (means 0, deviations 1).
 * Errors: MJP_ERR_ARG, MJP_ERR_ALLOC, MJP_ERR_CUDA. */
int mjp_mlp_create(mjp_mlp** out, uint64_t seed);
void mjp_mlp_destroy(mjp_mlp* net);

/* Copy parameters (MJP_MLP_NPAR floats) and standardisation
 * (MJP_MLP_NNORM doubles) in or out; either pointer may be NULL to skip it.
 * set rejects non-finite values and deviations <= 0 (MJP_ERR_ARG); Adam's
 * moments are reset by set. */
int mjp_mlp_set_params(mjp_mlp* net, const float* params, const double* norm, int where, void* stream);
int mjp_mlp_get_params(mjp_mlp* net, float* params, double* norm, int where, void* stream);

/* Fit the standardisation to n >= 1 rows: psi [n][4] and y [n] (FP64):
 * means and population standard deviations (a zero deviation becomes 1). */
int mjp_mlp_fit_norm(mjp_mlp* net, const double* psi, const double* y, int64_t n, int where, void* stream);

/* s(psi) for n >= 1 rows: psi [n][4] -> out [n] (FP64 in and out). */
int mjp_mlp_forward(mjp_mlp* net, const double* psi, int64_t n, double* out, int where, void* stream);

/* Mean squared error on the standardised data and its gradient:
 * loss = (1/n) sum_r (f(x_r) - t_r)^2, x = (psi - mu_x)/sd_x,
 * t = (y - mu_y)/sd_y; grad [MJP_MLP_NPAR] in FP32 (the kernels' precision),
 * loss in FP64.  Either output may be NULL. */
int mjp_mlp_loss_grad(mjp_mlp* net, const double* psi, const double* y, int64_t n, double* loss, float* grad,
                      int where, void* stream);

typedef struct {
  int64_t steps;  /* Adam steps (>= 1) */
  int64_t batch;  /* rows per step: all n rows in order when batch >= n, else n-row
                     draws with replacement, row r of step s = floor(w n / 2^32) for
                     word 0 w of Philox block (r, s, 0x4D4C5001, 0) */
  double lr;      /* learning rate (> 0) */
  double beta1;   /* Adam moment decay rates, in [0, 1) */
  double beta2;
  double eps;     /* Adam denominator offset (> 0) */
  uint64_t seed;  /* key of the row draws */
  int fit_norm;   /* 1: fit the standardisation to (psi, y) first */
} mjp_train_cfg;

/* Train with Adam (Kingma & Ba 2015): per step the minibatch gradient of the
 * loss above, then m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2, p -= lr
 * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps) with t counting steps
 * since the last set_params or create.  losses [steps] (FP64, may be NULL)
 * receives each step's minibatch loss, before the step's update. */
int mjp_mlp_train(mjp_mlp* net, const double* psi, const double* y, int64_t n, const mjp_train_cfg* cfg,
                  double* losses, int where, void* stream);

/* ---- sampler ----------------------------------------------------------- */
typedef struct mjp_sampler mjp_sampler;

/* A sampler of `chains` chains (1..4096) on a stencil model with 4 rates
 * (MJP_TWOSTATE, MJP_MRNA_PROT2D) and its observations.  The model and obs
 * must outlive the sampler.  `capacity` >= 1: samples kept per chain (a
 * ring: the newest `capacity`).  `eval_capacity` >= 0: (Psi', l(Psi'))
 * pairs of exact evaluations kept for surrogate training (the first ones
 * only).  Z starts as 1e-8 I (SI A.4.3).  Errors: MJP_ERR_ARG,
 * MJP_ERR_UNSUPPORTED (other model kinds), MJP_ERR_ALLOC. */
int mjp_sampler_create(mjp_sampler** out, mjp_model* m, const mjp_obs* obs, int chains, int64_t capacity,
                       int64_t eval_capacity, uint64_t seed);
void mjp_sampler_destroy(mjp_sampler* s);

/* Put every chain at psi [chains][4] (FP64) and evaluate its exact
 * log-likelihood (iteration counters and kept samples are not touched). */
int mjp_sampler_set_state(mjp_sampler* s, const double* psi, int where, void* stream);
/* Current Psi [chains][4] and exact log-likelihood [chains]; NULL skips. */
int mjp_sampler_get_state(mjp_sampler* s, double* psi, double* loglik, int where, void* stream);

/* Set the proposal covariance Z (4 x 4 row-major, symmetric positive
 * definite, host memory); its Cholesky factor is taken on the device.
 * MJP_ERR_ARG if Z is not symmetric positive definite. */
int mjp_sampler_set_cov(mjp_sampler* s, const double* Z, void* stream);
int mjp_sampler_get_cov(mjp_sampler* s, double* Z, void* stream);

/* Eq. update_S on the pooled newest `window` kept samples of every chain:
 * Z = (2.38/4)^2 [ mean(psi^T psi) - mean(psi)^T mean(psi) + eps I ].
 * MJP_ERR_ARG if fewer than `window` samples are kept. */
int mjp_sampler_adapt_cov(mjp_sampler* s, int64_t window, double eps, void* stream);

/* `iters` plain MH iterations of every chain: one batched exact
 * log-likelihood of all chains' proposals per iteration.  record = 1 keeps
 * each iteration's state. */
int mjp_sampler_run_plain(mjp_sampler* s, int64_t iters, int record, void* stream);

/* Delayed acceptance until every chain has done `iters` more iterations.
 * Per round, each unfinished chain screens up to max_inner (1..1024)
 * proposals with the surrogate -- each screened proposal is one full
 * iteration; a first-stage rejection keeps the state -- until one passes the
 * first stage; the round's survivors are compacted into one batch for the
 * exact log-likelihood and decided by the second stage. */
int mjp_sampler_run_da(mjp_sampler* s, mjp_mlp* net, int64_t iters, int max_inner, int record, void* stream);

/* Forget kept samples (and, with evals = 1, kept evaluation pairs) and zero
 * the counters below; chain states and iteration counters stay. */
int mjp_sampler_clear(mjp_sampler* s, int evals, void* stream);

typedef struct {
  int64_t iterations;   /* summed over chains */
  int64_t accepted;     /* moves (plain or second stage) */
  int64_t stage1;       /* proposals that passed the first stage */
  int64_t exact_evals;  /* exact log-likelihoods of proposals */
  int64_t rounds;       /* batched exact log-likelihood launches */
  int64_t kept;         /* kept samples per chain (<= capacity) */
  int64_t evals_kept;   /* kept evaluation pairs */
} mjp_sampler_stats;
int mjp_sampler_stats_get(mjp_sampler* s, mjp_sampler_stats* out, void* stream);

/* Kept samples in order, oldest first: out [chains][kept][4] (FP64). */
int mjp_sampler_trace(mjp_sampler* s, double* out, int where, void* stream);
/* Kept evaluation pairs: psi [evals_kept][4], loglik [evals_kept]; device
 * pointers into the sampler (valid until the next call on it). */
int mjp_sampler_evals(mjp_sampler* s, const double** psi, const double** loglik, int64_t* n);

/* Checkpoint and resume (the paper has no counterpart: it runs its chains
 * in one go).  A checkpoint holds everything a sampler carries from one run
 * to the next: every chain's Psi, exact and surrogate log-likelihoods and
 * iteration count (the Philox counter of its random numbers: with the seed,
 * the whole random state), the counters, best points, kept samples,
 * recorded evaluation pairs, Z and its Cholesky factor.  Restored into a
 * sampler created with the same chains, capacities and seed (on the same
 * model and observations, which the caller keeps), a run continues exactly
 * as it would have without the interruption.  The surrogate network is
 * saved separately (mjp_mlp_get_params / mjp_mlp_set_params).
 * mjp_sampler_checkpoint_size: bytes of a checkpoint of `s`.
 * mjp_sampler_save: writes it to host memory `buf` (`bytes` >= that size);
 * synchronises `stream`.  Call it between runs.
 * mjp_sampler_load: reads one written by mjp_sampler_save; MJP_ERR_ARG when
 * `buf` is not a checkpoint of this library version, is truncated, or comes
 * from a sampler with other chains, capacities or seed (then `s` is
 * unchanged); synchronises `stream`.  The layout is the host's byte order. */
int mjp_sampler_checkpoint_size(mjp_sampler* s, size_t* bytes);
int mjp_sampler_save(mjp_sampler* s, void* buf, size_t bytes, void* stream);
int mjp_sampler_load(mjp_sampler* s, const void* buf, size_t bytes, void* stream);

typedef struct {
  int64_t every;        /* H: iterations between updates of Z (300) */
  int64_t window;       /* H': samples per update (100) */
  int64_t cycle;        /* iterations per acceptance-rate cycle (100) */
  int64_t good_cycles;  /* cycles with acceptance in [acc_lo, acc_hi] that end a phase (10) */
  double z0;            /* Z = z0 I at the start of a phase (1e-8) */
  double eps;           /* epsilon of Eq. update_S (1e-12) */
  double acc_lo, acc_hi;/* 0.2, 0.5 */
  int restart_at_best;  /* 1: a second phase from Z = z0 I, every chain restarted at
                           the highest-posterior state seen (SI A.4.3) */
  int64_t max_iters;    /* per phase */
} mjp_adapt_cfg;
typedef struct {
  int64_t iters[2];     /* iterations per phase */
  int64_t good[2];      /* good cycles per phase */
  int converged;        /* every phase reached good_cycles */
  double acc_last;      /* pooled acceptance of the last cycle */
} mjp_adapt_report;
/* The adaptive protocol of SI A.2 and A.4.3 with pooled chains: plain MH in
 * cycles; Z updated every `every` iterations from the newest `window`
 * samples of all chains; a phase ends after good_cycles cycles whose pooled
 * acceptance rate lies in [acc_lo, acc_hi] (or max_iters).  Kept samples are
 * overwritten (the ring must hold `window`); evaluation pairs accumulate. */
int mjp_sampler_adapt(mjp_sampler* s, const mjp_adapt_cfg* cfg, mjp_adapt_report* report, void* stream);

/* ---- effective sample size --------------------------------------------- */
/* For trace [chains][len][params] (FP64, len >= 4): per parameter the pooled
 * mean and (population) variance, the ESS summed over chains (Geyer's initial
 * monotone sequence on each chain: Gamma_m = gamma(2m) + gamma(2m+1) summed
 * while positive and clipped to the previous, tau = (2 sum Gamma_m -
 * gamma(0)) / gamma(0) floored at 1 / log10(len), ESS = len / tau), and
 * Monte Carlo standard errors
 * sqrt(var / ESS) of the mean and, by the same estimator on the squared
 * deviations from the pooled mean, of the variance.  Outputs [params] each
 * (any may be NULL). */
int mjp_ess(const double* trace, int64_t chains, int64_t len, int params, double* ess, double* mean, double* var,
            double* mcse_mean, double* mcse_var, int where, void* stream);

#ifdef __cplusplus
}
#endif
#endif
