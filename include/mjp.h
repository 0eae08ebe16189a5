/*
 * mjp.h -- C ABI of the GB300 R-MJP library (libmjp.so).
 *
 * The library computes transient distributions rho(t) = rho(0) exp(A_theta t)
 * of a Markov jump process with the jump-truncated uniformisation series of
 * Pessoa, Schweiger & Presse (arXiv 2312.05647), Method #3 "R-MJP":
 *
 *   rho*(t) = sum_{k=0}^{K} rho0 B^k Poisson(k | Omega t)
 *             + (1 - sum_{k=0}^{K} Poisson(k | Omega t)) rho0 B^K,
 *   B = I + A/Omega (Eq. B_def), Omega = 1.1 max_n |a_nn|,
 *   K = floor(Omega t + 6 sqrt(Omega t)) + 1  (Eq. R-MJP_expansion, Alg. 2),
 *
 * and the snapshot log-likelihood built from it (Sec. 2.1.2).  All work runs
 * in the library's own CUDA kernels on the calling device; there is no CPU
 * fallback.  Plain C99: no C++ or framework types cross this boundary.
 *
 * Conventions for every entry point:
 *  - Return value: MJP_OK (0) or a negative MJP_ERR_* code; the message of
 *    the most recent failure on the calling thread is mjp_last_error().
 *  - "device" pointers are CUDA device addresses on the current device;
 *    "host" pointers are ordinary CPU memory.  The caller owns every buffer
 *    it passes; the library owns the handles it creates until *_destroy.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy stream).
 *    Calls with device inputs and outputs are asynchronous on that stream;
 *    calls that take or return host data synchronise it before returning.
 *  - A handle carries scratch memory, so calls on one handle must be ordered
 *    (one stream, or explicit synchronisation between streams).
 */
#ifndef MJP_H
#define MJP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
/* Every call that returns int returns one of these; no C++ exception crosses
 * this interface (a failed host allocation is MJP_ERR_ALLOC, any other
 * host-side exception MJP_ERR_ARG).  mjp_last_error() describes the last
 * failure on the calling thread. */
#define MJP_OK 0
#define MJP_ERR_ARG (-1)            /* invalid argument (NULL, size, NaN, t < 0, ...) */
#define MJP_ERR_CSR (-2)            /* malformed CSR (row_ptr not monotone, column out of range, diagonal entry, negative rate) */
#define MJP_ERR_ALLOC (-3)          /* device or host allocation failed */
#define MJP_ERR_CUDA (-4)           /* a CUDA runtime call failed */
#define MJP_ERR_DEVICE_TIMEOUT (-5) /* a bounded device wait ran out */
#define MJP_ERR_KCAP (-6)           /* truncation index K above the configured cap */
#define MJP_ERR_NUMERIC (-7)        /* non-finite or negative probability produced */
#define MJP_ERR_UNSUPPORTED (-8)    /* valid request the library does not handle */

/* ---- model kinds ------------------------------------------------------- */
/* Birth-death, Eq. BD_def (Sec. 3.1.1). dims = {N}; theta = {beta, gamma}:
 * lambda_{n,n+1} = beta (n < N-1), lambda_{n,n-1} = gamma n. */
#define MJP_BD1D 1
/* Two-state birth-death, Eq. Gene_def / Eq. 2S_chem (Sec. 3.1.2).
 * dims = {N_R}; N = 2 N_R, n = n_R + sigma N_R (sigma 0 active, 1 inactive);
 * theta = {beta, gamma, lambda_act, lambda_ina}: birth beta in the active
 * state (n_R < N_R-1), death gamma n_R, active->inactive lambda_ina,
 * inactive->active lambda_act. */
#define MJP_TWOSTATE 2
/* mRNA/protein birth-death (the R -> R+P production of Eq. STS_chem without
 * gene switching).  dims = {M, P}; n = m + M p; theta = {k_m, gamma_m, k_p,
 * gamma_p}: m+1 at k_m, m-1 at gamma_m m, p+1 at k_p m, p-1 at gamma_p p;
 * births that would leave the box are dropped. */
#define MJP_MRNA_PROT2D 3
/* General sparse rate matrix given as CSR (rows = source state). */
#define MJP_CSR 4
/* Autoregulatory gene network, Eq. STS_chem / Eq. autoReg_def (Sec. 3.1.3).
 * dims = {N_R, N_P} (both >= 2); N = 2 N_R N_P, n = n_R + N_R n_P +
 * N_R N_P sigma (sigma 0 active, 1 inactive); theta = {beta_R, beta_P,
 * gamma_R, gamma_P, lambda_act, lambda_ina}: transcription n_R+1 at beta_R
 * (active only), translation n_P+1 at beta_P n_R (either state), decays
 * gamma_R n_R and gamma_P n_P, binding (active, n_P) -> (inactive, n_P-1) at
 * lambda_ina n_P, unbinding (inactive, n_P) -> (active, n_P+1) at lambda_act;
 * transitions whose target leaves the box are dropped (reflecting).  The
 * chain kernels hold it as N_R columns by 2 N_P rows (row 2 n_P + sigma). */
#define MJP_AUTOREG 5

/* ---- chain precision --------------------------------------------------- */
#define MJP_FP32 1 /* FP32 chain, Kahan-compensated FP32 accumulation, FP64 Omega/K/weights */
#define MJP_FP64 2 /* FP64 chain and accumulation */

/* ---- truncation rule --------------------------------------------------- */
#define MJP_TRUNC_PAPER 0 /* K = floor(x + 6 sqrt x) + 1, x = Omega t (Algorithm 2) */
#define MJP_TRUNC_TOL 1   /* smallest K with Poisson tail mass <= tol (1e-20 <= tol < 0.5) */

/* ---- pointer kinds for batched calls ----------------------------------- */
#define MJP_PTR_HOST 0
#define MJP_PTR_DEVICE 1

/* ---- model options (rate_model_set_option) ----------------------------- */
#define MJP_OPT_RENORM_PERIOD 1 /* FP32 chains: every r jumps, add back to each state the defect of its FP32 exit
                                   coefficient (1 minus the rounded outflow coefficients of its column of B), which
                                   keeps the unit column sums of B (Eq. B_def) that rounding breaks.  Default 32;
                                   0 = off; else a multiple of 8 in [8, 2^20].  Identical across kernels.  FP64
                                   chains ignore it.  Also a batch option. */
#define MJP_OPT_K_CAP 2         /* largest K accepted (default 2^26) */
#define MJP_OPT_THREADS 3       /* threads per CTA for stencil chains, one warp of which forms the weights (0 = automatic; else a multiple of 32 in [64, 1024]) */
#define MJP_OPT_CLUSTER 4       /* CTAs per instance for stencil chains (0 = automatic; 1, 2, 4, 8, 16) */
#define MJP_OPT_PROFILE 5       /* 1: record CUDA events around each kernel of a call (see rate_model_last_timing) */
#define MJP_OPT_ARENA 6         /* capacity (elements) of the planner's Poisson-weight store; 0 = automatic.  Windows
                                   that do not fit are generated in the chain by Algorithm 2's recurrence instead. */
#define MJP_OPT_CHAIN 7         /* general CSR models: 0 or 1 = one launch per jump (default), 2 = the whole chain in
                                   one cooperative launch with a bounded grid barrier per jump (identical results;
                                   see MJP_OPT_WAIT_LIMIT).  Stencil models: 0 = automatic (the register-resident kernels for
                                   the log-likelihood of FP32 mRNA/protein boxes (automatic thread count or 256),
                                   of FP32 two-state models whose observation groups have at most two members (one
                                   CTA of MJP_OPT_THREADS / 32 <= 8 warps per theta; automatic when 0) and for
                                   expv_series of birth-death models (automatic thread count), none with a forced
                                   cluster size, else the shared-memory kernel), 1 = shared-memory
                                   kernel, 2 = register-resident kernel (MJP_ERR_UNSUPPORTED where it does not
                                   apply; other models' expv_series always runs the shared-memory kernel).  Also a batch option
                                   (expv_batch_set_option): 0 = the register-resident birth-death kernel wherever every
                                   instance fits it (N_j <= 8 x 6,720 states FP32, 8 x 3,360 FP64), 1 = shared-memory
                                   kernel, 2 = register-resident kernel */
#define MJP_OPT_HALO 8          /* batches, register-resident kernel: halo width h of an instance split over a cluster,
                                   i.e. jumps between two halo exchanges (default 32; 1 .. 1024) */
#define MJP_OPT_METHOD 9        /* expv_series method: 0 = R-MJP (Algorithm 2, default), 1 = fourth-order Runge-Kutta
                                   (Method #4), 2 = Krylov subspace steps (Method #5, Algorithm 3 with the full
                                   projection of Eq. Krylov_projection).  1 and 2: FP64 birth-death and two-state
                                   models of at most 4,096 states; the times are visited in ascending order and each interval is
                                   split into ceil(interval x max_n |a_nn| / D) equal steps, D = 1 (RK4) or
                                   2 kappa (Krylov, Sec. 2.3); the info report then gives omega = max_n |a_nn|,
                                   K_i = cumulative steps to t_i, eps_i = 0 */
#define MJP_OPT_KAPPA 10        /* Krylov subspace size kappa (default 20, the paper's; 1 .. 32) */
#define MJP_OPT_WAIT_LIMIT 11   /* polls of a bounded wait before it gives up (default 2^24, about a second; 0 = give up
                                   at once): general CSR models with MJP_OPT_CHAIN = 2 (a CTA at the grid barrier),
                                   the register-resident two-state log-likelihood chain (the hand-over of observation
                                   chunks between its chain and reducer warps) and the register-resident
                                   mRNA/protein log-likelihood chain (the hand-over of the block rows that cross
                                   from one CTA of a cluster to the next, every jump).  A wait that runs out stops
                                   the CSR and two-state chains; the mRNA/protein chain stops waiting and runs on to
                                   its end with invalid values.  rate_model_check then returns
                                   MJP_ERR_DEVICE_TIMEOUT */

typedef struct mjp_model mjp_model;
typedef struct mjp_obs mjp_obs;

/* Per-call report of the truncation (Eq. R-MJP_expansion, Alg. 2).  Arrays
 * are host memory of length ntimes supplied by the caller (or NULL). */
typedef struct {
  double omega;    /* Omega = 1.1 max_n |a_nn| (0 when every rate is zero) */
  int64_t* K;      /* K_i per time, in the caller's time order */
  double* eps;     /* epsilon_i = 1 - sum_{k<=K_i} Poisson(k|Omega t_i), the tail moved onto rho0 B^K */
} mjp_series_info;

/* Message of the last failure on this thread ("" if none). */
const char* mjp_last_error(void);

/* Library version string. */
const char* mjp_version(void);

/*
 * Create a stencil model (rates built matrix-free on the device from theta).
 * kind/dims/theta as documented beside MJP_BD1D, MJP_TWOSTATE,
 * MJP_MRNA_PROT2D; rates must be finite and >= 0.  precision is MJP_FP32 or
 * MJP_FP64.  Errors: MJP_ERR_ARG.
 * Paper: Eq. A_def (generator from rates), Eqs. BD_def and Gene_def.
 */
int rate_model_create_stencil(mjp_model** out, int kind, const int64_t* dims, int ndims,
                              const double* theta, int ntheta, int precision);

/*
 * Create a model from a general rate matrix Lambda in CSR form (host arrays):
 * row_ptr[n+1] (monotone, row_ptr[0] = 0), col[nnz] in [0, n) with no
 * diagonal entries, rate[nnz] >= 0 finite.  Rows are source states
 * (lambda_nm = rate of n -> m, Sec. 2.1).  The library copies the data,
 * forms the exit rates e_n = sum_m lambda_nm and stores B^T (incoming
 * transitions) on the device.  Errors: MJP_ERR_ARG, MJP_ERR_CSR, MJP_ERR_ALLOC.
 */
int rate_model_create_csr(mjp_model** out, int64_t n, const int64_t* row_ptr, const int32_t* col,
                          const double* rate, int precision);

/* Replace theta of a stencil model (host array). Errors: MJP_ERR_ARG. */
int rate_model_set_theta(mjp_model* m, const double* theta, int ntheta);

/* Set an MJP_OPT_* option.  Errors: MJP_ERR_ARG. */
int rate_model_set_option(mjp_model* m, int option, int64_t value);

/* Number of states N of the model (or -1 for a NULL handle). */
int64_t rate_model_num_states(const mjp_model* m);

/* Free the model and its device memory (NULL is ignored). */
void rate_model_destroy(mjp_model* m);

/*
 * Transient distributions at several times (Algorithm 2 per time; one jump
 * chain rho0 B^k is shared by all times, each time with its own K_i, window
 * of weights and tail).
 *   rho0   device, N values in the model's precision (float or double), >= 0.
 *   times  host, ntimes values, finite and >= 0, any order, 1 <= ntimes <= 256.
 *   out    device, ntimes x N row-major in the model's precision; row i is
 *          rho*(times[i]).
 *   info   host, nullable; when given the call synchronises `stream`.
 * Errors: MJP_ERR_ARG, MJP_ERR_KCAP, MJP_ERR_ALLOC, MJP_ERR_CUDA.
 */
int expv_series(mjp_model* m, const void* rho0, const double* times, int ntimes, void* out,
                mjp_series_info* info, int trunc_mode, double tol, void* stream);

/*
 * Snapshot observations (Sec. 2.1.2): at each time T^i a set of observation
 * groups; group g holds the states whose probabilities are summed (a hidden
 * component, e.g. the gene state of Sec. 3.1.2, is summed out this way) and a
 * count c_g >= 0.  Host arrays:
 *   times[ntimes]            observation times (>= 0, any order),
 *   group_ptr[ntimes+1]      groups of time i are [group_ptr[i], group_ptr[i+1]),
 *   counts[G]                multiplicity of each group,
 *   member_ptr[G+1]          states of group g are members[member_ptr[g] ..],
 *   members[]                state indices in [0, n),
 *   rho0[n]                  initial distribution rho(0) (FP64, >= 0).
 * The library copies everything.  Limits: ntimes <= 256, G <= 8192.
 * Errors: MJP_ERR_ARG, MJP_ERR_ALLOC.
 */
int mjp_obs_create(mjp_obs** out, int64_t n, int ntimes, const double* times,
                   const int64_t* group_ptr, const double* counts, const int64_t* member_ptr,
                   const int32_t* members, const double* rho0);
void mjp_obs_destroy(mjp_obs* obs);

/*
 * Log-likelihood of the observations for B parameter vectors:
 *   out[b] = sum_i sum_g c_g log( sum_{s in g} rho*(T^i | theta_b)_s ),
 * rho* from the R-MJP series above (p(s^i|theta) = rho(T^i)_{s^i}, Sec. 2.1.2;
 * hidden states summed as in Sec. 3.1.2).  The prior is not included.
 *   theta  B x ntheta row-major (stencil models; ignored for CSR, where B = 1)
 *   out    B values
 *   where  MJP_PTR_HOST: theta and out are host memory (the call copies and
 *          synchronises); MJP_PTR_DEVICE: both are device memory (async).
 * An observed group with probability 0 gives -inf (not an error).
 * Errors: MJP_ERR_ARG, MJP_ERR_KCAP, MJP_ERR_ALLOC, MJP_ERR_CUDA.
 */
int loglik(mjp_model* m, const mjp_obs* obs, const double* theta, int B, double* out, int where,
           int trunc_mode, double tol, void* stream);

/*
 * Device time of the kernels of the most recent expv_series/loglik call on
 * this model, measured with CUDA events recorded on the call's stream around
 * each kernel (needs MJP_OPT_PROFILE = 1 before the call).  Waits for the
 * call to finish.  ms_plan: the planner kernel (Omega, K, weights);
 * ms_chain: the jump-chain kernel.  Either pointer may be NULL.
 * Errors: MJP_ERR_ARG (profiling off or no call yet), MJP_ERR_CUDA.
 */
int rate_model_last_timing(mjp_model* m, double* ms_plan, double* ms_chain);

/*
 * J-MJP state probabilities (Method #2, Sec. 2.2.2, Algorithm 1): for the
 * model's theta, phi[i] = sum over observation i's group of (rho0 B^{k[i]}),
 * B = I + A / Omega, Omega = 1.1 max_n |a_nn| (Eq. B_def): one chain read at
 * every observation's own number of virtual jumps.  Birth-death and
 * two-state models (one CTA; the chain in shared memory, the observations
 * staged beside it in chunks sorted by k).
 *   rho0       device, N values in the model's precision.
 *   k          host, nobs jump counts in [0, 2^31 - 1) (any order).
 *   group_ptr  host, nobs + 1 (group_ptr[0] = 0): observation i sums the
 *              states members[group_ptr[i] .. group_ptr[i+1]) (e.g. both gene
 *              states of an observed n_R, Sec. 3.1.2); every group non-empty.
 *   phi        host, nobs results (FP64).  Synchronises `stream`.
 * Errors: MJP_ERR_ARG, MJP_ERR_UNSUPPORTED (other kinds, too many states),
 * MJP_ERR_ALLOC, MJP_ERR_CUDA.
 */
int jmjp_state_probs(mjp_model* m, const void* rho0, int64_t nobs, const int64_t* k, const int64_t* group_ptr,
                     const int32_t* members, double* phi, void* stream);

/*
 * ---- batches of uneven instances --------------------------------------
 * Many birth-death models (Eq. BD_def) with different sizes N_j, rates
 * theta_j = {beta_j, gamma_j} and one observation time t_j each, rho0 =
 * delta at s0_j, evaluated in one call: every instance is its own R-MJP
 * series (Algorithm 2).  The library orders instances by estimated work
 * (K_j N_j, longest first), runs light instances one CTA each and splits
 * heavy ones over a thread-block cluster, launching the groups concurrently;
 * the whole call can be captured once as a CUDA graph and replayed.
 */
typedef struct mjp_batch mjp_batch;

/* Host arrays of n_inst entries (theta: n_inst x 2; s0 may be NULL = 0).
 * precision: MJP_FP32 or MJP_FP64.  Errors: MJP_ERR_ARG, MJP_ERR_ALLOC. */
int expv_batch_create(mjp_batch** out, int kind, int n_inst, const int64_t* N, const double* theta,
                      const double* t, const int64_t* s0, int precision);

/* offsets[j] (host, n_inst + 1 entries): instance j's distribution occupies
 * out[offsets[j] .. offsets[j+1]) of the output of expv_batch_run. */
int expv_batch_offsets(const mjp_batch* b, int64_t* offsets);

/* Evaluate all instances; out is device memory of offsets[n_inst] values in
 * the batch precision.  Asynchronous on `stream`.  With use_graph = 1 the
 * launch sequence is captured as a CUDA graph on the first call for a given
 * (out, stream) and replayed afterwards.  Errors: MJP_ERR_ALLOC, MJP_ERR_CUDA. */
int expv_batch_run(mjp_batch* b, void* out, int use_graph, void* stream);

/* Autotune the launch configuration (threads of light CTAs, cluster size and
 * threads of heavy instances, the heavy threshold) by timing candidate
 * configurations on `stream` with CUDA events (runs the batch several times
 * into `out`).  Writes the chosen configuration as text into cfg (nullable,
 * cfg_len bytes).  Errors: as expv_batch_run. */
int expv_batch_tune(mjp_batch* b, void* out, void* stream, char* cfg, int cfg_len);

/* Device-side error check of the last run (synchronises `stream`). */
int expv_batch_check(mjp_batch* b, void* stream);

/* Batch options: MJP_OPT_CHAIN (0 automatic, 1 shared-memory kernel, 2
 * register-resident kernel; see beside MJP_OPT_CHAIN), MJP_OPT_CLUSTER (CTAs
 * per heavy instance, 0 = automatic, else 1 .. 8; instances that need more
 * CTAs to fit still get them), MJP_OPT_HALO (halo width of the
 * register-resident kernel's clusters), MJP_OPT_RENORM_PERIOD (FP32 exit-defect
 * correction period, as for models).  Takes effect at the next run or tune
 * (a captured graph is rebuilt).  Every setting gives the same results up to
 * the bit (the kernels share their arithmetic).  Errors: MJP_ERR_ARG. */
int expv_batch_set_option(mjp_batch* b, int option, int64_t value);

void expv_batch_destroy(mjp_batch* b);

/*
 * expv_series_static -- the same transient distributions as expv_series for a
 * stencil model in FP32, for callers that cannot allocate device memory while
 * they run (applications whose device memory belongs to their own pool or has
 * a fixed budget, plugins whose host framework owns the allocator, loops that
 * must not risk the device-wide synchronisation of cudaMalloc/cudaFree).  The
 * paper has no counterpart: this is an interface variant, not a method.
 *
 * No handle: kind/dims/theta describe the model as for
 * rate_model_create_stencil; rho0 (device, N floats) and out (device,
 * ntimes x N floats, row i = rho*(times[i])) are the caller's; times are host
 * memory.  The call allocates no device memory and no host heap memory on its
 * success path.  Its scratch (sorted times, truncation windows, status word
 * and the FP32 Kahan compensation, ntimes x N x 4 bytes) is one static array
 * of 16 MiB inside the library, which every GPU that loads the library keeps
 * until the process exits; larger requests fail with MJP_ERR_ARG and a
 * message giving the size needed.  The first call on a device looks up that
 * array's device address (once per device, with the device current).  All
 * calls share the array and it keeps the last call's contents (the call resets
 * what must start at zero): calls that overlap on the GPU -- on different
 * streams, threads or devices sharing a process -- race, so order them.  The
 * call copies from host stack memory, synchronises `stream` and reports
 * device-side errors (MJP_ERR_KCAP, MJP_ERR_NUMERIC) itself; it must not be
 * called while `stream` is capturing a graph (MJP_ERR_UNSUPPORTED).  Models of
 * more than 2^31 - 1 states are MJP_ERR_ARG; a launch shape the GPU cannot
 * hold is MJP_ERR_UNSUPPORTED.
 * Errors: MJP_ERR_ARG, MJP_ERR_UNSUPPORTED, MJP_ERR_KCAP, MJP_ERR_NUMERIC, MJP_ERR_CUDA.
 */
int expv_series_static(int kind, const int64_t* dims, int ndims, const double* theta, int ntheta,
                       const float* rho0, const double* times, int ntimes, float* out, void* stream);

/*
 * Measured on-chip peaks of the current device, for roofline denominators (the
 * paper has no counterpart; the benchmark reports the chain kernels against
 * them).  MJP_PEAK_FP32_FMA: FP32 fused multiply-adds from independent
 * chains on two 512-thread CTAs per SM, in TFLOP/s (2 flops per FMA), the
 * better of packed FP32x2 and scalar instructions; MJP_PEAK_SMEM: 16-byte shared-memory loads and stores of
 * consecutive vectors (no bank conflicts) on the same grid, in GB/s counting
 * read plus written bytes.  `iters` loop iterations per thread (a few hundred
 * thousand give ~10 ms); best of three timed launches with CUDA events on
 * `stream` after one untimed launch.  Allocates and frees a small device
 * buffer.  Errors: MJP_ERR_ARG, MJP_ERR_ALLOC, MJP_ERR_CUDA.
 */
#define MJP_PEAK_FP32_FMA 1
#define MJP_PEAK_SMEM 2
#define MJP_PEAK_L2_GATHER 3 /* 4-byte loads at random positions of an L2-resident 4 MB array, in G loads/s */
int mjp_measure_peak(int which, int iters, double* result, void* stream);

/*
 * Synchronise `stream` and report device-side errors recorded by earlier
 * asynchronous calls on this model (K above the cap, non-finite values, a
 * bounded wait that ran out).  Clears the record.  Returns MJP_OK or the
 * first recorded MJP_ERR_*.
 */
int rate_model_check(mjp_model* m, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* MJP_H */
