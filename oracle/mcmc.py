"""CPU oracle for the posterior sampler -- TEST INFRASTRUCTURE ONLY.

Plain FP64 NumPy restatement of the Metropolis-Hastings sampler of SI A.1-A.4
(proposal Eq. prop in Psi = log(theta), adaptive covariance Eq. update_S,
prior Eq. prior), of delayed acceptance (Christen & Fox, J. Comput. Graph.
Stat. 14(4), 2005) with a surrogate log-likelihood as the first stage, and of
the effective sample size (Geyer, Stat. Sci. 7(4), 1992, initial monotone
sequence estimator).  Only ``tests/`` and the CPU legs of ``bench.py`` may
import it; the CUDA library never does.

Random numbers come from one counter-based generator, Philox4x32-10 (Salmon,
Moraes, Dror & Shaw, SC'11), which the CUDA sampler implements independently
from the same published definition, so that both sides draw identical
numbers.  The assignment of counters to draws is the sampler's contract:

* proposal normals of chain c at its iteration h: counter (h, 0, c, 0) and
  (h, 0, c, 1), two Box-Muller pairs each giving (z0, z1) then (z2, z3);
* accept uniforms of chain c at iteration h: counter (h, 0, c, 2); the first
  uniform decides a plain MH step or the first delayed-acceptance stage, the
  second the exact (second) stage;
* key = (seed low 32 bits, seed high 32 bits).

Parity status: every function is pinned by ``tests/test_oracle_mcmc.py`` --
Philox's round structure against NumPy's Philox4x64-10, the delayed-acceptance
kernel by exact stationarity on a discrete target, ESS by the AR(1) closed form
and an FFT autocovariance, the adaptive update by the covariance of a known
sample.
"""
from __future__ import annotations

import math

import numpy as np

# Philox4xW-10 constants (Salmon et al. 2011): round multipliers and key Weyl
# increments for W = 32 and W = 64.
PHILOX32 = ((0xD2511F53, 0xCD9E8D57), (0x9E3779B9, 0xBB67AE85), 32)
PHILOX64 = ((0xD2E7470EE14C6C93, 0xCA5A826395121157), (0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B), 64)

ADAPT_SCALE = (2.38 / 4.0) ** 2   # (2.38 / eta)^2 of Eq. update_S with eta = 4 parameters
Z_INIT = 1e-8                     # z of Z = z I (SI A.4.3)
EPS_COV = 1e-12                   # epsilon of Eq. update_S (SI A.4.3)
ADAPT_EVERY = 300                 # H (SI A.4.3)
ADAPT_WINDOW = 100                # H' (SI A.4.3)
CYCLE = 100                       # samples per acceptance-rate cycle (SI A.4.3)
PRIOR_MU, PRIOR_SIGMA = 1.0, 1e5  # Eq. prior


def philox(ctr, key, spec=PHILOX32, rounds: int = 10):
    """Philox4xW-R block: four W-bit words of ``ctr`` under the two-word ``key``.

    Each round multiplies words 0 and 2 by the round multipliers, keeps the high
    and low halves of both products, and mixes the high halves with the other
    two words and the key; the key advances by the Weyl constants between
    rounds."""
    (m0, m1), (w0, w1), w = spec
    mask = (1 << w) - 1
    c = [int(x) & mask for x in ctr]
    k = [int(x) & mask for x in key]
    for _ in range(rounds):
        p0 = m0 * c[0]
        p1 = m1 * c[2]
        c = [(p1 >> w) ^ c[1] ^ k[0], p1 & mask, (p0 >> w) ^ c[3] ^ k[1], p0 & mask]
        k = [(k[0] + w0) & mask, (k[1] + w1) & mask]
    return c


def seed_key(seed: int):
    seed = int(seed) & (2**64 - 1)
    return (seed & 0xFFFFFFFF, seed >> 32)


def u52(a: int, b: int) -> float:
    """Uniform on (0, 1) from two 32-bit words: their top 26 bits each form a
    52-bit integer m, and (m + 0.5) / 2^52 is exact in FP64, so the result is
    never 0 or 1."""
    return ((a >> 6) * 67108864.0 + (b >> 6) + 0.5) / 4503599627370496.0


def box_muller(u1: float, u2: float):
    r = math.sqrt(-2.0 * math.log(u1))
    return r * math.cos(2.0 * math.pi * u2), r * math.sin(2.0 * math.pi * u2)


def normals4(seed: int, chain: int, it: int):
    key = seed_key(seed)
    z = []
    for s in (0, 1):
        w = philox((it & 0xFFFFFFFF, it >> 32, chain, s), key)
        z.extend(box_muller(u52(w[0], w[1]), u52(w[2], w[3])))
    return np.array(z)


def uniforms2(seed: int, chain: int, it: int):
    w = philox((it & 0xFFFFFFFF, it >> 32, chain, 2), seed_key(seed))
    return u52(w[0], w[1]), u52(w[2], w[3])


def log_prior(psi) -> float:
    """Eq. prior: independent Normal(mu, sigma) on each log-rate."""
    psi = np.asarray(psi, dtype=np.float64)
    return float(np.sum(-0.5 * ((psi - PRIOR_MU) / PRIOR_SIGMA) ** 2
                        - math.log(PRIOR_SIGMA * math.sqrt(2.0 * math.pi))))


def cholesky_lower(Z):
    """Lower Cholesky factor of a symmetric positive definite matrix (textbook
    column-by-column recurrence)."""
    Z = np.asarray(Z, dtype=np.float64)
    n = Z.shape[0]
    L = np.zeros_like(Z)
    for j in range(n):
        d = Z[j, j] - np.dot(L[j, :j], L[j, :j])
        if d <= 0.0:
            raise ValueError("covariance is not positive definite")
        L[j, j] = math.sqrt(d)
        for i in range(j + 1, n):
            L[i, j] = (Z[i, j] - np.dot(L[i, :j], L[j, :j])) / L[j, j]
    return L


def propose(psi, L, seed: int, chain: int, it: int):
    """Eq. prop: Psi' ~ Normal(Psi, Z) as Psi + L z with Z = L L^T."""
    return np.asarray(psi, dtype=np.float64) + L @ normals4(seed, chain, it)


def mh_alpha(lp_prop: float, lp_cur: float) -> float:
    """Acceptance probability of SI A.1 for a symmetric proposal (Eq. prop):
    min(1, exp(lp_prop - lp_cur)) of the log-posteriors; a NaN or -inf
    proposal is rejected."""
    r = lp_prop - lp_cur
    if math.isnan(r) or lp_prop == -math.inf:
        return 0.0
    return min(1.0, math.exp(min(0.0, r)))


def da_alpha1(s_prop: float, s_cur: float, lprior_prop: float, lprior_cur: float) -> float:
    """First-stage acceptance probability of delayed acceptance: the MH ratio of
    the surrogate posterior (surrogate log-likelihood plus prior)."""
    r = (s_prop + lprior_prop) - (s_cur + lprior_cur)
    if math.isnan(r):
        return 0.0
    return min(1.0, math.exp(min(0.0, r)))


def da_alpha2(l_prop: float, l_cur: float, s_prop: float, s_cur: float) -> float:
    """Second-stage probability (Christen & Fox 2005): the exact posterior ratio
    divided by the surrogate posterior ratio (the prior cancels)."""
    r = (l_prop - l_cur) - (s_prop - s_cur)
    if math.isnan(r) or l_prop == -math.inf:
        return 0.0
    return min(1.0, math.exp(min(0.0, r)))


def adapt_Z(window, eps: float = EPS_COV):
    """Eq. update_S over the samples of ``window`` (rows = samples of Psi):
    Z = (2.38/eta)^2 [ (1/H') sum psi^T psi - psibar^T psibar + eps I ]."""
    X = np.asarray(window, dtype=np.float64)
    n, d = X.shape
    mean = X.mean(axis=0)
    cov = (X.T @ X) / n - np.outer(mean, mean)
    return (2.38 / d) ** 2 * (cov + eps * np.eye(d))


class MHState:
    """State of C chains: Psi, exact log-likelihood, surrogate value, iteration
    counters (the Philox counter of each chain)."""

    def __init__(self, psi0, loglik_fn, surrogate_fn=None, seed: int = 0):
        self.psi = np.array(psi0, dtype=np.float64)
        self.C = self.psi.shape[0]
        self.loglik_fn = loglik_fn
        self.surrogate_fn = surrogate_fn
        self.seed = int(seed)
        self.it = np.zeros(self.C, dtype=np.int64)
        self.ll = np.array([loglik_fn(p) for p in self.psi])
        self.s = (np.array([surrogate_fn(p) for p in self.psi]) if surrogate_fn else None)
        self.trace = [[] for _ in range(self.C)]
        self.n_accept = 0
        self.n_stage1 = 0
        self.n_exact = 0
        # (chain, iteration, |u - alpha|) of every accept decision: how close
        # each was to going the other way.
        self.margins = []
        self.evals = []  # (Psi', exact log-likelihood) of every exact evaluation, in order

    def plain_step(self, L):
        """One MH iteration of every chain (SI A.1)."""
        for c in range(self.C):
            h = int(self.it[c])
            prop = propose(self.psi[c], L, self.seed, c, h)
            lp = self.loglik_fn(prop)
            self.n_exact += 1
            self.evals.append((prop.copy(), lp))
            ua, _ = uniforms2(self.seed, c, h)
            alpha = mh_alpha(lp + log_prior(prop), self.ll[c] + log_prior(self.psi[c]))
            self.margins.append((c, h, abs(ua - alpha)))
            if ua < alpha:
                self.psi[c] = prop
                self.ll[c] = lp
                self.n_accept += 1
            self.it[c] = h + 1
            self.trace[c].append(self.psi[c].copy())

    def da_round(self, L, max_inner: int, target: int):
        """One round of delayed acceptance: every chain below ``target``
        iterations screens proposals with the surrogate until one passes the
        first stage (or ``max_inner`` were screened); the survivors are then
        decided with the exact log-likelihood.  Each screened proposal is one
        full DA iteration, whose outcome is appended to the trace."""
        for c in range(self.C):
            for _ in range(max_inner):
                if len(self.trace[c]) >= target:
                    break
                h = int(self.it[c])
                prop = propose(self.psi[c], L, self.seed, c, h)
                sp = self.surrogate_fn(prop)
                ua, ub = uniforms2(self.seed, c, h)
                a1 = da_alpha1(sp, self.s[c], log_prior(prop), log_prior(self.psi[c]))
                self.margins.append((c, h, abs(ua - a1)))
                self.it[c] = h + 1
                if not ua < a1:
                    self.trace[c].append(self.psi[c].copy())
                    continue
                self.n_stage1 += 1
                lp = self.loglik_fn(prop)
                self.n_exact += 1
                self.evals.append((prop.copy(), lp))
                a2 = da_alpha2(lp, self.ll[c], sp, self.s[c])
                self.margins.append((c, h, abs(ub - a2)))
                if ub < a2:
                    self.psi[c] = prop
                    self.ll[c] = lp
                    self.s[c] = sp
                    self.n_accept += 1
                self.trace[c].append(self.psi[c].copy())
                break


def autocovariance(x, maxlag: int):
    """gamma(k) = (1/n) sum_{t<n-k} (x_t - xbar)(x_{t+k} - xbar), k = 0..maxlag."""
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    d = x - x.mean()
    return np.array([np.dot(d[:n - k], d[k:]) / n for k in range(min(maxlag, n - 1) + 1)])


def ess_geyer(x) -> float:
    """Effective sample size n / tau with Geyer's initial monotone sequence:
    Gamma_m = gamma(2m) + gamma(2m+1) summed while positive, each clipped to the
    previous one, tau = (-gamma(0) + 2 sum_m Gamma_m) / gamma(0), floored at
    1 / log10(n)."""
    x = np.asarray(x, dtype=np.float64)
    n = len(x)
    if n < 4:
        return float(n)
    d = x - x.mean()
    gamma = lambda k: float(np.dot(d[:n - k], d[k:]) / n)
    g0 = gamma(0)
    if g0 <= 0.0:
        return float(n)
    total = -g0
    prev = np.inf
    m = 0
    while 2 * m + 1 < n:
        G = gamma(2 * m) + gamma(2 * m + 1)
        if G <= 0.0:
            break
        G = min(G, prev)
        total += 2.0 * G
        prev = G
        m += 1
    # Antithetic or very short series can drive the estimate to zero or below.
    # Vehtari, Gelman, Simpson, Carpenter & Buerkner (2021, Bayesian Analysis
    # 16(2), "Rank-normalization, folding, and localization"), whose ESS
    # estimator also sums Geyer's initial monotone sequence, bound the
    # estimate by S log10 S for S draws to keep antithetic chains stable; the
    # same bound here: tau >= 1 / log10(n), so ESS stays in (0, n log10 n].
    tau = max(total / g0, 1.0 / math.log10(n))
    return float(n / tau)


def ess_chains(trace):
    """Per-parameter ESS of independent chains: the sum of the chains' ESS.
    ``trace`` has shape (chains, samples, params)."""
    tr = np.asarray(trace, dtype=np.float64)
    C, S, P = tr.shape
    return np.array([sum(ess_geyer(tr[c, :, a]) for c in range(C)) for a in range(P)])


def moments_mcse(trace):
    """Pooled posterior mean and variance of each parameter with their Monte
    Carlo standard errors: sd / sqrt(ESS) for the mean, and the same estimator
    applied to the squared deviations for the variance."""
    tr = np.asarray(trace, dtype=np.float64)
    C, S, P = tr.shape
    flat = tr.reshape(C * S, P)
    mean = flat.mean(axis=0)
    var = flat.var(axis=0)
    ess_m = ess_chains(tr)
    sq = (tr - mean) ** 2
    ess_v = ess_chains(sq)
    var_sq = sq.reshape(C * S, P).var(axis=0)
    return {"mean": mean, "var": var, "mcse_mean": np.sqrt(var / ess_m),
            "mcse_var": np.sqrt(var_sq / ess_v), "ess": ess_m}
