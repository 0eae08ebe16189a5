"""Pins for the CPU oracle: each check ties it to something other than itself
(a closed form, an independent library routine, brute force, or a statistical
test), chosen so that a dropped term, a wrong sign or index, or a transposed
operand in the oracle fails at least one of them."""
import json
import math
import os

import mpmath
import numpy as np
import pytest
import scipy.linalg
from scipy import special, stats

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _random_csr(n, deg, seed, scale=1.0):
    gen = np.random.default_rng(seed)
    rp, col, val = synth.random_csr(n, deg, gen)
    return oracle.CSR(rp, col, val * scale)


# --------------------------------------------------------------------------
# Truncation rule and weights (Algorithm 2, Eq. R-MJP_expansion)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("x", [0.0, 0.3, 1.0, 7.9, 10.0, 79.2, 396.0, 1234.5678, 67529.0, 3.2e5])
def test_K_is_algorithm2_loop_exit(x):
    # Run Algorithm 2's while-loop header literally (increment after the test).
    k = 0
    while k <= x + 6.0 * math.sqrt(x):
        k += 1
    assert oracle.K_paper(x) == k


def test_K_for_immigration_death_times():
    cfg = synth.bd_small()
    csr = oracle.build_model(cfg["kind"], cfg["dims"], cfg["theta"])
    _, info = oracle.expv(csr, cfg["rho0"], cfg["times"])
    assert info["omega"] == pytest.approx(79.2, rel=1e-15)
    assert list(info["K"]) == [25, 78, 133, 234, 516]


@pytest.mark.parametrize("x", [0.5, 5.0, 79.2, 700.0, 4389.0, 67529.0])
def test_weights_match_scipy_poisson(x):
    K = oracle.K_paper(x)
    P, eps = oracle.poisson_weights(x, K)
    # 40-digit reference at a spread of k (scipy's own pmf loses ~x*1e-16).
    mpmath.mp.dps = 40
    ks = sorted({0, 1, K // 3, int(x), int(x) + 1, (int(x) + K) // 2, K - 1, K})
    for k in ks:
        ref = mpmath.e ** (-mpmath.mpf(x) + k * mpmath.log(x) - mpmath.loggamma(k + 1)) \
            if x > 0 else mpmath.mpf(1 if k == 0 else 0)
        if ref < mpmath.mpf("1e-300"):
            assert P[k] < 1e-290
        else:
            assert P[k] == pytest.approx(float(ref), rel=2e-13)
    # eps = 1 - sum_{k<=K} P_k is the upper regularised incomplete gamma tail.
    ref_eps = special.gammainc(K + 1, x)  # P(X > K) for X ~ Poisson(x)
    assert eps == pytest.approx(ref_eps, rel=1e-6, abs=1e-13)


def test_truncation_bound_claim():
    g = _golden("truncation_bound.json")
    xs = np.concatenate([np.linspace(10.0001, 100.0, 300), np.geomspace(100.0, 1e5, 200)])
    worst = 0.0
    for x in xs:
        K = oracle.K_paper(x)
        eps = special.gammainc(K + 1, x)
        worst = max(worst, eps)
        assert eps < g["eps_upper"]
    assert worst < 3e-7  # the literal rule is in fact much tighter


@pytest.mark.parametrize("x,tol", [(3.0, 1e-15), (79.2, 1e-15), (500.0, 1e-12), (1e4, 1e-11)])
def test_K_tol_is_smallest(x, tol):
    K = oracle.K_tol(x, tol)
    assert stats.poisson.sf(K, x) <= tol * (1 + 1e-6)
    assert stats.poisson.sf(K - 1, x) > tol * (1 - 1e-6)


# --------------------------------------------------------------------------
# Dense expm (own Pade-13) against scipy and closed forms
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,seed,scale", [(1, 0, 3.0), (2, 1, 1.0), (5, 2, 10.0), (20, 3, 0.5),
                                          (60, 4, 40.0)])
def test_expm_matches_scipy(n, seed, scale):
    gen = np.random.default_rng(seed)
    A = gen.normal(size=(n, n)) * scale / math.sqrt(n)
    E = oracle.expm(A)
    R = scipy.linalg.expm(A)
    assert np.abs(E - R).max() <= 1e-12 * max(1.0, np.abs(R).max()) * (1 + scale)


def test_expm_closed_forms():
    d = np.array([0.3, -2.0, 5.0])
    np.testing.assert_allclose(oracle.expm(np.diag(d)), np.diag(np.exp(d)), rtol=1e-13)
    N = np.array([[0.0, 2.0, 3.0], [0.0, 0.0, 4.0], [0.0, 0.0, 0.0]])
    np.testing.assert_allclose(oracle.expm(N), np.eye(3) + N + N @ N / 2, atol=1e-14)
    a = 7.5
    R = oracle.expm(np.array([[0.0, a], [-a, 0.0]]))
    np.testing.assert_allclose(R, [[math.cos(a), math.sin(a)], [-math.sin(a), math.cos(a)]],
                               atol=1e-13)


# --------------------------------------------------------------------------
# Series against closed forms and the dense exponential
# --------------------------------------------------------------------------

def test_immigration_death_closed_form_paper_mode():
    cfg = synth.bd_small()
    csr = oracle.build_model(cfg["kind"], cfg["dims"], cfg["theta"])
    out, info = oracle.expv(csr, cfg["rho0"], cfg["times"])
    for i, t in enumerate(cfg["times"]):
        ref = stats.poisson.pmf(np.arange(64), 10.0 * (1 - math.exp(-t)))
        assert np.abs(out[i] - ref).max() <= 2 * info["eps"][i] + 1e-14


def test_immigration_death_closed_form_tol_mode():
    cfg = synth.bd_small()
    csr = oracle.build_model(cfg["kind"], cfg["dims"], cfg["theta"])
    out, _ = oracle.expv(csr, cfg["rho0"], cfg["times"], mode=oracle.TOL, tol=1e-15)
    for i, t in enumerate(cfg["times"]):
        ref = stats.poisson.pmf(np.arange(64), 10.0 * (1 - math.exp(-t)))
        assert np.abs(out[i] - ref).max() <= 1e-12


@pytest.mark.parametrize("a,b,t", [(1.0, 2.0, 0.3), (5.0, 0.2, 1.7), (0.01, 3.0, 10.0)])
def test_two_state_ctmc_closed_form(a, b, t):
    csr = oracle.CSR([0, 1, 2], [1, 0], [a, b])
    rho0 = np.array([0.8, 0.2])
    pi = np.array([b, a]) / (a + b)
    ref = pi + (rho0 - pi) * math.exp(-(a + b) * t)
    out, info = oracle.expv(csr, rho0, [t])
    assert np.abs(out[0] - ref).max() <= 2 * info["eps"][0] + 1e-15
    out, _ = oracle.expv(csr, rho0, [t], mode=oracle.TOL, tol=1e-16)
    assert np.abs(out[0] - ref).max() <= 1e-13


@pytest.mark.parametrize("n,deg,seed,t", [(12, 3, 0, 0.7), (40, 5, 1, 2.0), (50, 2, 2, 0.05)])
def test_series_matches_dense_expm(n, deg, seed, t):
    csr = _random_csr(n, deg, seed)
    A = csr.dense_generator()
    gen = np.random.default_rng(seed + 100)
    rho0 = gen.random(n)
    rho0 /= rho0.sum()
    out, _ = oracle.expv(csr, rho0, [t], mode=oracle.TOL, tol=1e-16)
    ref_scipy = rho0 @ scipy.linalg.expm(A * t)
    ref_own = rho0 @ oracle.expm(A * t)
    assert np.abs(out[0] - ref_scipy).max() <= 1e-12
    assert np.abs(out[0] - ref_own).max() <= 1e-12


def test_series_paper_mode_within_bound_of_expm():
    csr = oracle.build_model(oracle.TWOSTATE, [30], [12.0, 1.0, 2.0, 1.0])
    A = csr.dense_generator()
    rho0 = synth.delta(60, 0)
    times = [0.1, 1.0, 3.0]
    out, info = oracle.expv(csr, rho0, times)
    for i, t in enumerate(times):
        ref = rho0 @ scipy.linalg.expm(A * t)
        assert np.abs(out[i] - ref).sum() <= 2 * info["eps"][i] + 1e-13


# --------------------------------------------------------------------------
# Structural properties: conservation, positivity, semigroup, Omega choice
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind,dims,theta", [
    (oracle.BD1D, [200], [60.0, 0.7]),
    (oracle.TWOSTATE, [80], [40.0, 1.0, 2.0, 1.0]),
    (oracle.MRNA_PROT2D, [20, 30], [5.0, 1.0, 2.0, 0.3]),
])
def test_conservation_and_positivity(kind, dims, theta):
    csr = oracle.build_model(kind, dims, theta)
    A = csr.dense_generator()
    assert np.abs(A.sum(axis=1)).max() <= 1e-12 * np.abs(A).max()  # rows of A sum to 0
    rho0 = synth.delta(csr.n, 0)
    out, _ = oracle.expv(csr, rho0, [0.05, 0.5, 2.0, 8.0])
    assert np.abs(out.sum(axis=1) - 1).max() <= 1e-13
    assert out.min() >= 0.0


def test_semigroup():
    csr = oracle.build_model(oracle.TWOSTATE, [60], [30.0, 1.0, 2.0, 1.0])
    rho0 = synth.delta(120, 0)
    s, t = 0.6, 1.3
    a, _ = oracle.expv(csr, rho0, [s + t], mode=oracle.TOL, tol=1e-16)
    b, _ = oracle.expv(csr, rho0, [s], mode=oracle.TOL, tol=1e-16)
    c, _ = oracle.expv(csr, b[0], [t], mode=oracle.TOL, tol=1e-16)
    assert np.abs(a[0] - c[0]).max() <= 1e-12


def test_omega_choice_does_not_matter():
    csr = oracle.build_model(oracle.MRNA_PROT2D, [15, 25], [6.0, 1.0, 1.5, 0.2])
    rho0 = synth.delta(csr.n, 0)
    a, ia = oracle.expv(csr, rho0, [0.4, 1.5], mode=oracle.TOL, tol=1e-16, omega_factor=1.1)
    b, ib = oracle.expv(csr, rho0, [0.4, 1.5], mode=oracle.TOL, tol=1e-16, omega_factor=2.0)
    assert ib["omega"] == pytest.approx(ia["omega"] * 2.0 / 1.1)
    assert np.abs(a - b).max() <= 1e-12


def test_degenerate_cases():
    cfg = synth.bd_small()
    csr = oracle.build_model(cfg["kind"], cfg["dims"], cfg["theta"])
    out, info = oracle.expv(csr, cfg["rho0"], [0.0, 1.0, 0.0])
    np.testing.assert_array_equal(out[0], cfg["rho0"])
    np.testing.assert_array_equal(out[2], cfg["rho0"])
    assert info["K"][0] == 1  # the literal rule runs one (weightless) jump at t = 0
    zero = oracle.CSR([0, 1, 2, 2], [1, 0], [0.0, 0.0])
    out, info = oracle.expv(zero, [0.25, 0.75, 0.0], [3.0])
    np.testing.assert_array_equal(out[0], [0.25, 0.75, 0.0])
    assert info["omega"] == 0.0
    with pytest.raises(ValueError):
        oracle.expv(csr, cfg["rho0"], [-1.0])


def test_max_exit_rates_golden():
    g = _golden("max_exit_rates.json")
    for N, b, gm in g["birth_death"]["cases"]:
        csr = oracle.build_model(oracle.BD1D, [N], [b, gm])
        e = oracle.max_exit(csr)
        assert e == pytest.approx(max(b + gm * (N - 2), gm * (N - 1)), rel=1e-15)
        assert e <= b + gm * (N - 1)
    for NR, b, gm, la, li in g["two_state"]["cases"]:
        csr = oracle.build_model(oracle.TWOSTATE, [NR], [b, gm, la, li])
        assert oracle.max_exit(csr) <= b + gm * (NR - 1) + la + li
    dm = g["dense_memory"]
    assert dm["N"] ** 2 * 8 > dm["bytes_lower"]


def test_two_state_reduces_to_birth_death():
    NR, beta, gamma = 50, 20.0, 1.0
    two = oracle.build_model(oracle.TWOSTATE, [NR], [beta, gamma, 0.5, 0.0])
    bd = oracle.build_model(oracle.BD1D, [NR], [beta, gamma])
    assert oracle.max_exit(two) == oracle.max_exit(bd)
    times = [0.2, 1.0, 4.0]
    a, _ = oracle.expv(two, synth.delta(2 * NR, 0), times, mode=oracle.TOL, tol=1e-16)
    b, _ = oracle.expv(bd, synth.delta(NR, 0), times, mode=oracle.TOL, tol=1e-16)
    assert np.abs(a[:, :NR] - b).max() <= 1e-13
    assert np.abs(a[:, NR:]).max() == 0.0


def test_mrna_protein_mean_odes():
    km, gm, kp, gp = 20.0, 1.0, 5.0, 0.1
    M, P = 50, 160
    csr = oracle.build_model(oracle.MRNA_PROT2D, [M, P], [km, gm, kp, gp])
    times = np.array([0.1, 0.5, 1.0])
    out, _ = oracle.expv(csr, synth.delta(M * P, 0), times, mode=oracle.TOL, tol=1e-15)
    m = np.tile(np.arange(M), P)
    p = np.repeat(np.arange(P), M)
    for i, t in enumerate(times):
        Em = km / gm * (1 - math.exp(-gm * t))
        a = kp * km / gm
        Ep = a * ((1 - math.exp(-gp * t)) / gp - (math.exp(-gm * t) - math.exp(-gp * t)) / (gp - gm))
        assert out[i] @ m == pytest.approx(Em, rel=1e-10)
        assert out[i] @ p == pytest.approx(Ep, rel=1e-10)


# --------------------------------------------------------------------------
# Generator build against Gillespie (oracle's own SSA and the data recipe)
# --------------------------------------------------------------------------

def _chi2_p(counts, prob):
    n = counts.sum()
    exp = prob * n
    keep = exp >= 5
    c = np.append(counts[keep], counts[~keep].sum())
    e = np.append(exp[keep], exp[~keep].sum())
    if e[-1] < 5:
        c[-2] += c[-1]
        e[-2] += e[-1]
        c, e = c[:-1], e[:-1]
    chi2 = ((c - e) ** 2 / e).sum()
    return stats.chi2.sf(chi2, len(c) - 1)


@pytest.mark.parametrize("kind,dims,theta,times", [
    (oracle.BD1D, [40], [15.0, 1.0], [0.3, 2.0]),
    (oracle.TWOSTATE, [40], [25.0, 1.0, 2.0, 1.0], [0.5, 3.0]),
    (oracle.MRNA_PROT2D, [12, 30], [4.0, 1.0, 2.0, 0.5], [0.7]),
])
def test_oracle_gillespie_histograms(kind, dims, theta, times):
    csr = oracle.build_model(kind, dims, theta)
    rho, _ = oracle.expv(csr, synth.delta(csr.n, 0), times, mode=oracle.TOL, tol=1e-14)
    counts = oracle.gillespie(csr, 0, times, 40000, seed=1234 + kind)
    for i in range(len(times)):
        assert _chi2_p(counts[i], rho[i]) > 1e-4


@pytest.mark.parametrize("kind,dims,theta,times", [
    (oracle.BD1D, [40], [15.0, 1.0], [0.3, 2.0]),
    (oracle.TWOSTATE, [40], [25.0, 1.0, 2.0, 1.0], [0.5, 3.0]),
    (oracle.MRNA_PROT2D, [12, 30], [4.0, 1.0, 2.0, 0.5], [0.7]),
])
def test_data_recipe_histograms(kind, dims, theta, times):
    csr = oracle.build_model(kind, dims, theta)
    rho, _ = oracle.expv(csr, synth.delta(csr.n, 0), times, mode=oracle.TOL, tol=1e-14)
    gen = np.random.default_rng(99 + kind)
    snaps = synth.gillespie_snapshots(kind, dims, theta, times, 20000, gen)
    for i, smp in enumerate(snaps):
        if kind == oracle.BD1D:
            idx = smp[:, 0]
        elif kind == oracle.TWOSTATE:
            idx = smp[:, 0] + dims[0] * smp[:, 1]
        else:
            idx = smp[:, 0] + dims[0] * smp[:, 1]
        counts = np.bincount(idx, minlength=csr.n)
        assert _chi2_p(counts, rho[i]) > 1e-4


# --------------------------------------------------------------------------
# Likelihood and prior
# --------------------------------------------------------------------------

def test_loglik_matches_per_observation_sum():
    cfg = synth.twostate_promoter(N_R=40)
    theta = [12.0, 1.0, 2.0, 1.0]
    times = cfg["times"][::10]
    gen = np.random.default_rng(5)
    snaps = synth.gillespie_snapshots(cfg["kind"], cfg["dims"], theta, times, 30, gen)
    obs = synth.snapshot_obs(cfg["kind"], cfg["dims"], snaps)
    csr = oracle.build_model(cfg["kind"], cfg["dims"], theta)
    rho, _ = oracle.expv(csr, cfg["rho0"], times)
    ll = oracle.loglik_from_rho(rho, obs)
    brute = 0.0
    for i, smp in enumerate(snaps):
        for nr, _sg in smp:  # the gene state is not observed: sum it out
            brute += math.log(rho[i, nr] + rho[i, nr + 40])
    assert ll == pytest.approx(brute, rel=1e-13)


def test_log_prior_matches_scipy():
    psi = np.array([0.3, -2.0, 4.6, 1.0])
    assert oracle.log_prior(psi) == pytest.approx(stats.norm.logpdf(psi, 1.0, 1e5).sum(), rel=1e-14)


# ---- fourth-order Runge-Kutta (Method #4, Sec. 2.3) --------------------------

@pytest.mark.parametrize("n,deg,seed", [(6, 3, 3), (15, 4, 4)])
def test_rk4_step_is_degree4_taylor_polynomial(n, deg, seed):
    # For a linear system one RK4 step (Eqs. RKstep, RKintermediate) is
    # rho (I + hA + (hA)^2/2 + (hA)^3/6 + (hA)^4/24), formed here from dense
    # matrix powers (a different sequence of operations).
    csr = _random_csr(n, deg, seed)
    A = csr.dense_generator()
    maxe = oracle.max_exit(csr)
    h = 0.7 / maxe  # one step: ceil(0.7) = 1
    gen = np.random.default_rng(seed)
    rho0 = gen.random(n)
    rho0 /= rho0.sum()
    out, info = oracle.rk4(csr, rho0, [h])
    assert list(info["steps"]) == [1] and info["max_exit"] == maxe
    hA = h * A
    P = np.eye(n)
    term = np.eye(n)
    for j in range(1, 5):
        term = term @ hA / j
        P = P + term
    assert np.abs(out[0] - rho0 @ P).max() <= 1e-15


@pytest.mark.parametrize("a,b,t", [(2.0, 3.0, 0.9), (0.5, 7.5, 3.3), (1.0, 1.0, 10.0)])
def test_rk4_two_state_iterate_closed_form(a, b, t):
    # Two states, rates a (0 -> 1) and b (1 -> 0): A has eigenvalues 0 and
    # -(a + b), so n RK4 steps give exactly pi + (rho0 - pi) R(z)^n with
    # z = -(a + b) h and R the degree-4 Taylor polynomial of exp.
    csr = oracle.build_model(oracle.BD1D, [2], [a, b])
    rho0 = np.array([0.9, 0.1])
    out, info = oracle.rk4(csr, rho0, [t])
    ns = math.ceil(t * max(a, b))
    assert list(info["steps"]) == [ns]
    z = -(a + b) * (t / ns)
    R = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    pi = np.array([b, a]) / (a + b)
    ref = pi + (rho0 - pi) * R ** ns
    assert np.abs(out[0] - ref).max() <= 1e-14
    # ... and within the method's error of the exact solution.
    exact = pi + (rho0 - pi) * math.exp(-(a + b) * t)
    assert np.abs(out[0] - exact).max() <= ns * abs(z) ** 5 / 120 + 1e-15


def test_rk4_times_order_conservation_and_restart():
    csr = oracle.build_model(oracle.MRNA_PROT2D, [15, 12], [6.0, 1.0, 2.0, 0.3])
    rho0 = synth.delta(180, 0)
    times = [0.7, 0.0, 0.25, 0.7, 1.5]
    out, info = oracle.rk4(csr, rho0, times)
    assert np.array_equal(out[1], rho0) and info["steps"][1] == 0
    assert np.array_equal(out[0], out[3])
    assert np.abs(out.sum(axis=1) - 1.0).max() <= 1e-13
    # Integrating on from rho(0.25) gives rho(0.7) bit for bit (the step rule
    # depends only on the interval).
    rest, _ = oracle.rk4(csr, out[2], [0.7 - 0.25])
    assert np.array_equal(rest[0], out[0])
    ref = rho0 @ scipy.linalg.expm(csr.dense_generator() * 1.5)
    assert np.abs(out[4] - ref).max() <= 1e-5


# ---- Krylov subspace steps (Method #5, Sec. 2.3) ------------------------------

@pytest.mark.parametrize("kind,dims,theta,t", [(oracle.BD1D, [12], [3.0, 1.0], 2.0), (oracle.BD1D, [2], [2.0, 5.0], 1.7),
                                               (oracle.TWOSTATE, [6], [4.0, 1.0, 2.0, 1.0], 0.9)])
def test_krylov_exact_when_the_space_is_whole(kind, dims, theta, t):
    # kappa >= N: the Krylov space of every step is the whole space (or an
    # invariant subspace found early), so each step is exact up to rounding.
    csr = oracle.build_model(kind, dims, theta)
    n = csr.n
    gen = np.random.default_rng(n)
    rho0 = gen.random(n)
    rho0 /= rho0.sum()
    out, info = oracle.krylov(csr, rho0, [t, 0.0, t / 3], kappa=20)
    ref = rho0 @ scipy.linalg.expm(csr.dense_generator() * t)
    assert np.abs(out[0] - ref).max() <= 1e-13
    assert np.array_equal(out[1], rho0) and info["steps"][1] == 0
    # Ascending times 0, t/3, t: cumulative steps ceil(interval x max_exit / (2 kappa)).
    s1 = math.ceil(t / 3 * info["max_exit"] / 40)
    assert list(info["steps"]) == [s1 + math.ceil((t - t / 3) * info["max_exit"] / 40), 0, s1]


def test_krylov_one_vector_step_closed_form():
    # kappa = 1: H = <q, q A> (a Rayleigh quotient) and one step is
    # rho exp(dt rho A rho^T / rho rho^T).
    csr = _random_csr(9, 3, 7)
    A = csr.dense_generator()
    maxe = oracle.max_exit(csr)
    t = 1.5 / maxe  # kappa = 1: ceil(1.5 / 2) = 1 step
    rho0 = np.random.default_rng(7).random(9)
    out, info = oracle.krylov(csr, rho0, [t], kappa=1)
    assert list(info["steps"]) == [1]
    ray = rho0 @ A @ rho0 / (rho0 @ rho0)
    assert np.abs(out[0] - rho0 * math.exp(t * ray)).max() <= 1e-15


def test_krylov_immigration_death_accuracy():
    cfg = synth.bd_small()
    csr = oracle.build_model(oracle.BD1D, [64], cfg["theta"])
    out, info = oracle.krylov(csr, cfg["rho0"], cfg["times"])
    ref, _ = oracle.expv(csr, cfg["rho0"], cfg["times"], mode=oracle.TOL, tol=1e-16)
    assert list(info["steps"]) == [1, 2, 3, 5, 11]
    assert np.abs(out - ref).max() <= 1e-9


# ---- autoregulatory gene network (Sec. 3.1.3, Eq. STS_chem) ------------------

def _autoreg_generator_from_reactions(NR, NP, th):
    """Dense A built straight from the reaction list of Eq. STS_chem (state
    tuples, reflecting box): an independent construction of the model."""
    bR, bP, gR, gP, la, li = th
    idx = lambda r, p, s: r + NR * p + NR * NP * s
    N = 2 * NR * NP
    A = np.zeros((N, N))
    for s in (0, 1):
        for p in range(NP):
            for r in range(NR):
                moves = []
                if s == 0:
                    moves.append(((r + 1, p, 0), bR))          # transcription
                    moves.append(((r, p - 1, 1), li * p))      # sigma_act + P -> sigma_ina
                else:
                    moves.append(((r, p + 1, 0), la))          # sigma_ina -> sigma_act + P
                moves.append(((r, p + 1, s), bP * r))          # translation
                moves.append(((r - 1, p, s), gR * r))          # R decay
                moves.append(((r, p - 1, s), gP * p))          # P decay
                for (r2, p2, s2), rate in moves:
                    if 0 <= r2 < NR and 0 <= p2 < NP and rate > 0:
                        A[idx(r, p, s), idx(r2, p2, s2)] += rate
    A[np.diag_indices(N)] = -A.sum(axis=1)
    return A


@pytest.mark.parametrize("NR,NP,th", [(4, 3, [2.5, 0.125, 1.0, 0.1, 0.1, 0.05]), (5, 6, [20.0, 1.0, 1.0, 0.1, 0.1, 0.05]),
                                      (2, 2, [1.0, 2.0, 3.0, 4.0, 5.0, 6.0])])
def test_autoreg_generator_matches_the_reactions(NR, NP, th):
    csr = oracle.build_model(oracle.AUTOREG, [NR, NP], th)
    A = csr.dense_generator()
    assert np.array_equal(A, _autoreg_generator_from_reactions(NR, NP, th))
    # The paper's bound on the largest exit rate (Sec. 3.1.3, one decay rate
    # gamma; the larger of gamma_R, gamma_P keeps it a bound).
    g = max(th[2], th[3])
    bound = th[0] + (th[1] + g) * (NR - 1) + (g + th[5]) * (NP - 1) + th[4]
    assert oracle.max_exit(csr) <= bound


def test_autoreg_without_switching_is_the_mrna_protein_model():
    # lambda_act = lambda_ina = 0 and an active start: the inactive block stays
    # empty and the active block evolves as the mRNA/protein box.
    NR, NP = 9, 7
    th = [5.0, 0.5, 1.0, 0.3, 0.0, 0.0]
    auto = oracle.build_model(oracle.AUTOREG, [NR, NP], th)
    mp = oracle.build_model(oracle.MRNA_PROT2D, [NR, NP], [th[0], th[2], th[1], th[3]])
    rho0 = np.zeros(2 * NR * NP)
    rho0[: NR * NP] = np.random.default_rng(3).random(NR * NP)
    rho0 /= rho0.sum()
    times = [0.4, 2.0]
    a, _ = oracle.expv(auto, rho0, times, mode=oracle.TOL, tol=1e-16)
    b, _ = oracle.expv(mp, rho0[: NR * NP], times, mode=oracle.TOL, tol=1e-16)
    assert np.abs(a[:, : NR * NP] - b).max() <= 1e-14
    assert not a[:, NR * NP:].any()


def test_autoreg_series_matches_expm_and_gillespie():
    NR, NP = 6, 8
    th = [4.0, 0.6, 1.0, 0.2, 0.8, 0.3]
    csr = oracle.build_model(oracle.AUTOREG, [NR, NP], th)
    rho0 = synth.delta(2 * NR * NP, 0)
    out, _ = oracle.expv(csr, rho0, [1.5], mode=oracle.TOL, tol=1e-16)
    ref = rho0 @ scipy.linalg.expm(csr.dense_generator() * 1.5)
    assert np.abs(out[0] - ref).max() <= 1e-12
    counts = oracle.gillespie(csr, 0, [1.5], 200000, 11)[0]
    keep = out[0] * 200000 > 20
    chi2 = np.sum((counts[keep] - 200000 * out[0][keep]) ** 2 / (200000 * out[0][keep]))
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-4


# --------------------------------------------------------------------------
# J-MJP state probabilities (Method #2, Algorithm 1)
# --------------------------------------------------------------------------

def _twostate_generator_from_reactions(NR, th):
    """Dense A of the two-state promoter (Sec. 3.1.2) from its reactions:
    state (n_R, sigma), index n_R + N_R sigma, sigma 0 active; reflecting top."""
    beta, gamma, la, li = th
    A = np.zeros((2 * NR, 2 * NR))
    for s in (0, 1):
        for r in range(NR):
            i = r + NR * s
            if s == 0 and r + 1 < NR:
                A[i, i + 1] += beta                    # transcription while active
            if r >= 1:
                A[i, i - 1] += gamma * r               # mRNA decay
            A[i, r + NR * (1 - s)] += li if s == 0 else la  # promoter switching
    A[np.diag_indices(2 * NR)] = -A.sum(axis=1)
    return A


def test_jmjp_two_state_ctmc_closed_form():
    # B = I + A / Omega for a 2-state chain (rates a, b) has eigenvalues 1 and
    # 1 - (a + b) / Omega: rho0 B^k = pi + (rho0 - pi)(1 - (a + b) / Omega)^k.
    a, b = 3.0, 0.7
    csr = oracle.CSR([0, 1, 2], [1, 0], [a, b])
    rho0 = np.array([0.25, 0.75])
    omega = 1.1 * max(a, b)
    pi = np.array([b, a]) / (a + b)
    ks = np.array([0, 1, 2, 7, 40, 3, 7])
    phi0 = oracle.jmjp_probs(csr, rho0, ks, [np.array([0])] * len(ks))
    phi1 = oracle.jmjp_probs(csr, rho0, ks, [np.array([1])] * len(ks))
    lam = 1.0 - (a + b) / omega
    for i, k in enumerate(ks):
        ref = pi + (rho0 - pi) * lam ** int(k)
        assert abs(phi0[i] - ref[0]) <= 1e-15 and abs(phi1[i] - ref[1]) <= 1e-15


@pytest.mark.parametrize("kind,dims,theta", [(oracle.BD1D, [30], [6.0, 0.8]), (oracle.TWOSTATE, [15], [8.0, 1.0, 2.0, 1.0])])
def test_jmjp_matches_dense_matrix_powers(kind, dims, theta):
    # rho0 B^k by repeated dense products, A built from the reactions.
    if kind == oracle.BD1D:
        n = dims[0]
        A = np.diag([theta[0]] * (n - 1), 1) + np.diag([theta[1] * r for r in range(1, n)], -1)
        A[np.diag_indices(n)] = -A.sum(axis=1)
    else:
        A = _twostate_generator_from_reactions(dims[0], theta)
    n = A.shape[0]
    csr = oracle.build_model(kind, dims, theta)
    omega = 1.1 * np.max(-np.diag(A))
    B = np.eye(n) + A / omega
    gen = np.random.default_rng(n)
    rho0 = gen.random(n)
    rho0 /= rho0.sum()
    ks = gen.integers(0, 120, size=25)
    ks[0] = 0
    groups = [gen.choice(n, size=gen.integers(1, 4), replace=False) for _ in ks]
    phi = oracle.jmjp_probs(csr, rho0, ks, groups)
    for i, k in enumerate(ks):
        ref = (rho0 @ np.linalg.matrix_power(B, int(k)))[groups[i]].sum()
        assert abs(phi[i] - ref) <= 1e-13
    assert phi[0] == rho0[groups[0]].sum()          # k = 0 reads rho0 itself


def test_jmjp_poisson_mixture_is_the_transient_distribution():
    # Sum_k Poisson(k; Omega t) rho0 B^k = rho0 exp(A t) (Eq. ME_uniform): the
    # J-MJP chain at every k, mixed with Poisson weights, is the ME solution.
    NR, th, t = 12, [5.0, 1.0, 2.0, 1.0], 1.3
    A = _twostate_generator_from_reactions(NR, th)
    csr = oracle.build_model(oracle.TWOSTATE, [NR], th)
    omega = 1.1 * np.max(-np.diag(A))
    rho0 = synth.delta(2 * NR, 0)
    kmax = int(omega * t + 40 * math.sqrt(omega * t)) + 40
    ks = np.repeat(np.arange(kmax + 1), 2 * NR)
    groups = [np.array([s]) for s in np.tile(np.arange(2 * NR), kmax + 1)]
    phi = oracle.jmjp_probs(csr, rho0, ks, groups).reshape(kmax + 1, 2 * NR)
    w = stats.poisson.pmf(np.arange(kmax + 1), omega * t)
    ref = rho0 @ scipy.linalg.expm(A * t)
    assert np.abs(w @ phi - ref).max() <= 1e-13


def test_jmjp_order_and_grouping():
    csr = oracle.build_model(oracle.TWOSTATE, [20], [30.0, 1.0, 2.0, 1.0])
    rho0 = synth.delta(40, 0)
    ks = np.array([50, 3, 50, 0, 17])
    groups = [np.array([r, r + 20]) for r in (4, 1, 9, 0, 12)]
    phi = oracle.jmjp_probs(csr, rho0, ks, groups)
    perm = np.array([4, 2, 0, 3, 1])
    phi_p = oracle.jmjp_probs(csr, rho0, ks[perm], [groups[i] for i in perm])
    assert np.array_equal(phi_p, phi[perm])
    # A group of both gene states is the sum of its two singletons.
    a = oracle.jmjp_probs(csr, rho0, ks, [g[:1] for g in groups])
    b = oracle.jmjp_probs(csr, rho0, ks, [g[1:] for g in groups])
    assert np.abs(a + b - phi).max() <= 1e-16
    # All states at any k: B is stochastic, the mass stays 1.
    allg = [np.arange(40)] * 3
    assert np.abs(oracle.jmjp_probs(csr, rho0, [0, 200, 1000], allg) - 1.0).max() <= 1e-13


def test_rk4_two_state_step_from_the_reactions():
    # One RK4 step on the two-state promoter equals the degree-4 Taylor
    # polynomial of hA with A built from the reaction list (not the oracle's CSR).
    NR, th = 9, [6.0, 0.7, 1.3, 0.4]
    A = _twostate_generator_from_reactions(NR, th)
    csr = oracle.build_model(oracle.TWOSTATE, [NR], th)
    maxe = float(np.max(-np.diag(A)))
    assert oracle.max_exit(csr) == maxe
    h = 0.9 / maxe
    rho0 = np.random.default_rng(9).random(2 * NR)
    rho0 /= rho0.sum()
    out, info = oracle.rk4(csr, rho0, [h])
    assert list(info["steps"]) == [1]
    P, term = np.eye(2 * NR), np.eye(2 * NR)
    for j in range(1, 5):
        term = term @ (h * A) / j
        P = P + term
    assert np.abs(out[0] - rho0 @ P).max() <= 1e-15
