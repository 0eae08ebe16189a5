"""GPU parity of the surrogate and sampler kernels against the oracle
(oracle/mlp.py, oracle/mcmc.py): initialisation, forward pass, loss gradient,
Adam steps, ESS, and whole sampler trajectories (plain MH and delayed
acceptance) followed decision by decision."""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import mcmc, mlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_05647_gb300 import build as lib_build
    lib_build.build()
    torch.cuda.set_device(0)


def _sur():
    from paper_2312_05647_gb300 import surrogate
    return surrogate


def _net_params(seed, scale=0.25):
    """Oracle-side random parameters, rounded to FP32 (the kernels' weights)."""
    p = np.random.default_rng(seed).uniform(-scale, scale, mlp.NPAR)
    return p.astype(np.float32)


def _norm_vec(norm):
    return np.concatenate([norm["mu_x"], norm["sd_x"], [norm["mu_y"], norm["sd_y"]]])


def _norm_dict(v):
    return {"mu_x": v[0:4], "sd_x": v[4:8], "mu_y": float(v[8]), "sd_y": float(v[9])}


# --------------------------------------------------------------------------
# Network
# --------------------------------------------------------------------------

def test_init_matches_oracle_bitwise():
    S = _sur()
    net = S.MLP(seed=42)
    p, n = net.get_params()
    np.testing.assert_array_equal(p, mlp.init_params(42).astype(np.float32))
    np.testing.assert_array_equal(n, [0, 0, 0, 0, 1, 1, 1, 1, 0, 1])


def test_fit_norm_matches_oracle():
    S = _sur()
    gen = np.random.default_rng(1)
    psi = gen.normal([4.6, 0.0, 0.7, 0.0], [0.1, 0.2, 0.3, 0.05], size=(1001, 4))
    y = -20000.0 + 30.0 * gen.normal(size=1001)
    net = S.MLP(seed=1)
    net.fit_norm(psi, y)
    _, n = net.get_params()
    want = _norm_vec(mlp.fit_norm(psi, y))
    np.testing.assert_allclose(n, want, rtol=1e-13, atol=0)


@pytest.mark.parametrize("rows", [1, 31, 32, 33, 1000])
def test_forward_matches_oracle(rows):
    S = _sur()
    gen = np.random.default_rng(rows)
    p = _net_params(7)
    norm = {"mu_x": np.array([4.6, 0.0, 0.7, 0.0]), "sd_x": np.array([0.1, 0.2, 0.3, 0.05]),
            "mu_y": -20000.0, "sd_y": 40.0}
    psi = norm["mu_x"] + norm["sd_x"] * gen.normal(size=(rows, 4))
    net = S.MLP(seed=0)
    net.set_params(p, _norm_vec(norm))
    got = net.forward(psi)
    want = mlp.predict(p.astype(np.float64), norm, psi)
    f_err = np.abs(got - want) / norm["sd_y"]        # error in network units
    assert f_err.max() < 2e-5, f_err.max()


@pytest.mark.parametrize("rows", [200, 777, 5000])   # 8-, 16- and 32-row tiles, ragged last tile
def test_loss_gradient_matches_fp64_backprop(rows):
    S = _sur()
    gen = np.random.default_rng(100 + rows)
    p = _net_params(11)
    psi = gen.normal(size=(rows, 4))
    y = np.sin(psi[:, 0]) + psi[:, 1] * psi[:, 2] + 0.1 * gen.normal(size=rows)
    norm = mlp.fit_norm(psi, y)
    net = S.MLP(seed=0)
    net.set_params(p, _norm_vec(norm))
    loss, g = net.loss_grad(psi, y)
    xn = (psi - norm["mu_x"]) / norm["sd_x"]
    tn = (y - norm["mu_y"]) / norm["sd_y"]
    wl, wg = mlp.loss_grad(p.astype(np.float64), xn, tn)
    assert abs(loss - wl) <= 1e-5 * wl
    scale = np.abs(wg).max()
    assert np.abs(g - wg).max() <= 1e-3 * scale
    big = np.abs(wg) > 1e-2 * scale
    assert np.all(np.abs(g[big] - wg[big]) <= 1e-3 * np.abs(wg[big]))


def test_adam_steps_match_oracle():
    # Full batch, then minibatches drawn with the shared Philox rule.  A large
    # Adam eps keeps the update a smooth function of the gradient, so FP32
    # gradient rounding moves it by far less than the tolerance.
    S = _sur()
    gen = np.random.default_rng(5)
    psi = gen.normal(size=(300, 4))
    y = np.cos(psi[:, 0]) - psi[:, 3] ** 2
    p0 = _net_params(13)
    lr, eps = 1e-2, 1e-3
    for steps, batch in ((1, 300), (5, 64)):
        net = S.MLP(seed=0)
        net.set_params(p0, _norm_vec(mlp.fit_norm(psi, y)))
        losses = net.train(psi, y, steps=steps, batch=batch, lr=lr, eps=eps, seed=99, fit_norm=True)
        p_gpu, _ = net.get_params()
        p_or, _, l_or = mlp.train(p0.astype(np.float64), psi, y, steps=steps, batch=batch, lr=lr, seed=99, eps=eps)
        assert np.abs(p_gpu - p_or).max() <= 0.02 * lr * steps
        np.testing.assert_allclose(losses, l_or, rtol=1e-4)


def test_training_fits_a_smooth_function():
    S = _sur()
    gen = np.random.default_rng(12)
    psi = gen.normal(size=(4096, 4))
    y = -np.sum(psi**2, axis=1) + psi[:, 0] * psi[:, 1] + 1000.0
    net = S.MLP(seed=5)
    losses = net.train(psi, y, steps=1500, batch=512, lr=3e-3, seed=5)
    assert losses[-50:].mean() < 0.01 * losses[0]
    pred = net.forward(psi[:500])
    assert np.sqrt(np.mean((pred - y[:500]) ** 2)) < 0.1 * y.std()


def test_mlp_rejects_bad_arguments():
    S = _sur()
    from paper_2312_05647_gb300.capi import MJPError
    net = S.MLP(seed=0)
    bad = np.zeros(mlp.NPAR, np.float32)
    bad[5] = np.nan
    with pytest.raises(MJPError):
        net.set_params(bad)
    with pytest.raises(MJPError):
        net.set_params(None, np.array([0, 0, 0, 0, 1, 1, 0, 1, 0, 1.0]))
    with pytest.raises(MJPError):
        net.train(np.zeros((4, 4)), np.zeros(4), steps=0, batch=4)


# --------------------------------------------------------------------------
# Effective sample size
# --------------------------------------------------------------------------

def _ar1(gen, C, S, P, phi):
    x = np.empty((C, S, P))
    e = gen.normal(size=(C, S, P))
    x[:, 0] = e[:, 0]
    for t in range(1, S):
        x[:, t] = phi * x[:, t - 1] + e[:, t]
    return x + np.array([1.0, -2.0, 0.5, 3.0][:P])


@pytest.mark.parametrize("C,S,P,phi", [(6, 3000, 3, 0.7), (2, 30000, 1, 0.5), (3, 4, 2, 0.0)])
def test_ess_matches_oracle(C, S, P, phi):
    sur = _sur()
    tr = _ar1(np.random.default_rng(C * S), C, S, P, phi)
    got = sur.ess(tr)
    want = mcmc.moments_mcse(tr)
    for k_got, k_want in (("ess", "ess"), ("mean", "mean"), ("var", "var"), ("mcse_mean", "mcse_mean"),
                          ("mcse_var", "mcse_var")):
        np.testing.assert_allclose(got[k_got], want[k_want], rtol=1e-9, atol=1e-14)


# --------------------------------------------------------------------------
# Sampler trajectories
# --------------------------------------------------------------------------

THETA_SMALL = np.array([20.0, 1.0, 2.0, 1.0])
NR_SMALL = 60


def _small_problem():
    times = np.linspace(0.5, 3.0, 5)
    dims = [NR_SMALL]
    snaps = synth.gillespie_snapshots(synth.TWOSTATE, dims, THETA_SMALL, times, 20, synth.rng(5, 77))
    obs = synth.snapshot_obs(synth.TWOSTATE, dims, snaps)
    rho0 = synth.delta(2 * NR_SMALL, 0)

    def loglik_fn(psi):
        csr = oracle.build_model(synth.TWOSTATE, dims, np.exp(psi))
        return oracle.loglik(csr, rho0, times, obs)

    return dims, times, obs, rho0, loglik_fn


def _first_close_call(margins, C, thr):
    """Per chain, the first iteration whose accept decision was within thr of
    going the other way (infinity if none)."""
    first = np.full(C, np.iinfo(np.int64).max)
    for c, h, m in margins:
        if m < thr:
            first[c] = min(first[c], h)
    return first


def _compare_traces(gpu_tr, orc, C, iters, thr, tol):
    first = _first_close_call(orc.margins, C, thr)
    covered = 0
    for c in range(C):
        n = int(min(first[c], iters))
        ref = np.array(orc.trace[c][:n])
        if n:
            assert np.abs(gpu_tr[c, :n] - ref).max() <= tol, c
        covered += n
    assert covered >= 0.9 * C * iters, (covered, C * iters)


def _sampler(model, obs_h, C, cap, seed, psi0, Z):
    S = _sur()
    s = S.Sampler(model, obs_h, C, capacity=cap, eval_capacity=10000, seed=seed)
    s.set_cov(Z)
    s.set_state(psi0)
    return s


def test_plain_mh_trajectories_match_oracle():
    import paper_2312_05647_gb300 as mjp
    dims, times, obs, rho0, loglik_fn = _small_problem()
    C, iters, seed = 8, 40, 2024
    gen = np.random.default_rng(8)
    psi0 = np.log(THETA_SMALL) + 0.05 * gen.normal(size=(C, 4))
    Z = np.diag([0.08, 0.05, 0.1, 0.1]) ** 2
    model = mjp.Model(synth.TWOSTATE, dims, THETA_SMALL, mjp.FP64)
    ob = mjp.Obs(2 * NR_SMALL, times, obs, rho0)
    s = _sampler(model, ob, C, iters, seed, psi0, Z)
    ps, ll = s.get_state()
    np.testing.assert_array_equal(ps, psi0)
    for c in range(C):
        assert abs(ll[c] - loglik_fn(psi0[c])) <= 1e-12 * abs(ll[c])
    s.run_plain(iters)
    tr = s.trace()
    st = s.stats()

    orc = mcmc.MHState(psi0, loglik_fn, seed=seed)
    L = mcmc.cholesky_lower(Z)
    for _ in range(iters):
        orc.plain_step(L)
    _compare_traces(tr, orc, C, iters, thr=1e-8, tol=1e-10)
    first = _first_close_call(orc.margins, C, 1e-8)
    if np.all(first > iters):
        assert st["accepted"] == orc.n_accept
        assert st["iterations"] == C * iters and st["exact_evals"] == C * iters
        epsi, ell = s.evals()
        epsi, ell = epsi.cpu().numpy(), ell.cpu().numpy()
        assert len(ell) == len(orc.evals)
        np.testing.assert_allclose(epsi, np.array([e[0] for e in orc.evals]), rtol=0, atol=1e-10)
        np.testing.assert_allclose(ell, np.array([e[1] for e in orc.evals]), rtol=1e-12)
    assert 0.05 < st["accepted"] / st["iterations"] < 0.95

    # Eq. update_S over the newest 20 samples of every chain (the oracle's own trace).
    s.adapt_cov(20, 1e-12)
    window = np.concatenate([np.array(orc.trace[c][-20:]) for c in range(C)])
    np.testing.assert_allclose(s.get_cov(), mcmc.adapt_Z(window), rtol=1e-9, atol=1e-18)


def test_delayed_acceptance_trajectories_match_oracle():
    import paper_2312_05647_gb300 as mjp
    S = _sur()
    dims, times, obs, rho0, loglik_fn = _small_problem()
    C, iters, seed, max_inner = 8, 40, 77, 6
    gen = np.random.default_rng(9)
    psi0 = np.log(THETA_SMALL) + 0.05 * gen.normal(size=(C, 4))
    Z = np.diag([0.08, 0.05, 0.1, 0.1]) ** 2
    p32 = _net_params(21, scale=0.2)
    norm = {"mu_x": np.log(THETA_SMALL), "sd_x": np.array([0.1, 0.1, 0.1, 0.1]),
            "mu_y": loglik_fn(np.log(THETA_SMALL)), "sd_y": 2.0}
    net = S.MLP(seed=0)
    net.set_params(p32, _norm_vec(norm))
    model = mjp.Model(synth.TWOSTATE, dims, THETA_SMALL, mjp.FP64)
    ob = mjp.Obs(2 * NR_SMALL, times, obs, rho0)
    s = _sampler(model, ob, C, iters, seed, psi0, Z)
    s.run_da(net, iters, max_inner=max_inner)
    tr = s.trace()
    st = s.stats()

    sur_fn = lambda psi: float(mlp.predict(p32.astype(np.float64), norm, psi)[0])
    orc = mcmc.MHState(psi0, loglik_fn, sur_fn, seed=seed)
    L = mcmc.cholesky_lower(Z)
    while min(len(t) for t in orc.trace) < iters:
        orc.da_round(L, max_inner, iters)
    _compare_traces(tr, orc, C, iters, thr=1e-4, tol=1e-10)
    first = _first_close_call(orc.margins, C, 1e-4)
    if np.all(first > iters):
        assert st["stage1"] == orc.n_stage1 and st["exact_evals"] == orc.n_exact
        assert st["accepted"] == orc.n_accept
    assert st["iterations"] == C * iters
    assert st["exact_evals"] < C * iters   # the screen saved exact evaluations
    assert st["exact_evals"] == st["stage1"]
