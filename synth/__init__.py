"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds none of the R-MJP arithmetic (no generator matrix, no
uniformisation, no Poisson weights).  It only draws random numbers and follows
the paper's data recipes:

* workloads: the immigration-death, mRNA/protein, batched birth-death, random
  CSR and two-state promoter configurations, with shapes and distributions as
  described beside each function;
* snapshot data: each cell is an independent system started from the empty
  state and observed once at its time (Sec. 2.1.2 "snapshot data"; Sec. 3.1.1
  and 3.1.2 data recipes), simulated with Gillespie's direct method from the
  reaction lists Eqs. BD_chem, 2S_chem and the R -> R+P production of
  Eq. STS_chem (the paper's data are Gillespie-simulated).  Reactions that
  would leave the truncated box are blocked (reflecting boundary), the same
  convention the models use.

Seeds are fixed per configuration: ``seed = 20231205 + config number``.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 20231205
BD1D, TWOSTATE, MRNA_PROT2D, AUTOREG = 1, 2, 3, 5


def rng(config_no: int, salt: int = 0) -> np.random.Generator:
    return np.random.default_rng([SEED_BASE + config_no, salt])


def delta(n: int, s: int = 0) -> np.ndarray:
    r = np.zeros(n)
    r[s] = 1.0
    return r


def n_states(kind: int, dims) -> int:
    dims = list(dims)
    if kind == BD1D:
        return int(dims[0])
    if kind == TWOSTATE:
        return 2 * int(dims[0])
    if kind == MRNA_PROT2D:
        return int(dims[0]) * int(dims[1])
    raise ValueError(kind)


# --------------------------------------------------------------------------
# Workload configurations
# --------------------------------------------------------------------------

def bd_small():
    """Immigration-death, N = 64 (reflecting top), birth 10, death 1 per
    individual, rho0 = delta_0, times {0.1, 0.5, 1, 2, 5}, FP64."""
    return dict(kind=BD1D, dims=[64], theta=[10.0, 1.0], rho0=delta(64, 0),
                times=np.array([0.1, 0.5, 1.0, 2.0, 5.0]))


def mrna_protein():
    """mRNA/protein birth-death on a 200 x 200 box (N = 40,000), index
    n = m + 200 p; k_m = 20, gamma_m = 1, k_p = 5, gamma_p = 0.1;
    rho0 = delta(0,0); 20 log-spaced times in [0.1, 50]."""
    return dict(kind=MRNA_PROT2D, dims=[200, 200], theta=[20.0, 1.0, 5.0, 0.1],
                rho0=delta(40000, 0), times=np.logspace(np.log10(0.1), np.log10(50.0), 20))


def twostate_promoter(N_R: int = 300):
    """Two-state promoter (Sec. 3.1.2): theta = (beta, gamma, lambda_act,
    lambda_ina) = (100, 1, 2, 1), N = 2 N_R, 50 times evenly spaced in
    [0.5, 10], 100 cells per time, rho0 = (n_R = 0, active)."""
    return dict(kind=TWOSTATE, dims=[N_R], theta=[100.0, 1.0, 2.0, 1.0],
                rho0=delta(2 * N_R, 0), times=np.linspace(0.5, 10.0, 50), cells=100)


def autoreg():
    """Autoregulatory gene network (Sec. 3.1.3) with the paper's rates for
    (beta_R, beta_P) = (10, 0.5): gamma_R = 1, gamma_P = 0.1, lambda_act = 0.1,
    lambda_ina = 0.05; box N_R = 40, N_P = 120 (N = 9,600); 50 times evenly
    spaced in [0.5, 10], 120 cells each (6,000 observations); rho0 = (0, 0,
    active)."""
    return dict(kind=AUTOREG, dims=[40, 120], theta=[10.0, 0.5, 1.0, 0.1, 0.1, 0.05],
                rho0=delta(9600, 0), times=np.linspace(0.5, 10.0, 50), cells=120)


def jitter(theta, B: int, frac: float, gen: np.random.Generator) -> np.ndarray:
    """B parameter vectors theta * U(1 - frac, 1 + frac), component-wise."""
    theta = np.asarray(theta, dtype=np.float64)
    return theta[None, :] * gen.uniform(1.0 - frac, 1.0 + frac, size=(B, len(theta)))


def bd_batch(n: int = 4096, gen: np.random.Generator | None = None):
    """Uneven birth-death instances: N = floor(exp U(ln 100, ln 20000)),
    birth ~ U(1, N/4), death ~ U(0.5, 2), t ~ logU(0.01, 10), rho0 = delta_0."""
    gen = gen if gen is not None else rng(3)
    N = np.floor(np.exp(gen.uniform(np.log(100.0), np.log(20000.0), n))).astype(np.int64)
    lam = gen.uniform(1.0, N / 4.0)
    mu = gen.uniform(0.5, 2.0, n)
    t = np.exp(gen.uniform(np.log(0.01), np.log(10.0), n))
    return dict(N=N, theta=np.stack([lam, mu], axis=1), t=t)


def random_csr(N: int, deg: int, gen: np.random.Generator, max_exit: float | None = None,
               sigma: float = 1.0):
    """Random rate matrix: `deg` distinct uniform off-diagonal targets per row,
    lognormal(0, sigma) rates, optionally rescaled so that the largest row sum
    (exit rate) equals `max_exit`.  Rows = source states, columns ascending."""
    if N < deg + 1:
        raise ValueError("need N > deg")
    col = gen.integers(0, N - 1, size=(N, deg), dtype=np.int64)
    col += (col >= np.arange(N)[:, None])  # skip the diagonal
    col.sort(axis=1)
    while True:
        dup = np.any(col[:, 1:] == col[:, :-1], axis=1)
        if not dup.any():
            break
        rows = np.nonzero(dup)[0]
        c = gen.integers(0, N - 1, size=(len(rows), deg), dtype=np.int64)
        c += (c >= rows[:, None])
        c.sort(axis=1)
        col[rows] = c
    val = gen.lognormal(0.0, sigma, size=(N, deg))
    if max_exit is not None:
        val *= max_exit / val.sum(axis=1).max()
    row_ptr = np.arange(0, N * deg + 1, deg, dtype=np.int64)
    return row_ptr, col.reshape(-1).astype(np.int32), val.reshape(-1)


def csr_large(gen: np.random.Generator | None = None, N: int = 1 << 20, deg: int = 8):
    """N = 2^20 states, 8 distinct uniform targets per row, lognormal(0,1)
    rates scaled so the largest exit rate is 200, t = 1, rho0 uniform (1/1024)
    on 1024 distinct random states."""
    gen = gen if gen is not None else rng(4)
    row_ptr, col, val = random_csr(N, deg, gen, max_exit=200.0)
    rho0 = np.zeros(N)
    rho0[gen.choice(N, size=1024, replace=False)] = 1.0 / 1024.0
    return dict(row_ptr=row_ptr, col=col, val=val, rho0=rho0, times=np.array([1.0]))


# --------------------------------------------------------------------------
# Snapshot data by Gillespie's direct method (vectorised over cells)
# --------------------------------------------------------------------------

def _propensities(kind, dims, theta, st):
    """Reaction propensities (cells x R) and state changes for the reaction
    lists of Eqs. BD_chem / 2S_chem / the R->R+P production network."""
    if kind == BD1D:
        N = dims[0]
        b, g = theta
        n = st[:, 0]
        a = np.stack([np.where(n < N - 1, b, 0.0), g * n], axis=1)
        change = np.array([[1], [-1]])
    elif kind == TWOSTATE:
        NR = dims[0]
        b, g, lact, lina = theta
        n, s = st[:, 0], st[:, 1]
        a = np.stack([np.where((s == 0) & (n < NR - 1), b, 0.0), g * n,
                      np.where(s == 0, lina, 0.0), np.where(s == 1, lact, 0.0)], axis=1)
        change = np.array([[1, 0], [-1, 0], [0, 1], [0, -1]])
    elif kind == MRNA_PROT2D:
        M, P = dims
        km, gm, kp, gp = theta
        m, p = st[:, 0], st[:, 1]
        a = np.stack([np.where(m < M - 1, km, 0.0), gm * m,
                      np.where(p < P - 1, kp * m, 0.0), gp * p], axis=1)
        change = np.array([[1, 0], [-1, 0], [0, 1], [0, -1]])
    elif kind == AUTOREG:
        NR, NP = dims
        bR, bP, gR, gP, lact, lina = theta
        r, q, s = st[:, 0], st[:, 1], st[:, 2]
        a = np.stack([np.where((s == 0) & (r < NR - 1), bR, 0.0),            # transcription (active)
                      np.where(q < NP - 1, bP * r, 0.0),                     # translation
                      gR * r, gP * q,                                         # decays
                      np.where(s == 0, lina * q, 0.0),                        # active + P -> inactive
                      np.where((s == 1) & (q < NP - 1), lact, 0.0)], axis=1)  # inactive -> active + P
        change = np.array([[1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0], [0, -1, 1], [0, 1, -1]])
    else:
        raise ValueError(kind)
    return a, change


def gillespie_snapshots(kind: int, dims, theta, times, cells: int, gen: np.random.Generator):
    """For each time, `cells` independent systems started empty (and, for the
    two-state model, active) are simulated to that time; returns a list of
    integer arrays (cells x components): (n,), (n_R, sigma) or (m, p)."""
    times = np.asarray(times, dtype=np.float64)
    ncomp = 1 if kind == BD1D else (3 if kind == AUTOREG else 2)
    T = np.repeat(times, cells)
    st = np.zeros((len(T), ncomp), np.int64)
    tau = np.zeros(len(T))
    result = np.zeros_like(st)
    live = np.arange(len(T))
    while live.size:
        a, change = _propensities(kind, dims, theta, st[live])
        a0 = a.sum(axis=1)
        dt = np.where(a0 > 0, gen.exponential(1.0, live.size) / np.where(a0 > 0, a0, 1.0), np.inf)
        done = tau[live] + dt > T[live]
        result[live[done]] = st[live[done]]
        keep = ~done
        live, a, a0, dt = live[keep], a[keep], a0[keep], dt[keep]
        if not live.size:
            break
        tau[live] += dt
        u = gen.uniform(0.0, 1.0, live.size) * a0
        r = (np.cumsum(a, axis=1) <= u[:, None]).sum(axis=1)
        r = np.minimum(r, a.shape[1] - 1)
        st[live] += change[r]
    return [result[i * cells:(i + 1) * cells] for i in range(len(times))]


def snapshot_obs(kind: int, dims, samples):
    """Group the observations of each time by observed value.

    Returns a list over times of (members_list, counts).  For the two-state
    model only n_R is observed, so the group of value n_R holds the states
    n_R and n_R + N_R (Sec. 3.1.2); otherwise a group is one state."""
    out = []
    for smp in samples:
        if kind == BD1D:
            keys = smp[:, 0]
            vals, counts = np.unique(keys, return_counts=True)
            members = [np.array([v]) for v in vals]
        elif kind == TWOSTATE:
            NR = dims[0]
            vals, counts = np.unique(smp[:, 0], return_counts=True)
            members = [np.array([v, v + NR]) for v in vals]
        elif kind == AUTOREG:  # (n_R, n_P) observed, the gene state summed out (Sec. 3.1.3)
            NR, NP = dims
            vals, counts = np.unique(smp[:, 0] + NR * smp[:, 1], return_counts=True)
            members = [np.array([v, v + NR * NP]) for v in vals]
        else:
            M = dims[0]
            keys = smp[:, 0] + M * smp[:, 1]
            vals, counts = np.unique(keys, return_counts=True)
            members = [np.array([v]) for v in vals]
        out.append((members, counts.astype(np.float64)))
    return out


def flatten_obs(obs):
    """Flat arrays for the C ABI: gptr (ntimes+1), counts (G), mptr (G+1),
    members (int32)."""
    gptr, counts, mptr, members = [0], [], [0], []
    for mem_list, cnt in obs:
        for mem, c in zip(mem_list, cnt):
            members.extend(int(v) for v in mem)
            mptr.append(len(members))
            counts.append(float(c))
        gptr.append(len(counts))
    return (np.array(gptr, np.int64), np.array(counts, np.float64),
            np.array(mptr, np.int64), np.array(members, np.int32))
