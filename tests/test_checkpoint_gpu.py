"""Sampler checkpoint and resume (mjp_sampler_save / mjp_sampler_load): a run
interrupted halfway, saved, and restored into a freshly created sampler
continues exactly, bit for bit, as the uninterrupted run, for plain MH and
for delayed acceptance (the surrogate's parameters saved alongside); a
checkpoint of a sampler with another seed, a truncated or a damaged one is
refused and leaves the sampler as it was."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

THETA = np.array([20.0, 1.0, 2.0, 1.0])
NR = 40


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_05647_gb300 import build as lib_build
    lib_build.build()
    torch.cuda.set_device(0)


@pytest.fixture(scope="module")
def problem():
    import paper_2312_05647_gb300 as mjp
    times = np.linspace(0.5, 3.0, 5)
    dims = [NR]
    snaps = synth.gillespie_snapshots(synth.TWOSTATE, dims, THETA, times, 20, synth.rng(5, 31))
    obs = synth.snapshot_obs(synth.TWOSTATE, dims, snaps)
    model = mjp.Model(synth.TWOSTATE, dims, THETA, mjp.FP64)
    ob = mjp.Obs(2 * NR, times, obs, synth.delta(2 * NR, 0))
    return model, ob


C, CAP, EVCAP, SEED = 8, 64, 4096, 20261204
Z = np.diag([0.08, 0.05, 0.1, 0.1]) ** 2


def _psi0():
    return np.log(THETA) + 0.05 * np.random.default_rng(4).normal(size=(C, 4))


def _fresh(problem, seed=SEED):
    from paper_2312_05647_gb300 import surrogate as S
    model, ob = problem
    return S.Sampler(model, ob, C, capacity=CAP, eval_capacity=EVCAP, seed=seed)


def _started(problem):
    s = _fresh(problem)
    s.set_cov(Z)
    s.set_state(_psi0())
    return s


def _net():
    from paper_2312_05647_gb300 import surrogate as S
    net = S.MLP(seed=5)
    norm = np.concatenate([np.log(THETA), [0.1] * 4, [-300.0, 5.0]])
    net.set_params(norm=norm)
    return net


def _snapshot(s):
    ps, ll = s.get_state()
    st = s.stats()
    return ps, ll, s.trace(), st, s.get_cov()


def _evals_sorted(s):
    p, l = s.evals()
    rows = np.concatenate([p.cpu().numpy(), l.cpu().numpy()[:, None]], axis=1)
    return rows[np.lexsort(rows.T[::-1])]


@pytest.mark.parametrize("mode", ["plain", "da"])
def test_interrupted_run_resumes_bit_for_bit(problem, tmp_path, mode):
    iters = 30
    net = _net() if mode == "da" else None

    def run(s, n, nn):
        if mode == "plain":
            s.run_plain(n)
        else:
            s.run_da(nn, n, max_inner=6)

    a = _started(problem)
    run(a, iters, net)

    b = _started(problem)
    run(b, iters // 2, net)
    path = tmp_path / "ck.npz"
    b.checkpoint(path, net=net)

    c = _fresh(problem)            # no state, covariance or counters of its own
    net_c = _net() if mode == "da" else None
    if net_c is not None:
        net_c.set_params(params=np.zeros(17281, np.float32))  # overwritten by the resume
    c.resume(path, net=net_c)
    run(c, iters - iters // 2, net_c)

    pa, la, ta, sa, za = _snapshot(a)
    pc, lc, tc, sc, zc = _snapshot(c)
    np.testing.assert_array_equal(pa, pc)
    np.testing.assert_array_equal(la, lc)
    np.testing.assert_array_equal(za, zc)
    assert ta.shape == (C, iters, 4)
    np.testing.assert_array_equal(ta, tc)
    for key in ("iterations", "accepted", "stage1", "exact_evals", "kept", "evals_kept"):
        assert sa[key] == sc[key], key
    # Plain MH evaluates every chain each iteration, in chain order; delayed
    # acceptance batches the survivors of a round, so only the set of pairs
    # is the same.
    np.testing.assert_array_equal(_evals_sorted(a), _evals_sorted(c))
    if mode == "plain":
        assert sa["rounds"] == sc["rounds"] == iters


def test_checkpoint_of_another_sampler_or_damaged_is_refused(problem):
    from paper_2312_05647_gb300.capi import MJPError
    b = _started(problem)
    b.run_plain(5)
    ck = b.checkpoint()
    blob = ck["sampler"]

    c = _started(problem)
    before = _snapshot(c)

    other = _fresh(problem, seed=SEED + 1)
    with pytest.raises(MJPError) as e:
        other.resume(ck)
    assert e.value.code == -1
    for bad in (blob[: len(blob) // 2], np.concatenate([blob[:3], [blob[3] ^ 0xFF], blob[4:]]).astype(np.uint8)):
        with pytest.raises(MJPError) as e:
            c.resume({"sampler": bad})
        assert e.value.code == -1
    after = _snapshot(c)
    for x, y in zip(before[:3], after[:3]):
        np.testing.assert_array_equal(x, y)
    assert before[3] == after[3]
    # The intact checkpoint is accepted by a sampler created alike.
    c.resume(ck)
    np.testing.assert_array_equal(c.get_state()[0], b.get_state()[0])
