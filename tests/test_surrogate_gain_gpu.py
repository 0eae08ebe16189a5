"""What the trained surrogate gains: on the two-state promoter data (N_R = 300,
50 times x 100 Gillespie cells, 256 chains), delayed acceptance with the
network trained on the adaptation phase's own exact evaluations needs fewer
exact log-likelihoods and gives more effective samples per second than plain
MH with the same frozen covariance, at matched posterior moments."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2312_05647_gb300 import build as lib_build
    lib_build.build()
    torch.cuda.set_device(0)


def test_surrogate_delayed_acceptance_beats_plain_mh():
    import paper_2312_05647_gb300 as mjp
    from paper_2312_05647_gb300 import surrogate as S
    cfg = synth.twostate_promoter()
    snaps = synth.gillespie_snapshots(cfg["kind"], cfg["dims"], cfg["theta"], cfg["times"], 100, synth.rng(5, 0))
    obs = synth.snapshot_obs(cfg["kind"], cfg["dims"], snaps)
    model = mjp.Model(cfg["kind"], cfg["dims"], cfg["theta"], mjp.FP32)
    ob = mjp.Obs(600, cfg["times"], obs, cfg["rho0"])
    C = 256
    r = S.da_vs_plain(model, ob, S.promoter_initial_psi(obs, C), C, iters=300, adapt=dict(max_iters=900))
    p, d = r["plain"], r["da"]
    # The network learned the log-likelihood surface of the adaptation phase.
    first, last = r["train_loss_first_last"]
    assert last < 0.05 * first
    # Same number of iterations; DA needed exact values only for stage-1 survivors.
    assert p["stats"]["iterations"] == d["stats"]["iterations"] == C * 300
    assert d["stats"]["exact_evals"] == d["stats"]["stage1"] < 0.8 * p["stats"]["exact_evals"]
    # Surrogate good enough that most survivors are accepted by the exact stage.
    assert d["stats"]["accepted"] > 0.8 * d["stats"]["stage1"]
    # Matched posterior moments (within 3 combined Monte Carlo standard errors) ...
    assert max(r["z_mean"]) < 3.0 and max(r["z_var"]) < 3.0, (r["z_mean"], r["z_var"])
    # ... and more effective samples per second.
    assert r["ess_per_s_ratio"] > 1.2, r["ess_per_s_ratio"]
    # The posterior sits near the generating rates (log(100), 0, log 2, 0).
    assert np.all(np.abs(d["mean"] - np.log(cfg["theta"])) < 0.3)
