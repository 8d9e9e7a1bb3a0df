"""What the trained denoiser gains over Monte Carlo without it.

Small version of the experiment (paper_2111_11687_gb300/experiment.py): the
U-Net is trained on pairs of engine-generated dose maps (low count -> high
count) of seeded adult phantoms on a coarse grid, then on held-out phantoms
the organ-mean error (Eq. 2) of the low-count map after the denoiser is
compared with that of the same low-count map without it, both against a
high-count reference of the same phantom."""
import numpy as np
import pytest

from tests.parity_record import record

pytestmark = pytest.mark.gpu


def test_denoiser_reduces_low_count_organ_error():
    from paper_2111_11687_gb300 import experiment
    out = experiment.run(train_n=10, test_n=3, shape=(75, 64, 64), spacing=(0.8, 0.8, 1.2), low=int(2e5),
                         high=int(2e7), ref=int(2e8), denoise_low=int(2e5), steps=1200, patch=32, batch=4, lr=2e-3,
                         workers=1, step_decays=int(2e5), max_decays=int(2e8), candidates=2)
    assert out["final_loss"] < out["first_loss"]
    # two candidates trained, the one kept has the lower held-out loss
    assert len(out["candidate_val_losses"]) == 2 and all(v > 0 for v in out["candidate_val_losses"])
    dn = np.array([c["denoiser_mean_err"] for c in out["cases"]])
    lo = np.array([c["low_mc_mean_err"] for c in out["cases"]])
    # the trained network must lower the mean organ error of its own input
    record("denoiser_gain", mean_organ_err_denoised=dn.mean(), mean_organ_err_low_count=lo.mean())
    assert dn.mean() < lo.mean(), (dn, lo)
    for c in out["cases"]:
        assert c["plain_mc_s"] is not None   # plain MC reaches 2 % within the budget
