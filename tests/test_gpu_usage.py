"""The usage example of the documentation, on a reduced phantom: the calls a
user makes, in that order, must work as written."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_documented_usage_runs():
    import torch

    from paper_2111_11687_gb300 import build, inputs, nmdose as nm
    build.build()
    nm.load()
    ph = inputs.adult_phantom(shape=(75, 64, 64), spacing=(0.8, 0.8, 1.2), seed=2)
    den = torch.empty(ph.shape, dtype=torch.float32, device="cuda")
    mat = torch.empty(ph.shape, dtype=torch.uint8, device="cuda")
    nm.nm_ct_to_phantom(torch.from_numpy(ph.hu).cuda(), den, mat)
    mats = nm.Materials(inputs.MATERIAL_Z_OVER_A, inputs.MATERIAL_ZEFF, inputs.PE_COEFF, inputs.PE_EXP)
    with nm.Dose(den, mat, ph.spacing, mats, activity=ph.activity, labels=ph.labels,
                 n_labels=inputs.N_LABELS, activity_bq=inputs.ACTIVITY_BQ) as d:
        d.run(10_000_000, seed=1)
        dose, sigma = d.get()
        mean, eps, sig_mean, voxels = d.organs()
        image = d.checkpoint()
    assert dose.shape == ph.shape and np.isfinite(dose).all() and dose.max() > 0
    assert (sigma >= 0).all() and mean.shape == (inputs.N_LABELS + 1,)
    assert voxels[1:].sum() > 0 and image.dtype == np.uint8 and image.size > dose.size * 16
    with nm.Dose(den, mat, ph.spacing, mats, activity=ph.activity, labels=ph.labels,
                 n_labels=inputs.N_LABELS, activity_bq=inputs.ACTIVITY_BQ) as d2:
        d2.restore(image)
        np.testing.assert_array_equal(d2.get()[0], dose)
