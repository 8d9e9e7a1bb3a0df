"""Calibration of the voxel criterion the GPU parity tests apply (>= 99 % of
the voxels above 5 % of the maximum dose within three combined batch sigma):
applied to the FP64 oracle against itself with an independent seed at equal
counts, it passes with the margin the GPU shows, and the small negative mean
of (a - b) / sigma seen against the GPU appears here too.  That mean is a
property of the statistic, not of either side: the voxels are selected on one
run's noisy map, and a batch sigma grows with its batch mean for these skewed
per-voxel deposits."""
import numpy as np

from tests.parity_record import map_figures


def test_oracle_against_itself_passes_the_voxel_criterion(orc):
    from paper_2111_11687_gb300 import inputs
    ph = inputs.adult_phantom(shape=(75, 64, 64), spacing=(0.8, 0.8, 1.2), seed=21)
    den, mat = orc.hu_to_phantom(ph.hu)
    om = orc.Materials(inputs.MATERIAL_Z_OVER_A, inputs.MATERIAL_ZEFF, inputs.PE_COEFF, inputs.PE_EXP)

    def run(seed):
        return orc.run(den, mat, om, activity=ph.activity, labels=ph.labels, n_labels=inputs.N_LABELS,
                       spacing=ph.spacing, n_hist=2_000_000, seed=seed, batches=10, activity_bq=inputs.ACTIVITY_BQ)

    a, b = run(7), run(8)
    body = den >= 0.1
    sel = body & (b.dose_rate > 0.05 * b.dose_rate[body].max())
    comb = np.sqrt(a.sigma ** 2 + b.sigma ** 2)
    f = map_figures(a.dose_rate, b.dose_rate, b.sigma, sel, comb)
    assert f["voxels"] > 10000
    # the GPU against the oracle on this phantom: 0.9931 (table sampler), 0.9924 (Kahn)
    assert f["frac_within_3sigma"] >= 0.985, f
    assert -0.2 < f["z_mean"] < 0.0 and 0.95 < f["z_std"] < 1.15, f
    assert abs(f["mean_rel"]) < 0.005, f
    # organ means of the two runs agree within 4 combined sigma
    ok = (b.organ_mean > 0) & (np.arange(b.organ_mean.size) > 0)
    z = (a.organ_mean[ok] - b.organ_mean[ok]) / np.sqrt(a.organ_sigma[ok] ** 2 + b.organ_sigma[ok] ** 2)
    assert np.all(np.abs(z) < 4.0), z
