"""The beta+ spectrum variant of the decay on the GPU, through the C ABI: the
device's spectrum sampler, positron tracks against a brute-force expectation
and against the FP64 oracle, exact energy bookkeeping, launch-shape
independence and the argument checks."""
import math

import numpy as np
import pytest
from scipy import stats

from tests.parity_record import record
from tests.positron_expect import cube_positron_expectation

pytestmark = pytest.mark.gpu

F18_T_MAX = 0.6335     # MeV, 18F beta+ endpoint (nuclear data tables)
F18_T_MEAN = 0.2498    # MeV, 18F mean beta+ energy (nuclear data tables)
Q = 64e6               # tally units per MeV


def q_gpu(e):
    return int(np.rint(np.float32(e) * np.float32(6.4e7)))


@pytest.fixture(scope="module")
def nm():
    from paper_2111_11687_gb300 import build, nmdose
    build.build()
    nmdose.load()
    return nmdose


def test_device_spectrum_sampler(nm, orc):
    t = nm.nm_check_beta(F18_T_MAX, 8, 4_000_000, 5).astype(np.float64)
    assert 0.0 <= t.min() and t.max() <= F18_T_MAX
    assert abs(t.mean() / F18_T_MEAN - 1.0) < 0.005
    ref = orc.sample_beta(F18_T_MAX, 8, 400_000, 6)
    record("beta_spectrum", mean_rel_vs_tabulated=t.mean() / F18_T_MEAN - 1.0,
           mean_rel_vs_oracle=t.mean() / ref.mean() - 1.0, ks_p_vs_oracle=stats.ks_2samp(t[:400_000], ref).pvalue)
    assert stats.ks_2samp(t[:400_000], ref).pvalue > 1e-3
    # statistical-shape limit: Beta(3/2, 3) on [0, T_max]
    t0 = nm.nm_check_beta(1e-3, 0, 400_000, 7).astype(np.float64)
    assert stats.kstest(t0, stats.beta(1.5, 3.0, scale=1e-3).cdf).pvalue > 1e-3


def _cube(nm, rho, N, seed, **kw):
    n_side, vox = 5, 0.05
    den = np.full((n_side,) * 3, rho, np.float32)
    act = np.zeros((n_side,) * 3, np.float32)
    act[2, 2, 2] = 1.0
    gm = nm.Materials([0.0], [7.42], 0.0, 3.8)       # photons never interact
    with nm.Dose(den, np.zeros((n_side,) * 3, np.uint8), (vox,) * 3, gm, activity=act,
                 beta_max_mev=F18_T_MAX, beta_z=8, **kw) as d:
        d.run(N, seed=seed)
        return d.tally(), d.counters()


@pytest.mark.parametrize("rho", [1.0, 0.5])
def test_positron_tracks_in_a_cube(nm, orc, rho):
    N = 20_000_000
    t, c = _cube(nm, rho, N, 3)
    assert c["deposited"] + c["escaped"] + c["killed"] == c["emitted"]
    assert int(t.sum()) == c["deposited"] and c["killed"] == 0
    assert c["compton"] == 0 and c["photo"] == 0
    two_photons = 2 * q_gpu(0.511)
    # emitted = photons + the sampled positron energies (mean 0.2498 MeV)
    mean_t = (c["emitted"] - N * two_photons) / Q / N
    assert abs(mean_t / F18_T_MEAN - 1.0) < 0.005
    esc = (c["escaped"] - N * two_photons) / Q / N
    centre = t[2, 2, 2] / Q / N
    ts = orc.sample_beta(F18_T_MAX, 8, 2_000_000, 11)
    e_esc, e_centre = cube_positron_expectation(rho, 5, 0.05, ts, np.random.default_rng(12))
    for got, ref in ((esc, e_esc), (centre, e_centre)):
        sd = ref.std() * math.sqrt(1.0 / N + 1.0 / ref.size)
        # FP32 ranges and a table-interpolated spectrum: 0.3 % of the mean on top
        assert abs(got - ref.mean()) < 4.0 * sd + 3e-3 * ref.mean(), (got, ref.mean(), sd)
    # voxel by voxel against the oracle (its own sampler, traversal and FP64 ranges)
    No = 20_000_000
    r = orc.run(np.full((5,) * 3, float(rho)), np.zeros((5,) * 3, np.uint8),
                orc.Materials(z_over_a=[0.0], zeff=[7.42], pe_coeff=0.0),
                activity=np.pad(np.ones((1, 1, 1)), 2), spacing=(0.05,) * 3, n_hist=No, seed=4, batches=4,
                beta_max_mev=F18_T_MAX, beta_z=8)
    g = t / Q / N
    o = r.tally / Q / No
    # voxels that take at least 3e-4 MeV per decay (~80): two oracle runs of
    # 2e7 and 2e6 decays differ there by 0.6 % (median) and 4 % (worst)
    sel = o > 3e-4
    rel = np.abs(g[sel] / o[sel] - 1.0)
    record("positron_cube", voxels=int(sel.sum()), median_abs_rel=np.median(rel), max_abs_rel=rel.max(),
           escaped_rel_vs_expectation=esc / e_esc.mean() - 1, centre_rel_vs_expectation=centre / e_centre.mean() - 1)
    assert sel.sum() >= 27 and np.median(rel) < 0.01 and rel.max() < 0.04, (sel.sum(), rel)


def test_beta_phantom_matches_oracle(nm, orc):
    # Fine voxels (1 x 1 x 1.5 mm) so that the positron ranges (up to 2.3 mm in
    # tissue, ~9 mm in lung, tens of cm in air) move energy between voxels.
    from paper_2111_11687_gb300 import inputs
    from tests.test_gpu_parity import organ_check, voxel_criterion
    ph = inputs.adult_phantom(shape=(60, 64, 64), spacing=(0.1, 0.1, 0.15), seed=5)
    den = np.empty(ph.shape, np.float32)
    mat = np.empty(ph.shape, np.uint8)
    nm.nm_ct_to_phantom(ph.hu, den, mat)
    gmat = nm.Materials(inputs.MATERIAL_Z_OVER_A, inputs.MATERIAL_ZEFF, inputs.PE_COEFF, inputs.PE_EXP)
    N = 20_000_000
    # 40 batches on both sides: the oracle's batch sigma sets the combined one,
    # and with B batches |diff| / sigma follows a t law of ~B - 1 degrees of
    # freedom (P(|t| > 3) is 1.5 % at 9, 0.5 % at 39)
    with nm.Dose(den, mat, ph.spacing, gmat, activity=ph.activity, labels=ph.labels, n_labels=inputs.N_LABELS,
                 activity_bq=inputs.ACTIVITY_BQ, beta_max_mev=F18_T_MAX, beta_z=8, batches=40) as d:
        d.run(N, seed=9)
        g, sg = d.get()
        gm, ge, gs, cnt = d.organs()
        c = d.counters()
    assert c["deposited"] + c["escaped"] + c["killed"] == c["emitted"] and c["killed"] == 0
    oden, omat = orc.hu_to_phantom(ph.hu)
    om = orc.Materials(inputs.MATERIAL_Z_OVER_A, inputs.MATERIAL_ZEFF, inputs.PE_COEFF, inputs.PE_EXP)
    r = orc.run(oden, omat, om, activity=ph.activity, labels=ph.labels, n_labels=inputs.N_LABELS,
                spacing=ph.spacing, n_hist=1_000_000, seed=10, batches=40, activity_bq=inputs.ACTIVITY_BQ,
                beta_max_mev=F18_T_MAX, beta_z=8)
    body = den >= 0.1
    frac, nsel = voxel_criterion(g, sg, r.dose_rate, r.sigma, body)
    assert nsel > 1000 and frac >= 0.99, (frac, nsel)
    zmax, npow, worst, z, sel = organ_check(gm, gs, r.organ_mean, r.organ_sigma, cnt)
    assert zmax < 4.0, z[sel]


def test_beta_tallies_do_not_depend_on_the_launch_shape(nm):
    ref = None
    for kw in ({}, dict(block_threads=128, chunk=64, regroup=0), dict(block_threads=512, regroup=1,
                                                                       regroup_lanes=20)):
        t, c = _cube(nm, 1.0, 500_000, 21, **kw)
        if ref is None:
            ref = (t, c["emitted"], c["escaped"])
        else:
            np.testing.assert_array_equal(t, ref[0])
            assert (c["emitted"], c["escaped"]) == ref[1:]


def test_beta_argument_checks(nm):
    from paper_2111_11687_gb300.nmdose import NmError
    den = np.ones((4, 4, 4), np.float32)
    mat = np.zeros((4, 4, 4), np.uint8)
    act = np.ones((4, 4, 4), np.float32)
    gm = nm.Materials([0.5551], [7.42], 2e-9, 3.8)
    for kw in (dict(beta_max_mev=25.0), dict(beta_max_mev=-1.0), dict(beta_max_mev=0.6, beta_z=101),
               dict(beta_max_mev=0.6, warp_aggregate=1)):
        with pytest.raises(NmError):
            nm.Dose(den, mat, (0.1,) * 3, gm, activity=act, **kw)
    with nm.Dose(den, mat, (0.1,) * 3, gm, activity=act, beta_max_mev=0.6) as a, \
            nm.Dose(den, mat, (0.1,) * 3, gm, activity=act) as b:
        with pytest.raises(NmError):
            nm.nm_dose_run_batch([a.h, b.h], [1000, 1000], 1)
    with pytest.raises(NmError):
        nm.nm_check_beta(0.0, 8, 10, 1)
