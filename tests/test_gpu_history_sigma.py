"""History-by-history uncertainty on the GPU (the paper's method, §2.1;
Walters et al. 2002): every history's total deposit per voxel is squared into
an exact 128-bit sum.  Checked against the Bernoulli closed form (exact),
against the FP64 oracle's history-by-history sigma (statistically), and for
independence of the launch shape (bit-exact: the grouping per history does not
depend on the scheduling)."""
import numpy as np
import pytest

from tests.parity_record import record

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nm():
    from paper_2111_11687_gb300 import build, nmdose
    build.build()
    nmdose.load()
    return nmdose


@pytest.mark.parametrize("absorb", [False, True])
def test_history_sigma_bernoulli_closed_form(nm, absorb):
    # As the oracle's pin: each history deposits T in its decay voxel only, so
    # sigma / mean = sqrt((1 - p) / ((N - 1) p)) exactly, p the observed fraction.
    rng = np.random.default_rng(4)
    shape = (4, 4, 4)
    act = rng.uniform(0.2, 1.0, shape).astype(np.float32)
    if absorb:
        den = np.full(shape, 10.0, np.float32)
        gm = nm.Materials([0.0], [7.42], 1e3, 3.8)
    else:
        den = np.full(shape, 1e-9, np.float32)
        gm = nm.Materials([0.5551], [7.42], 2e-9, 3.8)
    N = 2_000_000
    with nm.Dose(den, np.zeros(shape, np.uint8), (1.0, 1.0, 1.0), gm, activity=act, history_sigma=1) as d:
        d.run(N, seed=9)
        dose, _ = d.get()
        sh = d.history_sigma()
        c = d.counters()
        t = d.tally()
    # fixed point of the GPU: rint of the FP32 product E * 6.4e7
    q = lambda e: int(np.rint(np.float32(e) * np.float32(6.4e7)))
    T = q(0.25) + (2 * q(0.511) if absorb else 0)
    assert c["deposited"] == N * T and c["history_splits"] == 0
    p = t / (T * N)
    expect = np.sqrt((1 - p) / ((N - 1) * p))
    ok = dose > 0
    record("history_sigma_closed_form", voxels=int(ok.sum()), max_abs_rel=np.abs(sh[ok] / dose[ok] / expect[ok] - 1).max())
    assert np.allclose(sh / dose, expect, rtol=2e-6, atol=0)


def _reduced(nm):
    from paper_2111_11687_gb300 import inputs
    ph = inputs.adult_phantom(shape=(75, 64, 64), spacing=(0.8, 0.8, 1.2), seed=21)
    den = np.empty(ph.shape, np.float32)
    mat = np.empty(ph.shape, np.uint8)
    nm.nm_ct_to_phantom(ph.hu, den, mat)
    gm = nm.Materials(inputs.MATERIAL_Z_OVER_A, inputs.MATERIAL_ZEFF, inputs.PE_COEFF, inputs.PE_EXP)
    return ph, den, mat, gm


def test_history_sigma_matches_oracle(nm, orc):
    from paper_2111_11687_gb300 import inputs
    ph, den, mat, gm = _reduced(nm)
    N = 2_000_000
    with nm.Dose(den, mat, ph.spacing, gm, activity=ph.activity, activity_bq=inputs.ACTIVITY_BQ,
                 history_sigma=1) as d:
        d.run(N, seed=7)
        g, sg = d.get()
        gh = d.history_sigma()
        c = d.counters()
    # a history that scatters through more than 16 voxels is squared in parts
    # (exact for every voxel it does not revisit after the split); rare
    assert c["history_splits"] < 0.01 * N
    oden, omat = orc.hu_to_phantom(ph.hu)
    om = orc.Materials(inputs.MATERIAL_Z_OVER_A, inputs.MATERIAL_ZEFF, inputs.PE_COEFF, inputs.PE_EXP)
    r = orc.run(oden, omat, om, activity=ph.activity, spacing=ph.spacing, n_hist=N, seed=8, batches=10,
                activity_bq=inputs.ACTIVITY_BQ, history_sigma=True)
    sel = (den >= 0.1) & (r.dose_rate > 0.05 * r.dose_rate[den >= 0.1].max())
    # relative sigmas: the two runs differ in their samples, not in what they estimate
    rg = gh[sel] / g[sel]
    ro = r.sigma_history[sel] / r.dose_rate[sel]
    ratio = rg / ro
    record("history_sigma_vs_oracle", voxels=int(sel.sum()), median_ratio=np.median(ratio),
           frac_within_20pct=np.mean(np.abs(ratio - 1) < 0.2), median_batch_over_history=np.median(sg[sel] / gh[sel]))
    assert sel.sum() > 1000
    assert abs(np.median(ratio) - 1) < 0.03, np.median(ratio)
    assert np.mean(np.abs(ratio - 1) < 0.2) > 0.95
    # history-by-history and batch sigma estimate the same quantity
    assert abs(np.median(sg[sel] / gh[sel]) - 1) < 0.05


def test_history_sigma_is_independent_of_launch_shape(nm):
    from paper_2111_11687_gb300 import inputs
    ph, den, mat, gm = _reduced(nm)
    out = []
    for kw in (dict(block_threads=128, chunk=64, regroup=0), dict(block_threads=512, chunk=1024, regroup=1)):
        with nm.Dose(den, mat, ph.spacing, gm, activity=ph.activity, history_sigma=1, warp_aggregate=0, **kw) as d:
            d.run(500_000, seed=3)
            out.append((d.tally(), d.history_sigma()))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


def test_history_sigma_state_errors(nm):
    from paper_2111_11687_gb300 import inputs
    ph, den, mat, gm = _reduced(nm)
    with nm.Dose(den, mat, ph.spacing, gm, activity=ph.activity) as d:
        d.run(10_000, seed=1)
        with pytest.raises(nm.NmError):
            d.history_sigma()
    with nm.Dose(den, mat, ph.spacing, gm, activity=ph.activity, history_sigma=1) as d:
        with pytest.raises(nm.NmError):
            nm.nm_dose_run_batch([d.h], [1000], 1)
        with pytest.raises(nm.NmError):
            nm.Dose(den, mat, ph.spacing, gm, activity=ph.activity, history_sigma=1, warp_aggregate=1)
