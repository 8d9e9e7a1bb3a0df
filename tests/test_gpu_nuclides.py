"""Other radionuclides (the paper's outlook, §4: 177Lu and 131I) and
multi-time-point dosimetry on the GPU, through the C ABI, against the FP64
oracle: beta- spectra of several branches tracked with their range, gamma
lines emitted from the decay site, no annihilation pair, exact energy
bookkeeping; the time-integrated activity element by element; and the
argument checks."""
import numpy as np
import pytest

from tests.parity_record import record
from tests.test_gpu_parity import organ_check, voxel_criterion
from tests.test_oracle_pins import I131, LU177

pytestmark = pytest.mark.gpu

# Main gamma lines (MeV, photons per decay; NNDC / ICRP 107).
LU177_GAMMA = [(0.2084, 0.104), (0.1130, 0.062)]
I131_GAMMA = [(0.3645, 0.815), (0.6370, 0.0716), (0.2843, 0.0612), (0.0802, 0.0262), (0.7229, 0.0177)]


@pytest.fixture(scope="module")
def nm():
    from paper_2111_11687_gb300 import build, nmdose
    build.build()
    nmdose.load()
    return nmdose


def _phantom():
    from paper_2111_11687_gb300 import inputs
    ph = inputs.adult_phantom(shape=(40, 36, 32), spacing=(1.6, 1.42, 2.25), seed=13)
    return ph


@pytest.mark.parametrize("nuc,gammas", [(LU177, LU177_GAMMA), (I131, I131_GAMMA)], ids=["177Lu", "131I"])
def test_beta_minus_emitter_matches_oracle(nm, orc, nuc, gammas):
    from paper_2111_11687_gb300 import inputs
    ph = _phantom()
    den = np.empty(ph.shape, np.float32)
    mat = np.empty(ph.shape, np.uint8)
    nm.nm_ct_to_phantom(ph.hu, den, mat)
    gm = nm.Materials(inputs.MATERIAL_Z_OVER_A, inputs.MATERIAL_ZEFF, inputs.PE_COEFF, inputs.PE_EXP)
    N, No = 20_000_000, 2_000_000
    kw = dict(no_annihilation=1, beta_electron=1, beta_z=nuc["z"], beta_branches=nuc["branches"],
              gamma_lines=gammas, positron_mev=0.0)
    with nm.Dose(den, mat, ph.spacing, gm, activity=ph.activity, labels=ph.labels, n_labels=inputs.N_LABELS,
                 batches=20, activity_bq=1.0, **kw) as d:
        d.run(N, seed=3)
        c = d.counters()
        g, sg = d.get()
        gmean, _, gsig, cnt = d.organs()
    assert c["emitted"] == c["deposited"] + c["escaped"] + c["killed"] and c["killed"] == 0
    assert c["device_status"] == 0
    # emitted energy per decay: mean beta energy of the device's table plus
    # the gamma lines at their yields (a few per mille statistically)
    per = c["emitted"] / 64e6 / N
    expect_gamma = sum(e * y for e, y in gammas)
    record("emitted_per_decay", mev=per, expected_mev=expect_gamma + nuc["mean"],
           rel=per / (expect_gamma + nuc["mean"]) - 1)
    assert abs(per - expect_gamma - nuc["mean"]) < 0.06 * nuc["mean"] + 0.01 * expect_gamma, per
    oden, omat = orc.hu_to_phantom(ph.hu)
    om = orc.Materials(inputs.MATERIAL_Z_OVER_A, inputs.MATERIAL_ZEFF, inputs.PE_COEFF, inputs.PE_EXP)
    r = orc.run(oden, omat, om, activity=ph.activity, labels=ph.labels, n_labels=inputs.N_LABELS,
                spacing=ph.spacing, n_hist=No, seed=4, batches=20, activity_bq=1.0, positron_mev=0.0,
                annihilation=False, beta_sign=-1, beta_z=nuc["z"], beta_branches=nuc["branches"],
                gamma_lines=gammas)
    body = oden >= 0.1
    frac, nsel = voxel_criterion(g, sg, r.dose_rate, r.sigma, body)
    assert nsel > 300 and frac >= 0.99, (frac, nsel)
    zmax, npow, worst, z, sel = organ_check(gmean, gsig, r.organ_mean, r.organ_sigma, cnt)
    assert sel.sum() >= 10 and zmax < 4.5, (zmax, z[sel])
    assert worst < 0.01 or npow == 0


def test_gamma_lines_and_no_annihilation_in_vacuum(nm):
    # No attenuation: every photon leaves, so escaped energy and escapes give
    # each line's count exactly; counts follow N x yield (binomial), and no
    # 0.511 MeV photon appears.  The constant local deposit stays in the tally.
    shape = (3, 3, 3)
    lines = [(0.2084, 0.104), (0.1130, 0.062)]
    gm = nm.Materials([0.0], [0.0], 0.0, 3.8)
    N = 4_000_000
    with nm.Dose(np.ones(shape, np.float32), np.zeros(shape, np.uint8), (1.0, 1.0, 1.0), gm,
                 activity=np.ones(shape, np.float32), no_annihilation=1, positron_mev=0.1336,
                 gamma_lines=lines) as d:
        d.run(N, seed=9)
        c = d.counters()
        t = d.tally()
    q = [int(np.rint(np.float32(e) * np.float32(6.4e7))) for e, _ in lines]
    esc, k = c["escaped"], c["escapes"]
    n2 = (esc - q[0] * k) / (q[1] - q[0])
    n1 = k - n2
    assert n1 == int(n1) and n2 == int(n2)
    for cnt, (_, y) in zip((n1, n2), lines):
        assert abs(cnt - N * y) < 4.5 * np.sqrt(N * y * (1 - y)), (cnt, N * y)
    qp = int(np.rint(np.float32(0.1336) * np.float32(6.4e7)))
    assert int(t.sum()) == N * qp == c["deposited"]
    assert c["emitted"] == N * qp + esc


def test_time_integrated_activity_matches_oracle(nm, orc):
    import torch
    rng = np.random.default_rng(2)
    shape = (7, 33, 65)
    t_h = [1.0, 4.0, 24.0, 72.0]
    maps = [rng.lognormal(0, 1, shape).astype(np.float32) * (rng.random(shape) < 0.8) for _ in t_h]
    ref = orc.time_integrated_activity(maps, t_h, 6.647 * 24)
    for dev in (False, True):
        ins = [torch.from_numpy(m).cuda() for m in maps] if dev else maps
        out = torch.empty(shape, dtype=torch.float32, device="cuda") if dev else np.empty(shape, np.float32)
        tot = nm.nm_time_integrated_activity(ins, t_h, 6.647 * 24, out)
        o = out.cpu().numpy() if dev else out
        # FP64 per voxel, one FP32 rounding at the end
        assert np.all(np.abs(o - ref) <= 2 ** -23 * np.abs(ref) + 1e-30)
        assert abs(tot / ref.sum() - 1) < 1e-12
    # argument checks: times out of order, negative activity, bad half-life
    out = np.empty(shape, np.float32)
    with pytest.raises(nm.NmError):
        nm.nm_time_integrated_activity(maps[:2], [4.0, 1.0], 6.0, out)
    bad = maps[0].copy()
    bad[0, 0, 0] = -1.0
    with pytest.raises(nm.NmError):
        nm.nm_time_integrated_activity([bad], [1.0], 6.0, out)
    with pytest.raises(nm.NmError):
        nm.nm_time_integrated_activity(maps[:1], [1.0], 0.0, out)


def test_absorbed_dose_from_time_points(nm):
    # The time-integrated activity as the decay map, its total as A of Eq. 1:
    # the dose map is then the absorbed dose (Gy) = dose rate per Bq x total.
    from paper_2111_11687_gb300 import inputs
    ph = _phantom()
    den = np.empty(ph.shape, np.float32)
    mat = np.empty(ph.shape, np.uint8)
    nm.nm_ct_to_phantom(ph.hu, den, mat)
    gm = nm.Materials(inputs.MATERIAL_Z_OVER_A, inputs.MATERIAL_ZEFF, inputs.PE_COEFF, inputs.PE_EXP)
    a1 = ph.activity
    a2 = (0.6 * ph.activity).astype(np.float32)
    cum = np.empty(ph.shape, np.float32)
    total = nm.nm_time_integrated_activity([a1, a2], [2.0, 24.0], 6.647 * 24, cum)
    assert total > 0
    with nm.Dose(den, mat, ph.spacing, gm, activity=cum, activity_bq=total) as d:
        d.run(2_000_000, seed=1)
        dose, _ = d.get()
    with nm.Dose(den, mat, ph.spacing, gm, activity=cum, activity_bq=1.0) as d:
        d.run(2_000_000, seed=1)
        per, _ = d.get()
    assert np.allclose(dose, per * total, rtol=1e-5, atol=0)


def test_radionuclide_argument_checks(nm):
    shape = (4, 4, 4)
    gm = nm.Materials([0.5551], [7.42])
    args = (np.ones(shape, np.float32), np.zeros(shape, np.uint8), (0.5, 0.5, 0.5), gm)
    act = np.ones(shape, np.float32)
    bad = [dict(gamma_lines=[(0.005, 0.5)]),            # below the photon cutoff
           dict(gamma_lines=[(1.2, 0.5)]),              # above 1 MeV (pair production absent)
           dict(gamma_lines=[(0.3, 1.5)]),              # yield above 1
           dict(beta_branches=[(0.5, -1.0)]),           # negative intensity
           dict(beta_branches=[(25.0, 1.0)]),           # endpoint out of range
           dict(no_annihilation=2)]
    for kw in bad:
        with pytest.raises(nm.NmError) as e:
            nm.Dose(*args, activity=act, **kw)
        assert e.value.status == nm.NM_ERR_ARG, kw
    # batched runs and the allocation-free tally refuse the nuclide variant
    with nm.Dose(*args, activity=act, gamma_lines=[(0.3, 0.5)]) as d, nm.Dose(*args, activity=act) as d2:
        with pytest.raises(nm.NmError):
            nm.nm_dose_run_batch([d, d2], [1000, 1000], 1)
