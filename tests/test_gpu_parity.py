"""GPU transport against the FP64 oracle and against closed forms, through the
C ABI.  Monte Carlo results agree statistically, never bitwise (different RNGs
and different sampling algorithms): the voxel criterion is |gpu - oracle| <=
3 combined batch sigma in >= 99 % of the voxels above 5 % of the maximum dose,
and organ (or radial-shell) means must agree within 4 combined sigma and
within 1 % wherever the combined sigma makes a 1 % test meaningful."""
import math
import os

import numpy as np
import pytest

try:
    from parity_record import map_figures, record
except ImportError:   # imported as tests.test_gpu_parity
    from tests.parity_record import map_figures, record

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nm():
    from paper_2111_11687_gb300 import build, nmdose
    build.build()
    nmdose.load()
    return nmdose


def voxel_criterion(g, sg, o, so, mask):
    sel = mask & (o > 0.05 * o[mask].max())
    comb = np.sqrt(sg.astype(np.float64) ** 2 + so ** 2)
    ok = np.abs(g.astype(np.float64) - o) <= 3 * comb
    record("dose_map", **map_figures(g, o, so, sel, comb))
    return ok[sel].mean(), sel.sum()


def organ_check(gm, gs, om, os_, cnt, min_voxels=20):
    """Returns (max |z|, organs tested at 1 %, worst relative difference there)."""
    sel = (cnt >= min_voxels) & (om > 0)
    sel[0] = False
    comb = np.sqrt(gs ** 2 + os_ ** 2)
    with np.errstate(divide="ignore", invalid="ignore"):
        z = np.where(sel, (gm - om) / comb, 0.0)
        rel = np.where(sel, np.abs(gm / om - 1), 0.0)
    powered = sel & (3 * comb < 0.01 * om)
    record("organs", organs=int(sel.sum()), max_abs_z=np.abs(z[sel]).max(), powered=int(powered.sum()),
           max_abs_rel_powered=rel[powered].max() if powered.any() else None,
           median_abs_rel=np.median(rel[sel]), max_abs_rel=rel[sel].max())
    return np.abs(z[sel]).max(), powered.sum(), (rel[powered].max() if powered.any() else 0.0), z, sel


def shells(shape, spacing, center, width, n):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(*[(np.arange(k) + 0.5) * d for k, d in zip((nz, ny, nx), spacing[::-1])], indexing="ij")
    r = np.sqrt((x - center[0]) ** 2 + (y - center[1]) ** 2 + (z - center[2]) ** 2)
    lab = np.minimum((r / width).astype(np.int64) + 1, n)
    return lab.astype(np.uint8)


def test_point_source_in_water_matches_oracle(nm, orc):
    # 64^3 water voxels of 5 mm, isotropic 0.511 MeV point source at the centre
    # (a voxel corner), 1e6 histories, 10 batches; radial shells as labels give
    # the dose-distance curve with its batch sigma.
    from paper_2111_11687_gb300 import inputs
    cube = inputs.water_cube(64, 0.5)
    lab = shells(cube.density.shape, cube.spacing, cube.point, 0.5, 30)
    N = 1_000_000
    gm = nm.Materials(inputs.WATER_Z_OVER_A, inputs.WATER_ZEFF, inputs.PE_COEFF, inputs.PE_EXP)
    with nm.Dose(cube.density, cube.material, cube.spacing, gm, labels=lab, n_labels=30,
                 source_mode=nm.NM_SOURCE_POINT, point=cube.point, activity_bq=1.0) as d:
        d.run(N, seed=1)
        g, sg = d.get()
        gmean, _, gsig, cnt = d.organs()
        c = d.counters()
    assert c["emitted"] == c["deposited"] + c["escaped"] and c["killed"] == 0
    om = orc.Materials(inputs.WATER_Z_OVER_A, inputs.WATER_ZEFF, inputs.PE_COEFF, inputs.PE_EXP)
    r = orc.run(cube.density, cube.material, om, labels=lab, n_labels=30, spacing=cube.spacing,
                point=cube.point, n_hist=N, seed=1, batches=10)
    frac, nsel = voxel_criterion(g, sg, r.dose_rate, r.sigma, np.ones(g.shape, bool))
    assert nsel > 50 and frac >= 0.99, (frac, nsel)
    zmax, npow, worst, z, sel = organ_check(gmean, gsig, r.organ_mean, r.organ_sigma, cnt)
    assert zmax < 4.0, z
    # At 1e6 histories only the inner shells resolve 1 %; those must agree.
    assert npow >= 1 and worst < 0.01, (npow, worst)
    # deposited fraction of the emitted energy
    fg = c["deposited"] / c["emitted"]
    fo = r.counters["deposited"] / r.counters["emitted"]
    record("deposited_fraction", gpu=fg, oracle=fo, diff=fg - fo, bound=5 * math.sqrt(2) * 0.5 / math.sqrt(N))
    assert abs(fg - fo) < 5 * math.sqrt(2) * 0.5 / math.sqrt(N)


def _ray_box(d, lo, hi):
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        ta, tb = lo[None] * inv, hi[None] * inv
    tmin = np.where(np.isnan(np.minimum(ta, tb)), -np.inf, np.minimum(ta, tb))
    tmax = np.where(np.isnan(np.maximum(ta, tb)), np.inf, np.maximum(ta, tb))
    return np.maximum(tmin.max(1), 0.0), tmax.min(1)


def test_absorber_matches_first_collision_kernel(nm):
    # No electrons (Z/A = 0): only photoabsorption, so a voxel's expected tally
    # is N q(E) times the uncollided kernel mu e^(-mu r)/(4 pi r^2) integrated
    # over the voxel -- computed here by quadrature over directions.
    n_side, vox = 8, 0.5
    mu_t = 0.4
    zeff = 7.42
    pe = mu_t * 0.511 ** 3 / zeff ** 3.8
    m = nm.Materials([0.0], [zeff], pe, 3.8)
    den = np.ones((n_side,) * 3, np.float32)
    src = np.array([2.0, 2.0, 2.0])
    N = 8_000_000
    with nm.Dose(den, np.zeros(den.shape, np.uint8), (vox,) * 3, m, source_mode=nm.NM_SOURCE_POINT,
                 point=tuple(src), activity_bq=1.0) as d:
        d.run(N, seed=9)
        t = d.tally()
        c = d.counters()
    q = 32703998   # fixed-point 0.511 MeV in FP32: rint(0.511f * 6.4e7f)
    assert c["compton"] == 0 and c["emitted"] == N * q
    mm = 1500
    cc = (np.arange(mm) + 0.5) / mm * 2 - 1
    ph = (np.arange(2 * mm) + 0.5) / (2 * mm) * 2 * np.pi
    C_, P_ = np.meshgrid(cc, ph, indexing="ij")
    s = np.sqrt(1 - C_ ** 2)
    dirs = np.stack([s * np.cos(P_), s * np.sin(P_), C_], -1).reshape(-1, 3)
    z = []
    for ix in range(1, 7):
        for iy in range(2, 6):
            for iz in range(2, 6):
                lo = np.array([ix, iy, iz]) * vox - src
                t0, t1 = _ray_box(dirs, lo, lo + vox)
                ok = t1 > t0
                prob = np.where(ok, np.exp(-mu_t * t0) - np.exp(-mu_t * np.where(ok, t1, t0)), 0).mean()
                sd = math.sqrt(N * prob * (1 - prob)) * q
                z.append((t[iz, iy, ix] - N * prob * q) / sd)
    z = np.array(z)
    record("closed_form_kernel", voxels=len(z), max_abs_z=np.abs(z).max(), z_mean=z.mean(), z_rms=np.sqrt((z ** 2).mean()))
    assert np.all(np.abs(z) < 5), z
    assert abs(z.mean()) < 5 / math.sqrt(len(z))
    assert abs((z ** 2).mean() - 1) < 0.5


def _phantom(shape, spacing, seed):
    from paper_2111_11687_gb300 import inputs
    return inputs.adult_phantom(shape=shape, spacing=spacing, seed=seed)


def _gpu_phantom_run(nm, ph, N, seed, batches=10, **kw):
    from paper_2111_11687_gb300 import inputs
    den = np.empty(ph.shape, np.float32)
    mat = np.empty(ph.shape, np.uint8)
    nm.nm_ct_to_phantom(ph.hu, den, mat)
    gm = nm.Materials(inputs.MATERIAL_Z_OVER_A, inputs.MATERIAL_ZEFF, inputs.PE_COEFF, inputs.PE_EXP)
    with nm.Dose(den, mat, ph.spacing, gm, activity=ph.activity, labels=ph.labels,
                 n_labels=inputs.N_LABELS, activity_bq=inputs.ACTIVITY_BQ, batches=batches, **kw) as d:
        d.run(N, seed=seed)
        g, sg = d.get()
        org = d.organs()
        c = d.counters()
        t = d.tally()
    return den, mat, g, sg, org, c, t


def _oracle_phantom_run(orc, ph, N, seed, batches=10):
    from paper_2111_11687_gb300 import inputs
    den, mat = orc.hu_to_phantom(ph.hu)
    om = orc.Materials(inputs.MATERIAL_Z_OVER_A, inputs.MATERIAL_ZEFF, inputs.PE_COEFF, inputs.PE_EXP)
    return orc.run(den, mat, om, activity=ph.activity, labels=ph.labels, n_labels=inputs.N_LABELS,
                   spacing=ph.spacing, n_hist=N, seed=seed, batches=batches, activity_bq=inputs.ACTIVITY_BQ)


@pytest.mark.parametrize("kn_sampler", [0, 1])
def test_reduced_phantom_matches_oracle(nm, orc, kn_sampler):
    # The adult phantom's field of view on a 64x64x75 grid of 8x8x12 mm voxels:
    # several alias columns per warp, ragged grid edges, all five materials;
    # Compton angles from the tabulated inverse CDF (0) and from Kahn's sampler (1).
    from paper_2111_11687_gb300 import inputs
    ph = _phantom((75, 64, 64), (0.8, 0.8, 1.2), seed=21)
    N = 2_000_000
    den, mat, g, sg, (gm, ge, gs, cnt), c, _ = _gpu_phantom_run(nm, ph, N, seed=7, kn_sampler=kn_sampler)
    assert c["emitted"] == c["deposited"] + c["escaped"] and c["killed"] == 0
    r = _oracle_phantom_run(orc, ph, N, seed=8)
    body = den >= 0.1
    frac, nsel = voxel_criterion(g, sg, r.dose_rate, r.sigma, body)
    assert nsel > 1000 and frac >= 0.99, (frac, nsel)
    zmax, npow, worst, z, sel = organ_check(gm, gs, r.organ_mean, r.organ_sigma, cnt)
    assert zmax < 4.0, z[sel]
    assert npow >= 2 and worst < 0.01, (npow, worst)
    # Eq. 3 organ uncertainties agree to within their own scatter (both ~ 1/sqrt(N)).
    ok = sel & (cnt >= 100)
    record("eq3_organ_eps", organs=int(ok.sum()), max_abs_rel=np.abs(ge[ok] / r.organ_eps[ok] - 1).max(),
           median_abs_rel=np.median(np.abs(ge[ok] / r.organ_eps[ok] - 1)))
    assert np.all(np.abs(ge[ok] / r.organ_eps[ok] - 1) < 0.25)
    # the organ means and sigmas without Eq. 3 (no pass over the voxels) equal
    # the full pass's to FP32 rounding of the voxel doses
    with nm.Dose(den, mat, ph.spacing, nm.Materials(inputs.MATERIAL_Z_OVER_A, inputs.MATERIAL_ZEFF,
                                                    inputs.PE_COEFF, inputs.PE_EXP),
                 activity=ph.activity, labels=ph.labels, n_labels=inputs.N_LABELS, activity_bq=inputs.ACTIVITY_BQ,
                 kn_sampler=kn_sampler) as d:
        d.run(N, seed=7)
        fm, fe, fs, fc = d.organs(eps=False)
        m2, _, s2, c2 = d.organs()
        dfull, _ = d.get()
        donly = np.empty_like(dfull)
        nm.nm_dose_get(d.h, donly, None, None)
    np.testing.assert_array_equal(donly, dfull)              # the dose-only pass, bit for bit
    assert fe is None and np.array_equal(fc, c2)
    np.testing.assert_allclose(fm, m2, rtol=2e-6, atol=0)
    np.testing.assert_allclose(fs, s2, rtol=1e-4, atol=1e-30)


def _golden_organs():
    """The oracle's organ means and their batch sigma for the benchmark phantom
    (tests/golden/make_adult_phantom_organs.py, 1e9 oracle decays)."""
    path = os.path.join(os.path.dirname(__file__), "golden", "adult_phantom_organs_oracle.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    lab = np.array([int(r[0]) for r in rows])
    assert np.array_equal(lab, np.arange(len(rows)))
    return (np.array([float(r[1]) for r in rows]), np.array([float(r[2]) for r in rows]),
            np.array([int(r[3]) for r in rows]))


def test_full_size_phantom_every_organ_within_1_percent(nm):
    # The benchmark workload, 256x256x300 voxels of 2x2x3 mm: 1e10 GPU decays
    # against the stored 1e9-decay oracle means.  Every one of the 27 organs
    # must be within 1 % and within 4 combined sigma; an organ whose three
    # combined sigma reach 1 % makes the check underpowered, which fails too
    # rather than passing on the organs that are resolvable.
    from paper_2111_11687_gb300 import inputs
    om, os_, ocnt = _golden_organs()
    ph = _phantom((300, 256, 256), (0.2, 0.2, 0.3), seed=1)
    N = 10_000_000_000
    den, mat, g, sg, (gm, ge, gs, cnt), c, t = _gpu_phantom_run(nm, ph, N, seed=1, batches=20)
    assert c["emitted"] == c["deposited"] + c["escaped"] and c["killed"] == 0
    assert int(t.sum()) == c["deposited"]
    assert np.array_equal(cnt, ocnt)
    organs = np.arange(1, inputs.N_LABELS + 1)
    comb = np.sqrt(gs[organs] ** 2 + os_[organs] ** 2)
    under = organs[3 * comb >= 0.01 * om[organs]]
    assert under.size == 0, f"underpowered: organs {under.tolist()} have 3 combined sigma >= 1 %"
    rel = gm[organs] / om[organs] - 1
    z = (gm[organs] - om[organs]) / comb
    record("organs", organs=int(organs.size), max_abs_z=np.abs(z).max(), powered=int(organs.size),
           max_abs_rel_powered=np.abs(rel).max(), median_abs_rel=np.median(np.abs(rel)),
           max_abs_rel=np.abs(rel).max(), max_oracle_rel_sigma=(os_[organs] / om[organs]).max(),
           max_gpu_rel_sigma=(gs[organs] / gm[organs]).max(), gpu_decays=N)
    assert np.all(np.abs(rel) < 0.01), dict(zip(organs[np.abs(rel) >= 0.01].tolist(), rel[np.abs(rel) >= 0.01]))
    assert np.all(np.abs(z) < 4.0), dict(zip(organs[np.abs(z) >= 4].tolist(), z[np.abs(z) >= 4]))


def test_reduced_size_phantom_voxel_criterion(nm, orc):
    # The adult phantom on the 128x128x150 grid of 4x4x6 mm (half the
    # benchmark's resolution): 1e9 GPU decays against 1e8 oracle decays, both
    # in 20 batches; >= 99 % of the body voxels above 5 % of the maximum dose
    # within 3 combined sigma, and every organ within 4 combined sigma.
    ph = _phantom((150, 128, 128), (0.4, 0.4, 0.6), seed=1)
    den, mat, g, sg, (gm, ge, gs, cnt), c, _ = _gpu_phantom_run(nm, ph, 1_000_000_000, seed=5, batches=20)
    r = _oracle_phantom_run(orc, ph, 100_000_000, seed=6, batches=20)
    frac, nsel = voxel_criterion(g, sg, r.dose_rate, r.sigma, den >= 0.1)
    assert nsel > 20000 and frac >= 0.99, (frac, nsel)
    zmax, npow, worst, z, sel = organ_check(gm, gs, r.organ_mean, r.organ_sigma, cnt)
    assert sel.sum() >= 20 and zmax < 4.0, z[sel]
    assert worst < 0.01, (npow, worst)


def test_whole_body_phantom_organs_match_oracle(nm, orc):
    # The whole-body workload: 512x512x600 voxels of 1x1x3 mm with high-uptake
    # lesions (157 M voxels, 1.26 GB of int64 tallies).  1e9 GPU decays against
    # 2e6 oracle decays: organ means within 4 combined sigma, exact energy
    # bookkeeping; then a whole-volume denoiser pass (z slabs at this size) of a
    # fresh network, whose zero head returns its input.
    from paper_2111_11687_gb300 import inputs
    import torch
    ph = inputs.whole_body_phantom()
    N = 1_000_000_000
    den, mat, g, sg, (gm, ge, gs, cnt), c, t = _gpu_phantom_run(nm, ph, N, seed=1)
    assert c["emitted"] == c["deposited"] + c["escaped"] and c["killed"] == 0
    assert int(t.sum()) == c["deposited"]
    r = _oracle_phantom_run(orc, ph, 2_000_000, seed=2)
    zmax, npow, worst, z, sel = organ_check(gm, gs, r.organ_mean, r.organ_sigma, cnt)
    assert sel.sum() >= 20 and zmax < 4.0, z[sel]
    assert npow == 0 or worst < 0.01, (npow, worst)
    del t, r
    net = nm.Denoiser(patch=32, batch=1, levels=4, base_width=16, seed=1)
    dose = torch.from_numpy(g).cuda()
    out = torch.empty_like(dose)
    net.apply(dose, torch.from_numpy(den).cuda(), torch.from_numpy(ph.activity).cuda(), out)
    o = out.cpu().numpy()
    net.close()
    assert np.all(np.isfinite(o))
    body = den >= 0.1
    assert np.allclose(o[body], g[body], rtol=1e-2, atol=1e-3 * g[body].max())


def test_rayleigh_on_matches_oracle(nm, orc):
    # The optional Rayleigh events (R4: mu_R/rho = c_R Zeff^2 / E^2, Thomson
    # angles) on the reduced phantom with a coefficient large enough that they
    # matter (mu_R is about 0.4 mu_c at 511 keV and grows as 1/E^2 below it):
    # voxel criterion and organs against the oracle with Rayleigh on, the
    # Rayleigh-to-Compton event ratio within binomial scatter, and no device
    # flag (the Thomson rejection loop never hits its trial limit).
    from paper_2111_11687_gb300 import inputs
    ph = _phantom((75, 64, 64), (0.8, 0.8, 1.2), seed=21)
    N = 2_000_000
    rc = 2.0e-4
    den = np.empty(ph.shape, np.float32)
    mat = np.empty(ph.shape, np.uint8)
    nm.nm_ct_to_phantom(ph.hu, den, mat)
    gmat = nm.Materials(inputs.MATERIAL_Z_OVER_A, inputs.MATERIAL_ZEFF, inputs.PE_COEFF, inputs.PE_EXP,
                        rayleigh_coeff=rc, rayleigh=1)
    with nm.Dose(den, mat, ph.spacing, gmat, activity=ph.activity, labels=ph.labels, n_labels=inputs.N_LABELS,
                 activity_bq=inputs.ACTIVITY_BQ, batches=10) as d:
        d.run(N, seed=7)
        g, sg = d.get()
        gm, ge, gs, cnt = d.organs()
        c = d.counters()
    assert c["device_status"] == 0 and c["rayleigh"] > 0.1 * c["compton"]
    assert c["emitted"] == c["deposited"] + c["escaped"] and c["killed"] == 0
    oden, omat = orc.hu_to_phantom(ph.hu)
    om = orc.Materials(inputs.MATERIAL_Z_OVER_A, inputs.MATERIAL_ZEFF, inputs.PE_COEFF, inputs.PE_EXP,
                       rayleigh_coeff=rc, rayleigh=1)
    r = orc.run(oden, omat, om, activity=ph.activity, labels=ph.labels, n_labels=inputs.N_LABELS,
                spacing=ph.spacing, n_hist=N, seed=8, batches=10, activity_bq=inputs.ACTIVITY_BQ)
    frac, nsel = voxel_criterion(g, sg, r.dose_rate, r.sigma, den >= 0.1)
    assert nsel > 1000 and frac >= 0.99, (frac, nsel)
    zmax, npow, worst, z, sel = organ_check(gm, gs, r.organ_mean, r.organ_sigma, cnt)
    assert zmax < 4.0, z[sel]
    # events per decay: Rayleigh / (Rayleigh + Compton) on both sides
    fg = c["rayleigh"] / (c["rayleigh"] + c["compton"])
    fo = r.counters["rayleigh"] / (r.counters["rayleigh"] + r.counters["compton"])
    ng = c["rayleigh"] + c["compton"]
    no = r.counters["rayleigh"] + r.counters["compton"]
    sd = math.sqrt(fg * (1 - fg) / ng + fo * (1 - fo) / no)
    record("rayleigh_fraction", gpu=fg, oracle=fo, diff_over_binomial_sigma=(fg - fo) / sd)
    # photon histories make events correlated within a decay: allow 8 binomial sigma
    assert abs(fg - fo) < 8 * sd, (fg, fo, sd)
