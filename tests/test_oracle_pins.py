"""Pins of the FP64 oracle against closed forms, invariants, brute force and the
paper's printed numbers.  CPU only.

Each test is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign or index, a transposed operand, a wrong unit) fails at least one of
them.  None of them compares the oracle with itself.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, stats

from tests.positron_expect import cube_positron_expectation

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ME = 0.51099895            # m_e c^2, MeV (CODATA 2018)
RE = 2.8179403262e-13      # classical electron radius, cm
SIGMA_T = 8.0 * math.pi * RE * RE / 3.0   # Thomson cross section


def water(orc, **kw):
    return orc.Materials(z_over_a=[0.5551], zeff=[7.42], **kw)


# ---------------------------------------------------------------------------
# Klein-Nishina
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("e", [0.011, 0.05, 0.2, 0.511])
def test_kn_total_equals_integral_of_differential(orc, e):
    # σ = 2π ∫ dσ/dΩ d(cosθ): the closed form and the angular form are separate
    # formulas, so a dropped term in either breaks the equality.
    val, err = integrate.quad(lambda c: orc.dsigma_kn(e, c), -1.0, 1.0, epsabs=0, epsrel=1e-13)
    assert abs(2 * math.pi * val / orc.sigma_kn(e) - 1.0) < 1e-10


def test_kn_thomson_limit(orc):
    # Low-energy expansion σ/σ_T = 1 - 2k + 26/5 k^2 - 133/10 k^3 + O(k^4), and
    # dσ/dΩ -> (r_e^2/2)(1 + cos^2θ) as k -> 0.
    e = 0.511e-3
    k = e / ME
    assert abs(orc.sigma_kn(e) / (SIGMA_T * (1 - 2 * k + 5.2 * k * k - 13.3 * k ** 3)) - 1.0) < 1e-9
    e = 1e-5
    for c in (-1.0, -0.3, 0.0, 0.7, 1.0):
        assert abs(orc.dsigma_kn(e, c) / (0.5 * RE * RE * (1 + c * c)) - 1.0) < 1e-4


def test_kn_forward_and_backward_values(orc):
    # Forward scattering: P = 1, dσ/dΩ = r_e^2 for any energy.
    for e in (0.05, 0.511):
        assert abs(orc.dsigma_kn(e, 1.0) / (RE * RE) - 1.0) < 1e-13
    # Backscatter at 511 keV: P = 1/(1+2k); dσ/dΩ = (r_e^2/2) P^2 (P + 1/P).
    k = 0.511 / ME
    p = 1.0 / (1.0 + 2.0 * k)
    assert abs(orc.dsigma_kn(0.511, -1.0) / (0.5 * RE * RE * p * p * (p + 1 / p)) - 1) < 1e-13
    # Published value of σ_KN at 511 keV: 0.2865 barn per electron.
    assert abs(orc.sigma_kn(0.511) / 0.2865e-24 - 1.0) < 2e-4


def _kn_bin_probs(e, edges):
    # Bin probabilities of cosθ from the textbook dσ/dΩ (written here on its own,
    # Compton's formula for P) -- not from the oracle.
    def f(c):
        k = e / ME
        p = 1.0 / (1.0 + k * (1.0 - c))
        return p * p * (p + 1.0 / p - (1.0 - c * c))
    z = integrate.quad(f, -1, 1, epsrel=1e-12)[0]
    return np.array([integrate.quad(f, a, b, epsrel=1e-12)[0] for a, b in zip(edges[:-1], edges[1:])]) / z


@pytest.mark.parametrize("e", [0.511, 0.2, 0.05])
def test_kn_sampler_chi2(orc, e):
    n = 1_000_000
    s = orc.sample_kn_cos(e, n, seed=12345)
    edges = np.linspace(-1, 1, 51)
    p = _kn_bin_probs(e, edges)
    h, _ = np.histogram(s, edges)
    chi2 = ((h - n * p) ** 2 / (n * p)).sum()
    assert stats.chi2.sf(chi2, len(p) - 1) > 1e-4, chi2


# ---------------------------------------------------------------------------
# Directions
# ---------------------------------------------------------------------------
def test_marsaglia_isotropic(orc):
    n = 1_000_000
    d = orc.sample_dirs(n, seed=7)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-12)
    # mean 0, <w_i^2> = 1/3, <w_i w_j> = 0 (closed forms for the uniform sphere).
    se = 1.0 / math.sqrt(3 * n)
    assert np.all(np.abs(d.mean(axis=0)) < 5 * se)
    m2 = (d ** 2).mean(axis=0)
    se2 = math.sqrt(4.0 / 45.0 / n)      # var(w^2) = 1/5 - 1/9
    assert np.all(np.abs(m2 - 1 / 3) < 5 * se2)
    # cosθ uniform on [-1, 1] and azimuth uniform: chi-square.
    h, _ = np.histogram(d[:, 2], np.linspace(-1, 1, 41))
    assert stats.chisquare(h).pvalue > 1e-4
    phi = np.arctan2(d[:, 1], d[:, 0])
    h, _ = np.histogram(phi, np.linspace(-np.pi, np.pi, 41))
    assert stats.chisquare(h).pvalue > 1e-4


def test_rotation_keeps_angle_and_is_symmetric(orc):
    rng = np.random.default_rng(3)
    for _ in range(50):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        c = rng.uniform(-1, 1)
        phis = np.linspace(0, 2 * np.pi, 64, endpoint=False)
        out = np.array([orc.rotate(d, c, ph) for ph in phis])
        assert np.allclose(np.linalg.norm(out, axis=1), 1.0, atol=1e-12)
        assert np.allclose(out @ d, c, atol=1e-12)
        # Averaged over the azimuth the new direction is c * d.
        assert np.allclose(out.mean(axis=0), c * d, atol=1e-12)


# ---------------------------------------------------------------------------
# Voxel traversal and free flight
# ---------------------------------------------------------------------------
def _slab_exit(p, d, L):
    # Distance from p (inside the box [0, L]) to the box boundary along d.
    t = np.inf
    for a in range(3):
        if d[a] > 0:
            t = min(t, (L[a] - p[a]) / d[a])
        elif d[a] < 0:
            t = min(t, -p[a] / d[a])
    return t


def _brute_lengths(shape_zyx, spacing, p, d, step):
    nz, ny, nx = shape_zyx
    L = np.array([nx * spacing[0], ny * spacing[1], nz * spacing[2]])
    t_exit = _slab_exit(p, d, L)
    t = (np.arange(int(t_exit / step) + 1) + 0.5) * step
    t = t[t < t_exit]
    pts = p[None, :] + t[:, None] * d[None, :]
    idx = np.floor(pts / np.array(spacing)).astype(np.int64)
    idx = np.clip(idx, 0, [nx - 1, ny - 1, nz - 1])
    flat = (idx[:, 2] * ny + idx[:, 1]) * nx + idx[:, 0]
    out = np.bincount(flat, minlength=nx * ny * nz).astype(np.float64) * step
    # last partial step
    out[flat[-1]] += t_exit - (t[-1] + 0.5 * step)
    return out, t_exit


def test_trace_matches_brute_force_stepping(orc):
    rng = np.random.default_rng(11)
    shape = (3, 4, 5)
    spacing = (0.7, 0.5, 1.1)
    L = np.array([5 * 0.7, 4 * 0.5, 3 * 1.1])
    step = 1e-5
    for _ in range(20):
        p = rng.uniform(0, 1, 3) * L
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        vox, ln = orc.trace(shape, spacing, p, d)
        got = np.zeros(60)
        np.add.at(got, vox, ln)
        ref, t_exit = _brute_lengths(shape, spacing, p, d, step)
        assert abs(ln.sum() - t_exit) < 1e-12
        assert np.all(np.abs(got - ref) < 2 * step), np.abs(got - ref).max()
        # Consecutive voxels are face neighbours (one index changes by one).
        v = np.stack([vox % 5, (vox // 5) % 4, vox // 20], axis=1)
        assert np.all(np.abs(np.diff(v, axis=0)).sum(axis=1) == 1)


def test_trace_axis_aligned_and_on_boundary(orc):
    # A ray along +x from a point on a voxel corner: floor convention puts it in
    # the upper voxel; it visits every voxel of its row with full length.
    vox, ln = orc.trace((4, 4, 4), (0.5, 0.5, 0.5), [1.0, 1.0, 1.0], [1.0, 0.0, 0.0])
    assert list(vox) == [2 * 16 + 2 * 4 + i for i in (2, 3)]
    assert np.allclose(ln, 0.5)
    vox, ln = orc.trace((4, 4, 4), (0.5, 0.5, 0.5), [1.0, 1.0, 1.0], [-1.0, 0.0, 0.0])
    assert list(vox) == [2 * 16 + 2 * 4 + i for i in (2, 1, 0)]
    assert np.allclose(ln, [0.0, 0.5, 0.5])


def test_first_flight_follows_exp_of_optical_depth(orc):
    rng = np.random.default_rng(5)
    mu = rng.uniform(0.05, 0.6, size=(2, 3, 4))
    spacing = (0.8, 0.6, 1.0)
    p = np.array([0.1, 0.9, 0.3])
    d = np.array([0.8, 0.3, 0.5])
    d /= np.linalg.norm(d)
    n = 400_000
    dist = orc.first_flight(mu, spacing, p, d, n, seed=99)
    lens, t_exit = _brute_lengths(mu.shape, spacing, p, d, 1e-5)
    tau = float((lens * mu.ravel()).sum())
    esc = np.mean(dist < 0)
    se = math.sqrt(math.exp(-tau) * (1 - math.exp(-tau)) / n)
    assert abs(esc - math.exp(-tau)) < 5 * se
    # P(collision before t) = 1 - exp(-tau(t)) at a few depths along the ray.
    for frac in (0.2, 0.5, 0.8):
        t = frac * t_exit
        l_t, _ = _brute_lengths(mu.shape, spacing, p, d, 1e-5)
        # optical depth up to t by brute-force stepping
        steps = np.arange(int(t / 1e-5)) * 1e-5 + 0.5e-5
        pts = p[None] + steps[:, None] * d[None]
        idx = np.floor(pts / np.array(spacing)).astype(int)
        tau_t = mu[idx[:, 2], idx[:, 1], idx[:, 0]].sum() * 1e-5
        pr = 1 - math.exp(-tau_t)
        got = np.mean((dist >= 0) & (dist < t))
        assert abs(got - pr) < 5 * math.sqrt(pr * (1 - pr) / n)


# ---------------------------------------------------------------------------
# HU -> density / material (§2.1)
# ---------------------------------------------------------------------------
def test_hu_curve_nodes_midpoints_and_clamps(orc):
    nodes_hu = [-1000, -750, -100, 40, 1000]
    nodes_rho = [0.0012, 0.26, 0.95, 1.03, 1.85]
    den, mat = orc.hu_to_phantom(np.array(nodes_hu, np.int16))
    assert np.allclose(den, nodes_rho, rtol=0, atol=1e-15)
    assert list(mat) == [0, 1, 2, 3, 4]
    mids = [(a + b) // 2 for a, b in zip(nodes_hu[:-1], nodes_hu[1:])]
    den, _ = orc.hu_to_phantom(np.array(mids, np.int16))
    exp = [nodes_rho[i] + (mids[i] - nodes_hu[i]) / (nodes_hu[i + 1] - nodes_hu[i]) * (nodes_rho[i + 1] - nodes_rho[i]) for i in range(4)]
    assert np.allclose(den, exp, rtol=0, atol=1e-15)
    den, mat = orc.hu_to_phantom(np.array([-1024, -3000, 1500, 3071], np.int16))
    assert np.allclose(den, [0.0012, 0.0012, 1.85, 1.85])
    assert list(mat) == [0, 0, 4, 4]
    # Nearest-node material: boundaries halfway between nodes, ties to the lower node.
    den, mat = orc.hu_to_phantom(np.array([-875, -874, -425, -424, -30, -29, 520, 521], np.int16))
    assert list(mat) == [0, 1, 1, 2, 2, 3, 3, 4]
    # Density is monotone in HU.
    h = np.arange(-1024, 3072, dtype=np.int16)
    den, _ = orc.hu_to_phantom(h)
    assert np.all(np.diff(den) >= 0)


# ---------------------------------------------------------------------------
# Whole-simulation pins
# ---------------------------------------------------------------------------
def _ray_box_interval(d, lo, hi):
    # Entry and exit distances of rays from the origin (direction d[n,3]) through
    # the axis-aligned box [lo, hi] (slab method); empty intervals give t0 >= t1.
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / d
        t_a = (lo[None, :]) * inv
        t_b = (hi[None, :]) * inv
    tmin = np.minimum(t_a, t_b)
    tmax = np.maximum(t_a, t_b)
    tmin = np.where(np.isnan(tmin), -np.inf, tmin)
    tmax = np.where(np.isnan(tmax), np.inf, tmax)
    t0 = np.maximum(tmin.max(axis=1), 0.0)
    t1 = tmax.min(axis=1)
    return t0, t1


def test_point_source_absorber_matches_first_collision_kernel(orc):
    # Pure absorber (no electrons, so no Compton): every photon deposits all its
    # energy at its first interaction, so the expected tally of voxel v is
    #   N q(E) ∫_{4π} dΩ/4π [exp(-mu r_in) - exp(-mu r_out)]
    # i.e. the uncollided kernel mu exp(-mu r)/(4 pi r^2) integrated over v.
    n_side, vox = 8, 0.5
    mu_target = 0.4                       # 1/cm at 0.511 MeV
    zeff = 7.42
    pe = mu_target * 0.511 ** 3 / zeff ** 3.8
    mat = orc.Materials(z_over_a=[0.0], zeff=[zeff], pe_coeff=pe)
    assert abs(orc.mu(mat, 0, 1.0, 0.511)[1] - mu_target) < 1e-12
    den = np.ones((n_side,) * 3)
    src = np.array([2.0, 2.0, 2.0])        # a voxel corner at the cube centre
    N = 2_000_000
    r = orc.run(den, np.zeros((n_side,) * 3, np.uint8), mat, spacing=(vox,) * 3, point=tuple(src),
                n_hist=N, seed=4, batches=10)
    q = round(0.511 * 64e6)
    assert r.counters["compton"] == 0
    # Quadrature over directions: a fine stratified grid in (cosθ, φ).
    m = 1500
    c = (np.arange(m) + 0.5) / m * 2 - 1
    ph = (np.arange(2 * m) + 0.5) / (2 * m) * 2 * np.pi
    C_, P_ = np.meshgrid(c, ph, indexing="ij")
    s = np.sqrt(1 - C_ ** 2)
    dirs = np.stack([s * np.cos(P_), s * np.sin(P_), C_], axis=-1).reshape(-1, 3)
    # Check the voxels of a 4x4x4 block around the source and a far corner.
    checks = [(i, j, k) for i in range(2, 6) for j in range(2, 6) for k in range(2, 6)] + [(7, 7, 7), (0, 3, 6)]
    z = []
    for (ix, iy, iz) in checks:
        lo = np.array([ix, iy, iz]) * vox - src
        hi = lo + vox
        t0, t1 = _ray_box_interval(dirs, lo, hi)
        ok = t1 > t0
        prob = np.where(ok, np.exp(-mu_target * t0) - np.exp(-mu_target * np.where(ok, t1, t0)), 0).mean()
        expect = N * prob * q
        got = r.tally[iz, iy, ix]
        sd = math.sqrt(N * prob * (1 - prob)) * q
        z.append((got - expect) / sd)
        assert abs(prob) > 0
    z = np.array(z)
    assert np.all(np.abs(z) < 5), z
    assert abs(z.mean()) < 5 / math.sqrt(len(z))


def test_energy_conservation_is_exact(orc):
    from paper_2111_11687_gb300 import inputs
    cube = inputs.water_cube(16, 1.0)
    mat = water(orc)
    r = orc.run(cube.density, cube.material, mat, spacing=cube.spacing, point=cube.point,
                n_hist=20000, seed=2, batches=4)
    c = r.counters
    assert c["emitted"] == 20000 * round(0.511 * 64e6)
    assert c["deposited"] + c["escaped"] == c["emitted"]
    assert int(r.tally.sum()) == c["deposited"]
    # Decay mode on a small phantom: positron energy plus two photons per decay.
    ph = inputs.adult_phantom(shape=(30, 24, 24), spacing=(2.1, 2.1, 3.0), seed=3)
    den, mt = orc.hu_to_phantom(ph.hu)
    mat5 = orc.Materials(z_over_a=inputs.MATERIAL_Z_OVER_A, zeff=inputs.MATERIAL_ZEFF)
    r = orc.run(den, mt, mat5, activity=ph.activity, labels=ph.labels, n_labels=27,
                spacing=ph.spacing, n_hist=20000, seed=5, batches=4)
    c = r.counters
    per_decay = 2 * round(0.511 * 64e6) + round(0.25 * 64e6)
    assert c["emitted"] == 20000 * per_decay
    assert c["deposited"] + c["escaped"] == c["emitted"]
    assert int(r.tally.sum()) == c["deposited"]
    # No photon gains energy: nothing deposited per event above 0.511 MeV
    # (pair production is absent below 1.02 MeV).
    assert c["compton"] > 0 and c["photo"] > 0


def test_infinite_medium_absorbs_everything(orc):
    # A 10 m water block: escape probability ~exp(-48), so absorbed = emitted.
    n = 5
    den = np.ones((n, n, n))
    r = orc.run(den, np.zeros((n, n, n), np.uint8), water(orc), spacing=(200.0,) * 3,
                point=(500.0, 500.0, 500.0), n_hist=20000, seed=9, batches=4)
    c = r.counters
    assert c["escaped"] == 0 and c["escapes"] == 0
    assert c["deposited"] == c["emitted"]


def test_eq1_to_eq3_on_a_deterministic_case(orc):
    # Opaque single voxel: mu huge, every photon is absorbed where it starts, so
    # each batch's tally is exact and the batch variance is zero.
    n = 3
    mat = orc.Materials(z_over_a=[0.0], zeff=[7.42], pe_coeff=1e3)
    den = np.full((n, n, n), 2.0)
    act = np.zeros((n, n, n))
    act[1, 1, 1] = 1.0
    lab = np.zeros((n, n, n), np.uint8)
    lab[1, 1, :] = 1          # organ 1: three voxels, one of them the source
    N, A = 1001, 3.0e8
    spacing = (0.4, 0.5, 0.6)
    r = orc.run(den, np.zeros((n, n, n), np.uint8), mat, activity=act, labels=lab, n_labels=1,
                spacing=spacing, n_hist=N, seed=1, batches=10, activity_bq=A)
    q = 2 * round(0.511 * 64e6) + round(0.25 * 64e6)
    assert r.tally[1, 1, 1] == N * q and r.tally.sum() == N * q
    mass = 2.0 * 0.4 * 0.5 * 0.6 * 1e-3                      # kg
    e_j = q / 64.0 * 1.602176634e-19                          # J per decay
    dr = e_j / mass * A                                       # Eq. 1
    assert abs(r.dose_rate[1, 1, 1] / dr - 1) < 1e-14
    assert r.sigma[1, 1, 1] < 1e-12 * dr
    # Eq. 2: unweighted mean over the organ's 3 voxels.
    assert abs(r.organ_mean[1] / (dr / 3) - 1) < 1e-14
    # Eq. 3: RMS of relative uncertainties: the source voxel 0, the two empty
    # voxels 1 (100 %) each.
    assert abs(r.organ_eps[1] - math.sqrt(2 / 3)) < 1e-14
    assert r.organ_sigma[1] < 1e-12 * dr


def test_batch_sigma_matches_spread_over_seeds(orc):
    # The batch estimate of sigma of the mean must match the scatter of the mean
    # over independent runs (consistency of the variance estimator).
    n = 6
    mat = orc.Materials(z_over_a=[0.5551], zeff=[7.42])
    den = np.ones((n, n, n))
    lab = np.zeros((n, n, n), np.uint8)
    lab[:3] = 1
    act = np.ones((n, n, n))
    means, sig, om, osg = [], [], [], []
    for s in range(40):
        r = orc.run(den, np.zeros((n, n, n), np.uint8), mat, activity=act, labels=lab, n_labels=1,
                    spacing=(1.0,) * 3, n_hist=4000, seed=100 + s, batches=8)
        means.append(r.dose_rate[2, 2, 2]); sig.append(r.sigma[2, 2, 2])
        om.append(r.organ_mean[1]); osg.append(r.organ_sigma[1])
    for m, sg in ((means, sig), (om, osg)):
        emp = np.std(m, ddof=1)
        est = math.sqrt(np.mean(np.square(sg)))
        # ratio of variances ~ F-distributed; 40 runs -> about +-25 % at 2 sigma
        assert 0.6 < emp / est < 1.5, (emp, est)


# ---------------------------------------------------------------------------
# Eq. 4 against the paper's Table 1
# ---------------------------------------------------------------------------
def _table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_organ_dose_rates.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, g, gu, a, au, d = line.split()
            rows.append((name, float(g), float(gu), float(a), float(au), float(d)))
    return rows


def test_eq4_reproduces_table1(orc):
    rows = _table1()
    assert len(rows) == 27
    g = np.array([r[1] for r in rows])
    a = np.array([r[3] for r in rows])
    d = np.array([r[5] for r in rows])
    got = orc.rel_diff_percent(a, g)
    # Printed rates have 4 significant digits: the recomputed difference can be
    # off by up to ~(0.5e-3/1.3)*100*2 percent from the printed one.
    assert np.all(np.abs(got - d) < 0.08), np.abs(got - d).max()
    summ = {}
    with open(os.path.join(GOLDEN, "table1_summary.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split()
            summ[k] = float(v)
    assert abs(d.min() - summ["diff_min"]) < 1e-9 and abs(d.max() - summ["diff_max"]) < 1e-9
    assert abs(np.abs(d).mean() - summ["mean_abs_diff"]) < 0.005
    assert abs(np.abs(got).mean() - summ["mean_abs_diff"]) < 0.01
    gu = np.array([r[2] for r in rows]); au = np.array([r[4] for r in rows])
    assert gu.min() == summ["gate_unc_min"] and gu.max() == summ["gate_unc_max"]
    assert au.min() == summ["archer_unc_min"] and au.max() == summ["archer_unc_max"]
    # Sign convention: test above reference -> positive.
    assert orc.rel_diff_percent(2.0, 1.0) == 100.0


def test_oracle_dose_rate_scale_matches_table1(orc):
    """The absolute scale of Eq. 1 (MeV -> J, g -> kg, voxel volume, A(t_s))
    against the dose rates Table 1 prints (§3.2).  The stored FP64 oracle
    organ means of the benchmark phantom carry the activity of the paper's
    patient (8.0 mCi of 18F, 60 min after injection, §2.2) in the body of a
    pelvis-to-head field of view, which weighs far less than that 79 kg
    patient.  At equal activity a mean dose rate goes as 1 / mass, so the
    median organ dose rate, times the phantom's body mass over 79 kg, must
    land within a factor of two of Table 1's median (it lands within 5 %,
    which the different anatomy and uptake make partly chance); a slip in any
    unit of Eq. 1 moves it by orders of magnitude."""
    from paper_2111_11687_gb300 import inputs
    rows = [l.split() for l in open(os.path.join(GOLDEN, "adult_phantom_organs_oracle.txt"))
            if l.strip() and not l.startswith("#")]
    organs = np.array([float(r[1]) for r in rows])[1:]
    assert organs.size == 27 and np.all(organs > 0)
    ph = inputs.adult_phantom()                 # the stored phantom: 256x256x300 x 2x2x3 mm, seed 1
    den, _ = orc.hu_to_phantom(ph.hu)
    body_kg = float(den[den >= 0.1].astype(np.float64).sum()) * 0.2 * 0.2 * 0.3 / 1000.0
    assert 15.0 < body_kg < 60.0, body_kg
    scaled = np.median(organs) * body_kg / 79.0
    table = np.median([r[1] for r in _table1()])   # GATE column (the paper's reference)
    assert 0.5 < scaled / table < 2.0, (scaled, table, body_kg)


@pytest.mark.parametrize("absorb", [False, True])
def test_history_sigma_bernoulli_closed_form(orc, absorb):
    # Every history deposits a fixed amount T in its decay voxel and nothing
    # elsewhere, so voxel v's per-history total is T with probability p_v and 0
    # otherwise: the sample variance of the history totals is exactly
    # T^2 p(1 - p) N / (N - 1) with p the observed fraction, and the
    # history-by-history sigma of the mean over the mean is
    # sqrt((1 - p) / ((N - 1) p)).
    #   absorb=False: a near-vacuum (photons escape), T = the positron energy;
    #   absorb=True: a dense photoelectric absorber, T = positron + two photons,
    #   deposited in three pieces: squaring the pieces instead of their sum
    #   would give a different answer.
    rng = np.random.default_rng(4)
    shape = (4, 4, 4)
    act = rng.uniform(0.2, 1.0, shape)
    if absorb:
        den = np.full(shape, 10.0)
        mat = orc.Materials(z_over_a=[0.0], zeff=[7.42], pe_coeff=1e3)
    else:
        den = np.full(shape, 1e-9)
        mat = orc.Materials(z_over_a=[0.5551], zeff=[7.42])
    N = 400_000
    r = orc.run(den, np.zeros(shape, np.uint8), mat, activity=act, spacing=(1.0, 1.0, 1.0), n_hist=N, seed=9,
                batches=10, history_sigma=True)
    q_pos = round(0.25 * 6.4e7)
    T = q_pos + (2 * round(0.511 * 6.4e7) if absorb else 0)
    assert r.counters["deposited"] == N * T          # every history deposits T, and only in one voxel
    p = r.tally / (T * N)
    assert np.allclose(p * T * N, r.tally)
    expect = np.sqrt((1 - p) / ((N - 1) * p))
    assert np.allclose(r.sigma_history / r.dose_rate, expect, rtol=1e-9, atol=0)
    # the batch sigma estimates the same quantity, with ~25 % scatter at 10 batches
    ratio = r.sigma / r.sigma_history
    assert 0.85 < np.median(ratio) < 1.15


# ---------------------------------------------------------------------------
# Positron: beta+ spectrum and range (the beta-spectrum variant of the decay)
# ---------------------------------------------------------------------------
F18_T_MAX = 0.6335     # MeV, 18F beta+ endpoint (nuclear data tables)
F18_T_MEAN = 0.2498    # MeV, 18F mean beta+ energy (nuclear data tables)


def test_beta_spectrum_mean_of_18f(orc):
    # The published mean of 18F's positrons, which is also the 0.25 MeV the
    # constant-deposit model uses.  Without the Fermi function the mean would
    # be 0.2404 MeV and with the electron's (attractive) one lower still, so a
    # missing or sign-flipped Coulomb factor fails here.
    t = orc.sample_beta(F18_T_MAX, 8, 2_000_000, 3)
    assert 0.0 < t.min() and t.max() < F18_T_MAX
    assert abs(t.mean() / F18_T_MEAN - 1.0) < 0.005
    assert abs(t.mean() / 0.25 - 1.0) < 0.005
    t0 = orc.sample_beta(F18_T_MAX, 0, 1_000_000, 4)
    assert t0.mean() < 0.243


def test_beta_spectrum_statistical_shape_limit(orc):
    # Z = 0 and an endpoint far below m c^2: p E (T_max - T)^2 tends to
    # sqrt(T) (T_max - T)^2, the Beta(3/2, 3) law on [0, T_max] (corrections
    # O(T_max / m c^2) = 0.2 %, far below the test's resolution).
    t_max = 1e-3
    t = orc.sample_beta(t_max, 0, 200_000, 5)
    ks = stats.kstest(t, stats.beta(1.5, 3.0, scale=t_max).cdf)
    assert ks.pvalue > 1e-3
    assert abs(t.mean() / (t_max / 3.0) - 1.0) < 0.01


# NIST ESTAR, electrons in liquid water: CSDA range (g/cm^2).  The Katz-Penfold
# relation is an empirical fit of practical ranges, within ~10 % of these.
ESTAR_WATER_CSDA = {0.1: 1.431e-2, 0.2: 4.488e-2, 0.5: 1.766e-1, 1.0: 4.367e-1}


def test_positron_range_against_estar(orc):
    for t, r in ESTAR_WATER_CSDA.items():
        assert abs(orc.range_kp(t) / r - 1.0) < 0.10, t
    for t in np.geomspace(1e-3, 2.0, 23):
        assert abs(orc.energy_at_range(orc.range_kp(t)) / t - 1.0) < 1e-12
    assert orc.range_kp(0.0) == 0.0 and orc.energy_at_range(0.0) == 0.0


@pytest.mark.parametrize("rho", [1.0, 0.5])
def test_positron_track_escape_and_local_deposit(orc, rho):
    # Photons that never interact (mu = 0) leave the 5^3 cube; what stays is
    # the positrons' energy.  The oracle's escaped positron energy and its
    # central-voxel deposit per decay must match the brute-force expectation
    # over the same spectrum (halving the density doubles every range).
    n_side, vox, N = 5, 0.05, 200_000
    den = np.full((n_side,) * 3, rho)
    act = np.zeros((n_side,) * 3)
    act[2, 2, 2] = 1.0
    mat = orc.Materials(z_over_a=[0.0], zeff=[7.42], pe_coeff=0.0)
    r = orc.run(den, np.zeros((n_side,) * 3, np.uint8), mat, activity=act, spacing=(vox,) * 3, n_hist=N,
                seed=8, batches=2, beta_max_mev=F18_T_MAX, beta_z=8)
    c = r.counters
    q = 64e6
    q_photon = round(0.511 * q)
    assert c["deposited"] + c["escaped"] == c["emitted"]
    assert c["compton"] == 0 and c["photo"] == 0
    esc_pos = (c["escaped"] - 2 * N * q_photon) / q / N          # MeV per decay
    centre = r.tally[2, 2, 2] / q / N
    rng = np.random.default_rng(17)
    t = orc.sample_beta(F18_T_MAX, 8, 1_000_000, 23)
    e_esc, e_centre = cube_positron_expectation(rho, n_side, vox, t, rng)
    for got, ref in ((esc_pos, e_esc), (centre, e_centre)):
        sd = ref.std() * math.sqrt(1.0 / N + 1.0 / ref.size)
        assert abs(got - ref.mean()) < 4.0 * sd + 1e-6, (got, ref.mean(), sd)
    assert esc_pos > 0.0 and centre > 0.03


# ---------------------------------------------------------------------------
# Interactions: the collision step orc_run takes at every real event (type
# choice, Compton kinematics, Rayleigh angle), called through a test entry of
# the same function.
# ---------------------------------------------------------------------------
NA = 6.02214076e23


def _sigma_tr(e):
    """Klein-Nishina energy-transfer cross section per electron (cm^2), the
    closed form of Attix (Introduction to Radiological Physics, eq. 7.20)."""
    k = e / ME
    a = 1.0 + 2.0 * k
    lg = math.log(a)
    return 2 * math.pi * RE * RE * (2 * (1 + k) ** 2 / (k * k * a) - (1 + 3 * k) / a ** 2
                                    - (1 + k) * (2 * k * k - 2 * k - 1) / (k * k * a * a) - 4 * k * k / (3 * a ** 3)
                                    - ((1 + k) / k ** 3 - 1 / (2 * k) + 1 / (2 * k ** 3)) * lg)


def _dsigma_dt(e, t):
    """Klein-Nishina spectrum of the recoil electron's kinetic energy T, per
    electron (cm^2/MeV), with s = T/E (Evans, The Atomic Nucleus, ch. 23)."""
    k = e / ME
    s = t / e
    return math.pi * RE * RE / (ME * k * k) * (2 + s * s / (k * k * (1 - s) ** 2) + s / (1 - s) * (s - 2 / k))


def test_energy_transfer_closed_form_matches_quadrature_of_recoil_spectrum():
    # The two published forms used below agree with each other: E sigma_tr =
    # integral of T dsigma/dT over 0..T_max.
    for e in (0.05, 0.2, 0.511):
        k = e / ME
        tmax = e * 2 * k / (1 + 2 * k)
        q = integrate.quad(lambda t: t * _dsigma_dt(e, t), 0, tmax, epsrel=1e-12)[0]
        assert abs(q / (e * _sigma_tr(e)) - 1) < 1e-9


@pytest.mark.parametrize("rayleigh", [0, 1])
def test_interaction_choice_follows_the_attenuation_coefficients(orc, rayleigh):
    # Photoelectric and Rayleigh constants chosen so that all three types are
    # common at 0.2 MeV; the expected fractions come from the definitions of
    # the coefficients (electron density x sigma_KN, C Zeff^3.8 / E^3,
    # c_R Zeff^2 / E^2), so swapped thresholds or a dropped term fail.
    e, za, zeff, rho = 0.2, 0.55, 7.4, 1.3
    pe_coeff, r_coeff = 6.0e-7, 1.0e-4
    m = orc.Materials(z_over_a=[za], zeff=[zeff], pe_coeff=pe_coeff, rayleigh_coeff=r_coeff, rayleigh=rayleigh)
    mu_c = rho * NA * za * orc.sigma_kn(e)
    mu_pe = rho * pe_coeff * zeff ** 3.8 / e ** 3
    mu_r = rho * r_coeff * zeff * zeff / e ** 2 if rayleigh else 0.0
    p = np.array([mu_c, mu_pe, mu_r]) / (mu_c + mu_pe + mu_r)
    assert p.min() > 0.1 or not rayleigh        # every type is well represented
    n = 600_000
    t, e2, c = orc.interactions(m, 0, rho, e, n, seed=31 + rayleigh)
    h = np.bincount(t, minlength=3)[:3].astype(float)
    used = p > 0
    assert h[~used].sum() == 0
    chi2 = ((h[used] - n * p[used]) ** 2 / (n * p[used])).sum()
    assert stats.chi2.sf(chi2, used.sum() - 1) > 1e-4, (h / n, p)
    # after a photoelectric event nothing is left; Rayleigh keeps the energy
    assert np.all(e2[t == 1] == 0.0)
    assert np.all(e2[t == 2] == e)


@pytest.mark.parametrize("e", [0.511, 0.1])
def test_compton_energy_transfer_matches_klein_nishina(orc, e):
    # Compton only: the electron's energy T = E - E' has mean E sigma_tr /
    # sigma_KN and the recoil spectrum dsigma/dT (published closed forms, not
    # the oracle's angle formula): E' = E/(1 + k(1 + cos)) or a cosine of the
    # wrong sign would move both.
    n = 1_000_000
    m = water(orc, pe_coeff=0.0)
    t, e2, c = orc.interactions(m, 0, 1.0, e, n, seed=77)
    assert np.all(t == 0)
    T = e - e2
    k = e / ME
    tmax = e * 2 * k / (1 + 2 * k)
    assert T.min() >= 0 and T.max() <= tmax * (1 + 1e-12)
    mean = e * _sigma_tr(e) / orc.sigma_kn(e)
    z = (T.mean() - mean) / (T.std() / math.sqrt(n))
    assert abs(z) < 4.5, (T.mean(), mean, z)
    edges = np.linspace(0.0, tmax, 41)
    tot = integrate.quad(lambda x: _dsigma_dt(e, x), 0, tmax, epsrel=1e-12)[0]
    pb = np.array([integrate.quad(lambda x: _dsigma_dt(e, x), a, b, epsrel=1e-12)[0]
                   for a, b in zip(edges[:-1], edges[1:])]) / tot
    hb, _ = np.histogram(T, edges)
    chi2 = ((hb - n * pb) ** 2 / (n * pb)).sum()
    assert stats.chi2.sf(chi2, len(pb) - 1) > 1e-4, chi2


def test_thomson_sampler_chi2(orc):
    # Rayleigh angle with the Thomson shape: p(cos) = 3/8 (1 + cos^2).
    n = 1_000_000
    s = orc.sample_thomson_cos(n, seed=5)
    assert s.min() >= -1 and s.max() <= 1
    edges = np.linspace(-1, 1, 41)
    a, b = edges[:-1], edges[1:]
    p = 3.0 / 8.0 * ((b - a) + (b ** 3 - a ** 3) / 3.0)
    assert abs(p.sum() - 1) < 1e-12
    h, _ = np.histogram(s, edges)
    chi2 = ((h - n * p) ** 2 / (n * p)).sum()
    assert stats.chi2.sf(chi2, len(p) - 1) > 1e-4, chi2
    # <cos^2> = 2/5 for this shape (isotropic would give 1/3)
    assert abs((s * s).mean() - 0.4) < 5 * math.sqrt(((s ** 4).mean() - 0.16) / n)


# ---------------------------------------------------------------------------
# Decay sampling inside orc_run (§2.1: linear PET -> decay PDF)
# ---------------------------------------------------------------------------
def _uneven_activity(shape, seed):
    rng = np.random.default_rng(seed)
    act = np.zeros(int(np.prod(shape)))
    # active voxels of unequal activity with inactive voxels between them; the
    # first voxel is inactive and the last one active (ends of the table)
    idx = np.array([3, 4, 9, 17, 18, 40, 57, 58, 90, act.size - 1])
    act[idx] = rng.uniform(0.2, 5.0, idx.size)
    return act.reshape(shape), idx


def test_decay_voxels_follow_the_activity_exactly(orc):
    # No attenuation at all: both photons leave the grid untouched, so each
    # voxel's tally is exactly (decays in it) x q(positron).  Counts follow
    # N A_v / sum A (chi-square); inactive voxels get exactly none.
    shape = (4, 5, 6)
    act, idx = _uneven_activity(shape, 3)
    n = 2_000_000
    q = round(0.25 * 64e6)
    vac = orc.Materials(z_over_a=[0.0], zeff=[0.0], pe_coeff=0.0)
    r = orc.run(np.ones(shape), np.zeros(shape, np.uint8), vac, activity=act, spacing=(0.7, 0.9, 1.1),
                n_hist=n, seed=8, batches=4, positron_mev=0.25)
    t = r.tally.ravel()
    assert np.all(t % q == 0)
    cnt = t // q
    assert cnt.sum() == n
    inactive = np.ones(t.size, bool)
    inactive[idx] = False
    assert np.all(cnt[inactive] == 0)
    p = act.ravel()[idx] / act.sum()
    chi2 = ((cnt[idx] - n * p) ** 2 / (n * p)).sum()
    assert stats.chi2.sf(chi2, idx.size - 1) > 1e-4, (cnt[idx] / n, p)
    assert r.counters["compton"] == 0 and r.counters["photo"] == 0
    assert r.counters["escaped"] == 2 * n * round(0.511 * 64e6)


def test_decay_positions_stay_in_the_decay_voxel(orc):
    # A pure absorber with a free path of ~1e-13 cm: both photons end where the
    # decay happened, so every voxel keeps (decays in it) x (positron + 2
    # photons).  Unequal voxel sides catch a position scaled by the wrong side.
    shape = (4, 5, 6)
    act, idx = _uneven_activity(shape, 4)
    n = 500_000
    per = round(0.25 * 64e6) + 2 * round(0.511 * 64e6)
    absorber = orc.Materials(z_over_a=[0.0], zeff=[1.0], pe_coeff=1e12)
    r = orc.run(np.ones(shape), np.zeros(shape, np.uint8), absorber, activity=act, spacing=(0.3, 1.7, 0.8),
                n_hist=n, seed=9, batches=4, positron_mev=0.25)
    t = r.tally.ravel()
    assert np.all(t % per == 0) and t.sum() == n * per
    cnt = t // per
    inactive = np.ones(t.size, bool)
    inactive[idx] = False
    assert np.all(cnt[inactive] == 0)
    p = act.ravel()[idx] / act.sum()
    chi2 = ((cnt[idx] - n * p) ** 2 / (n * p)).sum()
    assert stats.chi2.sf(chi2, idx.size - 1) > 1e-4


# ---------------------------------------------------------------------------
# Other radionuclides (paper §4: 177Lu, 131I) and multi-time-point dosimetry
# ---------------------------------------------------------------------------
# Published decay data (NNDC / ICRP 107): beta- branches (endpoint MeV,
# fraction of decays), mean beta- energy per decay, daughter Z.
LU177 = dict(branches=[(0.4983, 0.794), (0.3849, 0.091), (0.1765, 0.116)], mean=0.1336, z=72)
I131 = dict(branches=[(0.6063, 0.896), (0.3338, 0.0723), (0.2479, 0.0208), (0.8069, 0.0039)], mean=0.1819, z=54)


@pytest.mark.parametrize("nuc", [LU177, I131], ids=["177Lu", "131I"])
def test_beta_minus_spectra_against_published_mean_energies(orc, nuc):
    # The allowed shape with the non-relativistic Fermi function of an
    # electron is an approximation for these heavy daughters (forbidden
    # branches, relativistic and screening corrections): its mean lies a few
    # percent above the tabulated one.  A positron's Fermi function (the wrong
    # sign) would move the mean by far more than the 6 % allowed here.
    n = 400_000
    e = [b[0] for b in nuc["branches"]]
    s = orc.sample_beta_branches(e, [b[1] for b in nuc["branches"]], nuc["z"], -1, n, seed=21)
    assert s.min() > 0 and s.max() < max(e)
    assert abs(s.mean() / nuc["mean"] - 1) < 0.06, (s.mean(), nuc["mean"])
    wrong = orc.sample_beta_branches(e, [b[1] for b in nuc["branches"]], nuc["z"], +1, n, seed=21)
    assert abs(wrong.mean() / nuc["mean"] - 1) > 0.15, wrong.mean()


def test_beta_branch_mixture_chi2(orc):
    # Samples of a two-branch electron spectrum against the mixture of the
    # normalised branch densities (quadrature of the pinned density).
    br = [(0.5, 0.7), (0.2, 0.3)]
    z = 30
    n = 400_000
    s = orc.sample_beta_branches([b[0] for b in br], [b[1] for b in br], z, -1, n, seed=3)
    edges = np.linspace(0, 0.5, 26)
    p = np.zeros(len(edges) - 1)
    for tm, w in br:
        f = lambda t: orc.beta_density_signed(t, tm, z, -1)
        norm = integrate.quad(f, 0, tm, limit=200)[0]
        p += w * np.array([integrate.quad(f, a, min(b, tm), limit=100)[0] if a < tm else 0.0
                           for a, b in zip(edges[:-1], edges[1:])]) / norm
    h, _ = np.histogram(s, edges)
    ok = p > 0
    chi2 = ((h[ok] - n * p[ok]) ** 2 / (n * p[ok])).sum()
    assert stats.chi2.sf(chi2, ok.sum() - 1) > 1e-4, chi2


def test_gamma_lines_follow_their_yields(orc):
    # No attenuation: every photon leaves, so the escaped energy and the
    # number of escapes give each line's count exactly (two lines, two
    # equations); counts against N x yield (binomial).  No annihilation pair.
    lines = [(0.2084, 0.104), (0.1130, 0.062)]
    n = 1_000_000
    vac = orc.Materials(z_over_a=[0.0], zeff=[0.0], pe_coeff=0.0)
    shape = (3, 3, 3)
    act = np.ones(shape)
    r = orc.run(np.ones(shape), np.zeros(shape, np.uint8), vac, activity=act, spacing=(1.0, 1.0, 1.0), n_hist=n,
                seed=5, batches=2, positron_mev=0.1336, annihilation=False, gamma_lines=lines)
    q1, q2 = (round(e * 64e6) for e, _ in lines)
    esc, k = r.counters["escaped"], r.counters["escapes"]
    n2 = (esc - q1 * k) / (q2 - q1)
    n1 = k - n2
    assert n1 == int(n1) and n2 == int(n2) and n1 >= 0 and n2 >= 0
    for cnt, (_, y) in zip((n1, n2), lines):
        assert abs(cnt - n * y) < 4.5 * math.sqrt(n * y * (1 - y)), (cnt, n * y)
    # emitted = local beta energy + gamma photons; deposited = the beta part
    assert r.counters["emitted"] == n * round(0.1336 * 64e6) + esc
    assert r.tally.sum() == n * round(0.1336 * 64e6)


def test_time_integrated_activity_by_hand(orc):
    # Points (1 h, 100 Bq) and (3 h, 80 Bq), half-life 6 h:
    #   uptake 100 x 3600 / 2 = 180000; trapezoid (100 + 80)/2 x 7200 = 648000;
    #   tail 80 x 6 x 3600 / ln 2 = 2492977.03...; total 3320977.03... Bq s
    out = orc.time_integrated_activity([np.array([100.0]), np.array([80.0])], [1.0, 3.0], 6.0)
    assert abs(out[0] - (180000 + 648000 + 80 * 21600 / math.log(2))) < 1e-6
    assert abs(out[0] - 3320977.0307) < 1e-3


def test_time_integrated_activity_exact_for_physical_decay(orc):
    # A map measured at t = 0 that then only decays physically integrates to
    # A_0 T_1/2 / ln 2 exactly, and the result is linear in the maps.
    a = np.array([1.0, 2.5, 0.0, 7.0])
    out = orc.time_integrated_activity([a], [0.0], 109.77 / 60.0)
    assert np.allclose(out, a * 109.77 * 60.0 / math.log(2), rtol=1e-15, atol=0)
    b = np.array([3.0, 0.5, 1.0, 2.0])
    t = [0.5, 2.0, 24.0]
    lhs = orc.time_integrated_activity([2 * a, 2 * b, a + b], t, 6.65 * 24)
    rhs = 2 * orc.time_integrated_activity([a, b, 0.5 * (a + b)], t, 6.65 * 24)
    assert np.allclose(lhs, rhs, rtol=1e-14, atol=0)
