"""GPU checks of the device building blocks through the C ABI: Philox against
its published known answers, Kahn's and the tabulated Klein-Nishina samplers against the
analytic distribution, CT conversion against the oracle (bit-exact materials),
the alias table against exact reconstruction, the source sampler against the
activity map."""
import math
import os

import numpy as np
import pytest
from scipy import integrate, stats

from tests.parity_record import record

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ME = 0.51099895


@pytest.fixture(scope="module")
def nm():
    from paper_2111_11687_gb300 import build, nmdose
    build.build()
    nmdose.load()
    return nmdose


def test_philox_known_answers(nm):
    ctr, key, out = [], [], []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            t = line.split()
            ctr.append([int(x, 16) for x in t[1:5]])
            key.append([int(x, 16) for x in t[6:8]])
            out.append([int(x, 16) for x in t[9:13]])
    got = nm.nm_check_philox(np.array(ctr, np.uint32), np.array(key, np.uint32))
    assert (got == np.array(out, np.uint32)).all()


def test_philox_uniformity(nm):
    n = 1 << 18
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = np.arange(n)
    ctr[:, 2] = 12345
    key = np.tile(np.array([[7, 9]], np.uint32), (n, 1))
    out = nm.nm_check_philox(ctr, key).astype(np.float64).ravel() / 2 ** 32
    h, _ = np.histogram(out, np.linspace(0, 1, 65))
    assert stats.chisquare(h).pvalue > 1e-4


def _kn_bins(e, edges):
    def f(c):
        k = e / ME
        p = 1.0 / (1.0 + k * (1.0 - c))
        return p * p * (p + 1.0 / p - (1.0 - c * c))
    z = integrate.quad(f, -1, 1, epsrel=1e-12)[0]
    return np.array([integrate.quad(f, a, b, epsrel=1e-12)[0] for a, b in zip(edges[:-1], edges[1:])]) / z


@pytest.mark.parametrize("e", [0.511, 0.2, 0.05, 0.0101])
def test_kahn_sampler_chi2(nm, e):
    n = 4_000_000
    c = nm.nm_check_kahn(e, n, seed=2024).astype(np.float64)
    assert np.all(c >= -1) and np.all(c <= 1)
    edges = np.linspace(-1, 1, 81)
    p = _kn_bins(e, edges)
    h, _ = np.histogram(c, edges)
    chi2 = ((h - n * p) ** 2 / (n * p)).sum()
    assert stats.chi2.sf(chi2, len(p) - 1) > 1e-4, chi2
    # Mean energy transfer against the same distribution.
    k = e / ME
    mean_ep = np.mean(1.0 / (1.0 + k * (1.0 - c)))
    ref = integrate.quad(lambda x: _kn_w(x, e) / (1 + k * (1 - x)), -1, 1)[0] / integrate.quad(lambda x: _kn_w(x, e), -1, 1)[0]
    record("kn_sampler", sampler="kahn", mev=e, draws=n, chi2_p=stats.chi2.sf(chi2, len(p) - 1),
           mean_e_ratio_rel=mean_ep / ref - 1)
    assert abs(mean_ep - ref) < 5 * np.std(1.0 / (1.0 + k * (1.0 - c))) / math.sqrt(n)


@pytest.mark.parametrize("e", [0.511, 0.2, 0.05, 0.0101, 0.137])
def test_kn_table_sampler_chi2(nm, e):
    # the transport's default sampler: interpolated inverse CDF built for
    # photons between the 10 keV cutoff and 0.511 MeV (0.137 MeV lies between
    # table energies); 16 M draws resolve CDF errors of ~3e-4
    n = 16_000_000
    c = nm.nm_check_kn_table(e, 0.01, 0.511, n, seed=77).astype(np.float64)
    assert np.all(c >= -1) and np.all(c <= 1)
    edges = np.linspace(-1, 1, 81)
    p = _kn_bins(e, edges)
    h, _ = np.histogram(c, edges)
    chi2 = ((h - n * p) ** 2 / (n * p)).sum()
    assert stats.chi2.sf(chi2, len(p) - 1) > 1e-4, chi2
    k = e / ME
    w = 1.0 / (1.0 + k * (1.0 - c))
    ref = integrate.quad(lambda x: _kn_w(x, e) / (1 + k * (1 - x)), -1, 1)[0] / integrate.quad(lambda x: _kn_w(x, e), -1, 1)[0]
    record("kn_sampler", sampler="table", mev=e, draws=n, chi2_p=stats.chi2.sf(chi2, len(p) - 1),
           mean_e_ratio_rel=w.mean() / ref - 1)
    assert abs(w.mean() - ref) < 5 * w.std() / math.sqrt(n)


def _kn_w(c, e):
    k = e / ME
    p = 1.0 / (1.0 + k * (1.0 - c))
    return p * p * (p + 1.0 / p - (1.0 - c * c))


def test_ct_to_phantom_matches_oracle(nm, orc):
    hu = np.arange(-1100, 3072, dtype=np.int16)
    rng = np.random.default_rng(1)
    hu = np.concatenate([hu, rng.integers(-1024, 3072, 100_001).astype(np.int16)])
    den = np.empty(hu.shape, np.float32)
    mat = np.empty(hu.shape, np.uint8)
    nm.nm_ct_to_phantom(hu, den, mat)
    oden, omat = orc.hu_to_phantom(hu)
    record("ct_to_phantom", values=hu.size, material_mismatches=int((mat != omat).sum()),
           max_density_ulps=(np.abs(den - oden) / np.spacing(oden.astype(np.float32))).max())
    assert (mat == omat).all()                              # integer decision: exact
    assert np.all(np.abs(den - oden) <= 2 * np.spacing(oden.astype(np.float32)))  # FP32 vs FP64
    # device pointers, ragged size, empty input
    import torch
    if torch.cuda.is_available():
        t = torch.from_numpy(hu[:777]).cuda()
        d = torch.empty(777, dtype=torch.float32, device="cuda")
        m = torch.empty(777, dtype=torch.uint8, device="cuda")
        nm.nm_ct_to_phantom(t, d, m)
        assert (m.cpu().numpy() == omat[:777]).all()
        assert np.array_equal(d.cpu().numpy(), den[:777])
    nm.nm_ct_to_phantom(hu[:0], den[:0], mat[:0])


def _alias_mass(prob, vox, ali, V):
    mass = np.zeros(V)
    p = prob.astype(np.float64)
    np.add.at(mass, vox, p)
    np.add.at(mass, ali, 1.0 - p)
    return mass / len(prob)


@pytest.mark.parametrize("shape,kind", [((3, 5, 7), "lognormal"), ((17, 13, 11), "sparse"),
                                        ((40, 41, 43), "spiky"), ((1, 1, 1), "single")])
def test_alias_table_reconstructs_pdf(nm, shape, kind):
    rng = np.random.default_rng({"lognormal": 1, "sparse": 2, "spiky": 3, "single": 4}[kind])
    V = int(np.prod(shape))
    if kind == "lognormal":
        act = rng.lognormal(0, 1.0, V)
    elif kind == "sparse":
        act = rng.lognormal(0, 0.3, V) * (rng.random(V) < 0.2)
        act[0] = 0.0
    elif kind == "spiky":
        act = rng.random(V) ** 8
        act[rng.integers(0, V, 5)] = 1e6
        act[rng.random(V) < 0.3] = 0.0
    else:
        act = np.ones(1)
    act = act.astype(np.float32).reshape(shape)
    den = np.ones(shape, np.float32)
    mat = np.zeros(shape, np.uint8)
    m = nm.Materials([0.5551], [7.42])
    with nm.Dose(den, mat, (0.5, 0.5, 0.5), m, activity=act) as d:
        prob, vox, ali = nm.nm_dose_alias_table(d.h)
    active = np.flatnonzero(act.ravel() > 0)
    assert np.array_equal(vox, active)                       # columns in index order
    assert np.all((prob >= 0) & (prob <= 1))
    assert np.all(act.ravel()[ali] > 0)                      # aliases are active voxels
    target = act.ravel().astype(np.float64) / act.astype(np.float64).sum()
    got = _alias_mass(prob, vox, ali, V)
    # each column's split is rounded to FP32 once: error <= (#columns touching v) 2^-24 / n
    touch = np.bincount(ali, minlength=V) + (act.ravel() > 0)
    record("alias_table", voxels=V, max_abs_err=np.abs(got - target).max(),
           max_err_over_bound=(np.abs(got - target) / (touch * 2.0 ** -24 / len(prob) + 1e-15)).max())
    assert np.all(np.abs(got - target) <= touch * 2.0 ** -24 / len(prob) + 1e-15)


def test_source_sampler_follows_activity(nm):
    rng = np.random.default_rng(3)
    shape = (4, 5, 6)
    act = (rng.lognormal(0, 1, shape) * (rng.random(shape) < 0.7)).astype(np.float32)
    den = np.ones(shape, np.float32)
    mat = np.zeros(shape, np.uint8)
    spacing = (0.3, 0.4, 0.5)
    m = nm.Materials([0.5551], [7.42])
    n = 2_000_000
    with nm.Dose(den, mat, spacing, m, activity=act) as d:
        vox, pos, dr = nm.nm_check_source(d.h, 10**12, n, seed=77)
    p = act.ravel().astype(np.float64) / act.sum()
    cnt = np.bincount(vox, minlength=act.size)
    assert cnt[p == 0].sum() == 0
    nz = p > 0
    chi2 = ((cnt[nz] - n * p[nz]) ** 2 / (n * p[nz])).sum()
    record("source_voxels", draws=n, chi2_p=stats.chi2.sf(chi2, nz.sum() - 1))
    assert stats.chi2.sf(chi2, nz.sum() - 1) > 1e-4
    # position inside the sampled voxel, uniform there
    ix, iy, iz = vox % 6, (vox // 6) % 5, vox // 30
    fx = pos[:, 0] / 0.3 - ix
    fy = pos[:, 1] / 0.4 - iy
    fz = pos[:, 2] / 0.5 - iz
    for f in (fx, fy, fz):
        assert f.min() >= -1e-5 and f.max() <= 1 + 1e-5
        h, _ = np.histogram(np.clip(f, 0, 1 - 1e-9), np.linspace(0, 1, 21))
        assert stats.chisquare(h).pvalue > 1e-4
    # isotropic unit directions
    assert np.allclose(np.linalg.norm(dr, axis=1), 1, atol=1e-5)
    assert np.all(np.abs(dr.mean(0)) < 5 / math.sqrt(3 * n))
    h, _ = np.histogram(dr[:, 2], np.linspace(-1, 1, 41))
    assert stats.chisquare(h).pvalue > 1e-4


@pytest.mark.parametrize("kind", ["blocks", "noise"])
def test_organ_voxel_counts_are_exact(nm, kind):
    """The per-organ voxel counts (the denominators of Eq. 2) counted on the
    device, warp-aggregated, against np.bincount of the label map: blocky
    organs (warps mostly see one label) and labels random per voxel (every
    lane a different one)."""
    rng = np.random.default_rng(3)
    shape = (23, 41, 37)
    n_labels = 27
    if kind == "blocks":
        lab = np.zeros(shape, np.uint8)
        for _ in range(40):
            z, y, x = (rng.integers(0, s) for s in shape)
            lab[z:z + rng.integers(2, 9), y:y + rng.integers(3, 15), x:x + rng.integers(3, 15)] = rng.integers(0, 28)
    else:
        lab = rng.integers(0, n_labels + 1, shape).astype(np.uint8)
    den = np.ones(shape, np.float32)
    with nm.Dose(den, np.zeros(shape, np.uint8), (0.5, 0.5, 0.5), nm.Materials([0.5551], [7.42]),
                 activity=np.ones(shape, np.float32), labels=lab, n_labels=n_labels, batches=1) as d:
        d.run(10_000, seed=1)
        _, _, _, cnt = d.organs(eps=False, sigma=False)
    assert np.array_equal(cnt, np.bincount(lab.ravel(), minlength=n_labels + 1))
