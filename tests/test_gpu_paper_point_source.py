"""The paper's own validation case (§2.2): a 0.511 MeV point photon source in
water, CT and PET of 101^3 voxels of 0.5 mm, the source in the central PET
voxel, 1e8 decays, compared through the dose-distance curve and the mean
difference over the voxels above 10 % of the maximum dose (the paper states
under 0.3 % against GATE; here the FP64 oracle takes GATE's place).

Every decay gives two back-to-back photons from a uniform point inside the
central voxel; the paper's source is a photon source, so no positron energy
is deposited (positron_mev = 0)."""
import time

import numpy as np
import pytest

from parity_record import map_figures, record
from test_gpu_parity import organ_check, shells

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nm():
    from paper_2111_11687_gb300 import build, nmdose
    build.build()
    nmdose.load()
    return nmdose


def test_paper_point_source_matches_oracle(nm, orc):
    from paper_2111_11687_gb300 import inputs
    ph = inputs.paper_point_source()
    n = ph.hu.shape[0]
    c = (n // 2 + 0.5) * ph.spacing[0]
    lab = shells(ph.hu.shape, ph.spacing, (c, c, c), 0.1, 15)    # 1 mm shells
    den = np.empty(ph.hu.shape, np.float32)
    mat = np.empty(ph.hu.shape, np.uint8)
    nm.nm_ct_to_phantom(ph.hu, den, mat)
    gm = nm.Materials(inputs.MATERIAL_Z_OVER_A, inputs.MATERIAL_ZEFF, inputs.PE_COEFF, inputs.PE_EXP)
    N = 100_000_000
    with nm.Dose(den, mat, ph.spacing, gm, activity=ph.activity, labels=lab, n_labels=15, positron_mev=0.0,
                 activity_bq=1.0, batches=20) as d:
        d.run(1_000_000, seed=3)               # warm-up and launch-shape choice
        d.reset()
        import torch
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d.run(N, seed=1)
        g, sg = d.get()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        gmean, _, gsig, cnt = d.organs()
        cn = d.counters()
    print(f"paper point source: {N:.0e} decays in {wall * 1e3:.1f} ms on the GPU (paper: 2.4 s on a Titan V)")
    assert cn["emitted"] == cn["deposited"] + cn["escaped"] and cn["killed"] == 0
    No = 20_000_000
    oden, omat = orc.hu_to_phantom(ph.hu)
    om = orc.Materials(inputs.MATERIAL_Z_OVER_A, inputs.MATERIAL_ZEFF, inputs.PE_COEFF, inputs.PE_EXP)
    r = orc.run(oden, omat, om, activity=ph.activity, labels=lab, n_labels=15, spacing=ph.spacing, n_hist=No,
                seed=2, batches=20, positron_mev=0.0)
    # voxel criterion: the central voxel holds every source point, so the dose
    # falls steeply; the criterion runs over the voxels above 0.5 % of the maximum
    top = r.dose_rate > 0.005 * r.dose_rate.max()
    comb = np.sqrt(sg.astype(np.float64) ** 2 + r.sigma ** 2)
    zv = (g.astype(np.float64) - r.dose_rate) / comb
    ctr = ph.hu.shape[0] // 2
    print(f"central voxel: gpu {g[ctr, ctr, ctr]:.6g} oracle {r.dose_rate[ctr, ctr, ctr]:.6g} z {zv[ctr, ctr, ctr]:.2f}; "
          f"|z| > 3 in {(np.abs(zv[top]) > 3).sum()} of {top.sum()} voxels")
    zz, yy, xx = np.nonzero(top & (np.abs(zv) > 3))
    print(f"z over those voxels: mean {zv[top].mean():.3f} std {zv[top].std():.3f}; |z| > 3 at distances (voxels) "
          f"{np.round(np.sqrt((zz - ctr) ** 2 + (yy - ctr) ** 2 + (xx - ctr) ** 2), 1).tolist()}")
    # 20 batches per side: |t| > 3 with ~38 degrees of freedom has probability ~0.5 %
    frac, nsel = (np.abs(zv[top]) <= 3).mean(), top.sum()
    record("dose_map", **map_figures(g, r.dose_rate, r.sigma, top, comb))
    assert nsel > 500 and frac >= 0.99, (frac, nsel)
    zmax, npow, worst, z, sel = organ_check(gmean, gsig, r.organ_mean, r.organ_sigma, cnt, min_voxels=1)
    assert zmax < 4.0, z[sel]
    assert npow >= 5 and worst < 0.01, (npow, worst)
    # the paper's metric: mean |relative difference| over the voxels above 10 %
    # of the maximum.  Against a 2e7-decay oracle it is set by the oracle's own
    # noise, so it is compared with the mean combined relative sigma there.
    hi = r.dose_rate > 0.1 * r.dose_rate.max()
    rel = np.abs(g[hi].astype(np.float64) / r.dose_rate[hi] - 1)
    comb = np.sqrt(sg[hi].astype(np.float64) ** 2 + r.sigma[hi] ** 2) / r.dose_rate[hi]
    print(f"voxels above 10 % of max: {hi.sum()}, mean |diff| {rel.mean() * 100:.2f} %, "
          f"mean combined sigma {comb.mean() * 100:.2f} %")
    record("paper_metric", voxels=int(hi.sum()), mean_abs_rel=rel.mean(), mean_combined_rel_sigma=comb.mean(),
           gpu_ms=wall * 1e3)
    assert rel.mean() < 1.5 * comb.mean() * np.sqrt(2 / np.pi) + 1e-3
