"""Bit-identical tallies: a history's random numbers depend only on (seed,
history id) and the tally is int64, so launch shape, warp aggregation, event
regrouping and the split into run calls must not change a single bit."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nm():
    from paper_2111_11687_gb300 import build, nmdose
    build.build()
    nmdose.load()
    return nmdose


@pytest.fixture(scope="module")
def phantom(nm):
    from paper_2111_11687_gb300 import inputs
    ph = inputs.adult_phantom(shape=(50, 40, 40), spacing=(1.28, 1.28, 1.8), seed=5)
    den = np.empty(ph.shape, np.float32)
    mat = np.empty(ph.shape, np.uint8)
    nm.nm_ct_to_phantom(ph.hu, den, mat)
    gm = nm.Materials(inputs.MATERIAL_Z_OVER_A, inputs.MATERIAL_ZEFF, inputs.PE_COEFF, inputs.PE_EXP)
    return ph, den, mat, gm


def _tally(nm, phantom, runs, **kw):
    ph, den, mat, gm = phantom
    with nm.Dose(den, mat, ph.spacing, gm, activity=ph.activity, labels=ph.labels, n_labels=27, **kw) as d:
        for n, seed in runs:
            d.run(n, seed=seed)
        t = d.tally()
        c = d.counters()
    assert c["emitted"] == c["deposited"] + c["escaped"] and c["killed"] == 0
    return t, c


def test_same_seed_same_bits_any_launch_shape(nm, phantom):
    ref, c0 = _tally(nm, phantom, [(300_001, 5)])
    for kw in [dict(block_threads=128), dict(block_threads=512, chunk=1024), dict(chunk=32),
               dict(warp_aggregate=1), dict(warp_aggregate=0), dict(regroup=1),
               dict(regroup=1, warp_aggregate=1, block_threads=64), dict(batches=3)]:
        t, c = _tally(nm, phantom, [(300_001, 5)], **kw)
        assert np.array_equal(t, ref), kw
        for k in ("steps", "compton", "photo", "escapes", "escaped", "deposited"):
            assert c[k] == c0[k], (kw, k)


def test_split_runs_equal_one_run(nm, phantom):
    ref, _ = _tally(nm, phantom, [(250_000, 11)])
    t, c = _tally(nm, phantom, [(100_003, 11), (1, 11), (149_996, 11)])
    assert np.array_equal(t, ref)
    assert c["histories"] == 250_000


def test_other_seed_other_bits(nm, phantom):
    a, _ = _tally(nm, phantom, [(100_000, 1)])
    b, _ = _tally(nm, phantom, [(100_000, 2)])
    assert not np.array_equal(a, b)
    # but the same expected dose: totals within statistics
    assert abs(a.sum() / b.sum() - 1) < 0.01


def test_point_source_repeat(nm):
    from paper_2111_11687_gb300 import inputs
    cube = inputs.water_cube(32, 0.5)
    gm = nm.Materials(inputs.WATER_Z_OVER_A, inputs.WATER_ZEFF)
    out = []
    for wa in (0, 1):
        with nm.Dose(cube.density, cube.material, cube.spacing, gm, source_mode=nm.NM_SOURCE_POINT,
                     point=cube.point, warp_aggregate=wa) as d:
            d.run(200_000, seed=3)
            out.append(d.tally())
    assert np.array_equal(out[0], out[1])


def test_one_batch_per_call_equals_the_same_batches_in_one_call(nm, phantom):
    """Batches may be split over run calls: two calls of one batch each give
    the batches of one two-batch call (the same histories in the same order),
    so the statistics are the same bits; the organ means are available after
    one batch, the uncertainties from the second on (odd and even batches run
    on different streams, their folds in batch order)."""
    ph, den, mat, gm = phantom
    n = 400_000
    shape = den.shape
    res = []
    for batches, calls in ((2, [n]), (1, [n // 2, n // 2])):
        with nm.Dose(den, mat, ph.spacing, gm, activity=ph.activity, labels=ph.labels, n_labels=27,
                     batches=batches) as d:
            for k, m in enumerate(calls):
                d.run(m, seed=6)
                if batches == 1 and k == 0:
                    mean1, _, sig1, _ = d.organs(eps=False, sigma=False)
                    assert sig1 is None and np.all(np.isfinite(mean1))
                    with pytest.raises(nm.NmError):
                        d.organs(eps=False)          # the batch sigma needs two batches
            dose = np.empty(shape, np.float32)
            sigma = np.empty(shape, np.float32)
            nm.nm_dose_get(d.h, dose, sigma, None)
            mean, _, sig, _ = d.organs(eps=False)
            res.append((d.tally(), dose, sigma, mean, sig, d.counters()["batches"]))
    a, b = res
    assert a[5] == b[5] == 2
    for x, y in zip(a[:5], b[:5]):
        assert np.array_equal(x, y)
