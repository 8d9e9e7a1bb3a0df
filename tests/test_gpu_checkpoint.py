"""Shards, checkpoints and merges of a handle's statistics through the C ABI.

A history's random numbers depend only on (seed, history id), so shards of
one run on disjoint id ranges, merged, must give the tally, the counters and
the dose of the whole run bit for bit; a restored checkpoint must continue
exactly as the handle that wrote it.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N = 3_000_000
SPLIT = 1_234_567
SEED = 5


@pytest.fixture(scope="module")
def nm():
    from paper_2111_11687_gb300 import build, nmdose
    build.build()
    nmdose.load()
    return nmdose


@pytest.fixture(scope="module")
def case(nm):
    from paper_2111_11687_gb300 import inputs
    ph = inputs.adult_phantom(shape=(60, 48, 48), spacing=(1.0, 1.0, 1.5), seed=13)
    den = np.empty(ph.shape, np.float32)
    mat = np.empty(ph.shape, np.uint8)
    nm.nm_ct_to_phantom(ph.hu, den, mat)
    gm = nm.Materials(inputs.MATERIAL_Z_OVER_A, inputs.MATERIAL_ZEFF, inputs.PE_COEFF, inputs.PE_EXP)
    return ph, den, mat, gm, inputs.N_LABELS


def _dose(nm, case, **kw):
    ph, den, mat, gm, nl = case
    return nm.Dose(den, mat, ph.spacing, gm, activity=ph.activity, labels=ph.labels, n_labels=nl, **kw)


_SUMMED = ("histories", "emitted", "deposited", "escaped", "killed", "steps", "compton", "photo", "rayleigh",
           "cutoff", "escapes")


@pytest.mark.parametrize("device_image", [False, True])
def test_merged_shards_equal_the_whole_run(nm, case, device_image):
    import torch
    with _dose(nm, case) as whole, _dose(nm, case) as a, _dose(nm, case) as b, _dose(nm, case) as seq:
        whole.run(N, SEED)
        a.run(SPLIT, SEED)                 # ids [0, SPLIT)
        b.seek(SPLIT)
        b.run(N - SPLIT, SEED)             # ids [SPLIT, N)
        seq.run(SPLIT, SEED)               # the same two runs, in turn, on one handle
        seq.run(N - SPLIT, SEED)
        img = b.checkpoint()
        assert img.nbytes == b.checkpoint_size()
        if device_image:
            img = torch.from_numpy(img).cuda()
        a.merge(img)
        tw, ta = whole.tally(), a.tally()
        np.testing.assert_array_equal(ta, tw)
        cw, ca, cs = whole.counters(), a.counters(), seq.counters()
        for k in _SUMMED:
            assert ca[k] == cw[k], k
        assert ca["batches"] == cs["batches"] == 20
        dw, _ = whole.get()
        da, sa = a.get()
        ds, ss = seq.get()
        np.testing.assert_array_equal(da, dw)
        # the merged batch sums equal the sequential handle's up to the FP64 order
        np.testing.assert_allclose(sa, ss, rtol=1e-5, atol=0)
        ow, oa = whole.organs(), a.organs()
        np.testing.assert_array_equal(oa[0], ow[0])
        # the next id after a merge is the larger of the two
        a.run(1000, SEED)
        seq.run(1000, SEED)
        np.testing.assert_array_equal(a.tally(), seq.tally())


def test_restored_checkpoint_continues_exactly(nm, case):
    with _dose(nm, case, history_sigma=1) as d, _dose(nm, case, history_sigma=1) as e:
        d.run(SPLIT, SEED)
        img = d.checkpoint()
        e.run(77_777, SEED + 1)            # state that the restore must replace
        e.restore(img)
        d.run(N - SPLIT, SEED)
        e.run(N - SPLIT, SEED)
        np.testing.assert_array_equal(e.tally(), d.tally())
        dd, sd = d.get()
        de, se = e.get()
        np.testing.assert_array_equal(de, dd)
        np.testing.assert_array_equal(se, sd)
        np.testing.assert_array_equal(e.history_sigma(), d.history_sigma())
        cd, ce = d.counters(), e.counters()
        for k in _SUMMED + ("batches", "history_splits"):
            assert ce[k] == cd[k], k


def test_history_sums_merge_exactly(nm, case):
    with _dose(nm, case, history_sigma=1) as whole, _dose(nm, case, history_sigma=1) as a, \
            _dose(nm, case, history_sigma=1) as b:
        whole.run(N, SEED)
        a.run(SPLIT, SEED)
        b.seek(SPLIT)
        b.run(N - SPLIT, SEED)
        a.merge(b.checkpoint())
        # 128-bit sums of squared history totals add exactly: same sigma bit for bit
        np.testing.assert_array_equal(a.history_sigma(), whole.history_sigma())


def test_mismatched_images_are_refused(nm, case):
    from paper_2111_11687_gb300.nmdose import NmError
    ph, den, mat, gm, nl = case
    with _dose(nm, case) as d, _dose(nm, case, history_sigma=1) as h, \
            nm.Dose(den[:, :, :40].copy(), mat[:, :, :40].copy(), ph.spacing, gm,
                    activity=ph.activity[:, :, :40].copy()) as small:
        d.run(100_000, SEED)
        t0 = d.tally()
        img = d.checkpoint()
        for target in (h, small):
            with pytest.raises(NmError):
                target.restore(img)
            with pytest.raises(NmError):
                target.merge(img)
        with pytest.raises(NmError):
            d.restore(img[:-8].copy())
        bad = img.copy()
        bad[0] ^= 0xFF
        with pytest.raises(NmError):
            d.merge(bad)
        with pytest.raises(NmError):
            d.checkpoint(np.empty(img.nbytes - 1, np.uint8))
        with pytest.raises(NmError):
            d.seek((1 << 62) + 1)
        np.testing.assert_array_equal(d.tally(), t0)
