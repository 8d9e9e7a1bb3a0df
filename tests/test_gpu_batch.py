"""Many patients in one launch (nm_dose_run_batch) and the autotuner.

The batched graph launch must reproduce, bit for bit, each patient's tally and
counters from a plain nm_dose_run with the same seed, whatever the launch
shape, with patients of uneven grids sharing warps; the autotuner must leave
no trace of its trial launches."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nm():
    from paper_2111_11687_gb300 import build, nmdose
    build.build()
    nmdose.load()
    return nmdose


def _setup(nm, ph):
    from paper_2111_11687_gb300 import inputs
    den = np.empty(ph.shape, np.float32)
    mat = np.empty(ph.shape, np.uint8)
    nm.nm_ct_to_phantom(ph.hu, den, mat)
    gm = nm.Materials(inputs.MATERIAL_Z_OVER_A, inputs.MATERIAL_ZEFF, inputs.PE_COEFF, inputs.PE_EXP)
    return den, mat, gm


def _single(nm, ph, n, seed, **kw):
    den, mat, gm = _setup(nm, ph)
    with nm.Dose(den, mat, ph.spacing, gm, activity=ph.activity, labels=ph.labels, n_labels=27, **kw) as d:
        d.run(n, seed=seed)
        return d.tally(), d.counters(), d.organs()


KEYS = ("steps", "compton", "photo", "cutoff", "escapes", "escaped", "deposited", "emitted", "histories")


@pytest.mark.parametrize("shape", [{}, dict(block_threads=128, chunk=64, regroup=1, regroup_lanes=8),
                                   dict(block_threads=256, chunk=1024, regroup=0, warp_aggregate=1)])
def test_batch_equals_single_runs(nm, shape):
    from paper_2111_11687_gb300 import inputs
    phs = [inputs.adult_phantom(shape=s, spacing=d, seed=k) for k, (s, d) in
           enumerate([((30, 24, 24), (2.13, 2.13, 3.0)), ((45, 40, 36), (1.42, 1.28, 2.0)),
                      ((20, 16, 16), (3.2, 3.2, 4.5)), ((33, 29, 31), (1.65, 1.77, 2.73))])]
    ns = [150_000, 0, 60_001, 250_000]
    seed = 42
    handles = []
    try:
        for ph in phs:
            den, mat, gm = _setup(nm, ph)
            handles.append(nm.Dose(den, mat, ph.spacing, gm, activity=ph.activity, labels=ph.labels,
                                   n_labels=27, **shape))
        nm.nm_dose_run_batch(handles, ns, seed)
        for h, ph, n in zip(handles, phs, ns):
            c = h.counters()
            assert c["emitted"] == c["deposited"] + c["escaped"] and c["killed"] == 0
            if n == 0:
                assert c["histories"] == 0 and not h.tally().any()
                continue
            t_ref, c_ref, org_ref = _single(nm, ph, n, seed, **shape)
            assert np.array_equal(h.tally(), t_ref)
            for k in KEYS:
                assert c[k] == c_ref[k], k
            # statistics folded per batch in the graph match the plain run's
            om, oe, osg, cnt = h.organs()
            assert np.array_equal(cnt, org_ref[3])
            assert np.allclose(om, org_ref[0], rtol=1e-12, atol=0)
            assert np.allclose(osg, org_ref[2], rtol=1e-9, atol=0)
        # a second batched call continues the history ids
        nm.nm_dose_run_batch(handles[:1], [50_000], seed)
        t_ref, _, _ = _single(nm, phs[0], 200_000, seed, **shape)
        assert np.array_equal(handles[0].tally(), t_ref)
    finally:
        for h in handles:
            h.close()


def test_batch_rejects_mixed_physics(nm):
    from paper_2111_11687_gb300 import inputs
    ph = inputs.adult_phantom(shape=(10, 8, 8), spacing=(6.4, 6.4, 9.0), seed=1)
    den, mat, gm = _setup(nm, ph)
    gm2 = nm.Materials(inputs.MATERIAL_Z_OVER_A, inputs.MATERIAL_ZEFF, inputs.PE_COEFF * 2, inputs.PE_EXP)
    with nm.Dose(den, mat, ph.spacing, gm, activity=ph.activity) as a, \
            nm.Dose(den, mat, ph.spacing, gm2, activity=ph.activity) as b:
        with pytest.raises(nm.NmError) as e:
            nm.nm_dose_run_batch([a, b], [10, 10], 1)
        assert e.value.status == nm.NM_ERR_ARG
        with pytest.raises(nm.NmError):
            nm.nm_dose_run_batch([a, a], [10, 10], 1)


def test_autotuner_leaves_no_trace(nm):
    from paper_2111_11687_gb300 import inputs
    ph = inputs.adult_phantom(shape=(40, 32, 32), spacing=(1.6, 1.6, 2.25), seed=8)
    t_auto, c_auto, _ = _single(nm, ph, 300_000, 9)            # every knob on auto
    t_fix, c_fix, _ = _single(nm, ph, 300_000, 9, block_threads=256, chunk=256, warp_aggregate=0,
                              regroup=1, regroup_lanes=12)
    assert np.array_equal(t_auto, t_fix)
    for k in KEYS:
        assert c_auto[k] == c_fix[k], k
    assert c_auto["block_threads"] in (128, 256, 512) and c_auto["chunk"] in (64, 256, 1024)


def test_sixteen_uneven_patients_in_one_graph(nm):
    # The batched-patients workload: 16 seeded phantoms with grids from
    # 128x128x160 to 256x256x320 and 2-4 mm voxels, 2e6 decays each here
    # (the property holds at any count); every patient bit-identical to its own run.
    from paper_2111_11687_gb300 import inputs
    phs = inputs.batch_phantoms(16)
    n = 2_000_000
    handles = []
    try:
        for ph in phs:
            den, mat, gm = _setup(nm, ph)
            handles.append(nm.Dose(den, mat, ph.spacing, gm, activity=ph.activity, labels=ph.labels, n_labels=27))
        nm.nm_dose_run_batch(handles, [n] * 16, 5)
        for i in (0, 7, 15):
            t_ref, c_ref, _ = _single(nm, phs[i], n, 5)
            assert np.array_equal(handles[i].tally(), t_ref)
        for h in handles:
            c = h.counters()
            assert c["emitted"] == c["deposited"] + c["escaped"] and c["histories"] == n
    finally:
        for h in handles:
            h.close()
