"""Argument and state errors come back as status codes with a message."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nm():
    from paper_2111_11687_gb300 import build, nmdose
    build.build()
    nmdose.load()
    return nmdose


def _mk(nm, act=None, den=None, mat=None, labels=None, **kw):
    shape = (4, 5, 6)
    den = np.ones(shape, np.float32) if den is None else den
    mat = np.zeros(shape, np.uint8) if mat is None else mat
    act = np.ones(shape, np.float32) if act is None else act
    return nm.Dose(den, mat, (0.5, 0.5, 0.5), nm.Materials([0.5551], [7.42]), activity=act, labels=labels, **kw)


@pytest.mark.parametrize("case", ["neg_activity", "nan_activity", "zero_activity", "nan_density",
                                  "zero_density", "bad_material", "bad_label", "batches", "point_outside"])
def test_invalid_inputs_are_rejected(nm, case):
    shape = (4, 5, 6)
    kw = {}
    act = den = mat = lab = None
    if case == "neg_activity":
        act = np.ones(shape, np.float32); act[1, 2, 3] = -1
    elif case == "nan_activity":
        act = np.ones(shape, np.float32); act[0, 0, 0] = np.nan
    elif case == "zero_activity":
        act = np.zeros(shape, np.float32)
    elif case == "nan_density":
        den = np.ones(shape, np.float32); den[3, 4, 5] = np.nan
    elif case == "zero_density":
        den = np.ones(shape, np.float32); den[2, 2, 2] = 0
    elif case == "bad_material":
        mat = np.zeros(shape, np.uint8); mat[1, 1, 1] = 1
    elif case == "bad_label":
        # two offending voxels: the message names the first (flat index 8) and its label
        lab = np.zeros(shape, np.uint8); lab[0, 1, 2] = 5; lab[3, 4, 5] = 7
        kw["n_labels"] = 3
    elif case == "batches":
        kw["batches"] = 0
    elif case == "point_outside":
        kw.update(source_mode=nm.NM_SOURCE_POINT, point=(3.0, 0.1, 0.1))
    with pytest.raises(nm.NmError) as e:
        _mk(nm, act, den, mat, lab, **kw)
    assert e.value.status == nm.NM_ERR_ARG
    assert nm.nm_last_error()
    if case == "bad_label":
        assert "label 5 at voxel 8 " in nm.nm_last_error(), nm.nm_last_error()


def test_get_before_run_is_a_state_error(nm):
    with _mk(nm) as d:
        with pytest.raises(nm.NmError) as e:
            d.get()
        assert e.value.status == nm.NM_ERR_STATE
        d.run(1000, seed=1)
        d.get()
        d.reset()
        with pytest.raises(nm.NmError):
            d.get()


def test_overflow_is_refused(nm):
    with _mk(nm) as d:
        with pytest.raises(nm.NmError) as e:
            d.run(2 ** 62, seed=1)
        assert e.value.status == nm.NM_ERR_OVERFLOW


def test_step_limit_reports_device_status(nm):
    # A bounded loop that runs out: photons stop after 2 steps, the run returns
    # NM_ERR_DEVICE, and the stopped energy is accounted for exactly.
    with _mk(nm, max_steps=2) as d:
        with pytest.raises(nm.NmError) as e:
            d.run(20000, seed=1)
        assert e.value.status == nm.NM_ERR_DEVICE
        c = d.counters()
        assert c["killed"] > 0
        assert c["emitted"] == c["deposited"] + c["escaped"] + c["killed"]


def test_bounded_wait_gives_up_and_the_context_survives(nm):
    # the wait every tensor-core kernel uses, on an mbarrier that nothing
    # completes: it must return NM_ERR_TIMEOUT, and the device stays usable
    for cycles in (0, 1_000_000):
        with pytest.raises(nm.NmError) as e:
            nm._check(nm.load().nm_check_wait_timeout(cycles))
        assert e.value.status == nm.NM_ERR_TIMEOUT
    with _mk(nm) as d:
        d.run(10_000, seed=3)
        assert d.counters()["deposited"] > 0


def test_allocation_failures_are_reported_and_leave_nothing_behind(nm):
    import torch
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failed = 0
    try:
        for n in range(1, 40):
            nm.load().nm_debug_fail_alloc(n)
            try:
                with _mk(nm, labels=np.zeros((4, 5, 6), np.uint8), n_labels=2) as d:
                    d.run(1000, seed=1)
            except nm.NmError as e:
                assert e.status == nm.NM_ERR_OOM, e
                failed += 1
            else:
                break   # n is past the last allocation: creation went through
    finally:
        nm.load().nm_debug_fail_alloc(0)
    assert failed >= 10
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (64 << 20)
    with _mk(nm) as d:
        d.run(10_000, seed=3)
        assert d.counters()["deposited"] > 0


def test_device_buffers_are_recycled_and_released(nm):
    """A destroyed handle's buffers stay with the library for the next handle
    of the same grid (the memory is not returned), nm_release_cached_memory
    gives them back, and a handle built on recycled buffers tallies exactly
    what one on fresh buffers does."""
    import torch
    shape = (96, 128, 128)                           # 1.57 M voxels: about 80 MB of handle buffers
    nm.nm_release_cached_memory()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    with _mk(nm, act=np.ones(shape, np.float32), den=np.ones(shape, np.float32),
             mat=np.zeros(shape, np.uint8)) as d:
        d.run(200_000, seed=4)
        t1 = d.tally()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 > 40 * 2 ** 20, (free0, free1)      # kept, not returned
    with _mk(nm, act=np.ones(shape, np.float32), den=np.ones(shape, np.float32),
             mat=np.zeros(shape, np.uint8)) as d:
        d.run(200_000, seed=4)
        t2 = d.tally()
    assert np.array_equal(t1, t2)
    free2 = torch.cuda.mem_get_info()[0]
    assert abs(free2 - free1) < 16 * 2 ** 20, (free1, free2)  # the second handle reused them
    nm.nm_release_cached_memory()
    free3 = torch.cuda.mem_get_info()[0]
    assert free3 - free2 > 40 * 2 ** 20, (free2, free3)      # released
