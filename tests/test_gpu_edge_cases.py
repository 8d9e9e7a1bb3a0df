"""Degenerate inputs through the C ABI: no histories, one history, fewer
histories than a warp, a one-voxel grid, a point source on the grid's corner.
Every case keeps the exact energy bookkeeping and the documented statuses."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nm():
    from paper_2111_11687_gb300 import build, nmdose
    build.build()
    nmdose.load()
    return nmdose


def _water(nm):
    return nm.Materials([0.5551], [7.42], 2e-9, 3.8)


def _balanced(c):
    return c["deposited"] + c["escaped"] + c["killed"] == c["emitted"]


def test_zero_histories_change_nothing(nm):
    shape = (3, 4, 5)
    with nm.Dose(np.ones(shape, np.float32), np.zeros(shape, np.uint8), (0.5,) * 3, _water(nm),
                 activity=np.ones(shape, np.float32)) as d:
        d.run(0, seed=1)
        c = d.counters()
        assert c["histories"] == 0 and c["batches"] == 0 and c["emitted"] == 0
        with pytest.raises(nm.NmError) as e:
            d.get()
        assert e.value.status == nm.NM_ERR_STATE
        assert not d.tally().any()


def test_one_history_and_fewer_than_a_warp(nm):
    shape = (6, 6, 6)
    act = np.zeros(shape, np.float32)
    act[2, 3, 1] = 1.0
    for n in (1, 7, 31):
        with nm.Dose(np.ones(shape, np.float32), np.zeros(shape, np.uint8), (0.4,) * 3, _water(nm),
                     activity=act) as d:
            d.run(n, seed=5)
            c = d.counters()
            assert c["histories"] == n and _balanced(c)
            assert int(d.tally().sum()) == c["deposited"]
            dose = np.empty(shape, np.float32)
            nm.nm_dose_get(d.h, dose, None, None)        # the dose alone needs no second batch
            assert np.all(np.isfinite(dose)) and dose[2, 3, 1] > 0
            if c["batches"] < 2:
                with pytest.raises(nm.NmError) as e:
                    d.get()                               # sigma needs two batches
                assert e.value.status == nm.NM_ERR_STATE
    # the same few histories on another launch shape give the same tally
    ts = []
    for kw in ({}, dict(block_threads=128, chunk=64, regroup=0)):
        with nm.Dose(np.ones(shape, np.float32), np.zeros(shape, np.uint8), (0.4,) * 3, _water(nm),
                     activity=act, **kw) as d:
            d.run(7, seed=5)
            ts.append(d.tally())
    np.testing.assert_array_equal(ts[0], ts[1])


def test_one_voxel_grid(nm):
    shape = (1, 1, 1)
    with nm.Dose(np.ones(shape, np.float32), np.zeros(shape, np.uint8), (2.0,) * 3, _water(nm),
                 activity=np.ones(shape, np.float32)) as d:
        d.run(100_000, seed=2)
        c = d.counters()
        dose, sigma = d.get()
        assert _balanced(c) and c["killed"] == 0
        # the positron always stays; most photons leave a 2 cm cube of water
        q = lambda e: int(np.rint(np.float32(e) * np.float32(6.4e7)))
        assert c["deposited"] >= 100_000 * q(0.25) and c["escaped"] > c["deposited"]
        assert np.isfinite(dose).all() and dose[0, 0, 0] > 0 and sigma[0, 0, 0] > 0


def test_point_source_on_the_grid_corner(nm):
    shape = (8, 8, 8)
    with nm.Dose(np.ones(shape, np.float32), np.zeros(shape, np.uint8), (0.5,) * 3, _water(nm),
                 source_mode=nm.NM_SOURCE_POINT, point=(0.0, 0.0, 0.0)) as d:
        d.run(200_000, seed=3)
        c = d.counters()
        t = d.tally()
    assert _balanced(c) and c["killed"] == 0
    # a point on a plane belongs to the upper voxel: the corner voxel is inside
    assert t[0, 0, 0] > 0 and int(t.sum()) == c["deposited"]
