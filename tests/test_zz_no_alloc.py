"""The allocation-free tally entry point, for callers that cannot call
cudaMalloc (they run inside another framework's memory pool, or under a
no-allocation-after-start-up rule).  Its tallies must equal, bit for bit, the
tallies of the ordinary handle path (nm_dose_create + nm_dose_run +
nm_dose_get_tally) on the same inputs and seed, on consecutive calls that
reuse the same fixed scratch array.  This file is collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nm():
    from paper_2111_11687_gb300 import build, nmdose
    build.build()
    nmdose.load()
    return nmdose


def _handle_tally(nm, den, mat, spacing, m, n, seed, **kw):
    with nm.Dose(den, mat, spacing, m, **kw) as d:
        d.run(n, seed=seed)
        return d.tally()


def test_noalloc_matches_handle_path_on_consecutive_calls(nm):
    import torch
    from paper_2111_11687_gb300 import inputs

    # Call 1: point source in a 32^3 water cube.
    cube = inputs.water_cube(32, 0.5)
    wm = nm.Materials(inputs.WATER_Z_OVER_A, inputs.WATER_ZEFF, inputs.PE_COEFF, inputs.PE_EXP)
    ref1 = _handle_tally(nm, cube.density, cube.material, cube.spacing, wm, 300_000, 7,
                         source_mode=nm.NM_SOURCE_POINT, point=cube.point)
    den1 = torch.from_numpy(cube.density).cuda()
    mat1 = torch.from_numpy(cube.material).cuda()
    out1 = torch.full(cube.density.shape, -1, dtype=torch.int64, device="cuda")
    c1 = nm.nm_dose_tally_noalloc(den1, mat1, cube.spacing, wm, out1, 300_000, 7,
                                  opts=nm.options(source_mode=nm.NM_SOURCE_POINT, point=cube.point))
    assert np.array_equal(out1.cpu().numpy(), ref1)
    assert c1["emitted"] == c1["deposited"] + c1["escaped"] and c1["device_status"] == 0

    # Call 2, straight after on the same scratch: decay mode on a 40x36x30
    # phantom (different size, alias table built in the scratch array).
    ph = inputs.adult_phantom(shape=(30, 36, 40), spacing=(1.28, 1.42, 3.0), seed=4)
    den = np.empty(ph.shape, np.float32)
    mat = np.empty(ph.shape, np.uint8)
    nm.nm_ct_to_phantom(ph.hu, den, mat)
    pm = nm.Materials(inputs.MATERIAL_Z_OVER_A, inputs.MATERIAL_ZEFF, inputs.PE_COEFF, inputs.PE_EXP)
    ref2 = _handle_tally(nm, den, mat, ph.spacing, pm, 200_001, 3, activity=ph.activity)
    out2 = torch.zeros(ph.shape, dtype=torch.int64, device="cuda")
    c2 = nm.nm_dose_tally_noalloc(torch.from_numpy(den).cuda(), torch.from_numpy(mat).cuda(), ph.spacing, pm,
                                  out2, 200_001, 3, activity=torch.from_numpy(ph.activity).cuda())
    assert np.array_equal(out2.cpu().numpy(), ref2)
    assert int(out2.sum().item()) == c2["deposited"]

    # Call 3: the first problem again gives the first answer again.
    out1b = torch.zeros_like(out1)
    nm.nm_dose_tally_noalloc(den1, mat1, cube.spacing, wm, out1b, 300_000, 7,
                             opts=nm.options(source_mode=nm.NM_SOURCE_POINT, point=cube.point))
    assert torch.equal(out1b, out1)


def test_noalloc_at_its_voxel_limit_in_decay_mode(nm):
    """Exactly 64^3 = 2^18 voxels, the documented maximum, in decay mode: the
    packed voxels, the alias table and the alias build's FP64 scans all fit in
    the fixed array, and the tally equals the handle path's bit for bit."""
    import torch
    from paper_2111_11687_gb300 import inputs

    ph = inputs.adult_phantom(shape=(64, 64, 64), spacing=(0.8, 0.8, 1.40625), seed=6)
    den = np.empty(ph.shape, np.float32)
    mat = np.empty(ph.shape, np.uint8)
    nm.nm_ct_to_phantom(ph.hu, den, mat)
    pm = nm.Materials(inputs.MATERIAL_Z_OVER_A, inputs.MATERIAL_ZEFF, inputs.PE_COEFF, inputs.PE_EXP)
    ref = _handle_tally(nm, den, mat, ph.spacing, pm, 400_000, 9, activity=ph.activity)
    out = torch.full(ph.shape, -1, dtype=torch.int64, device="cuda")
    c = nm.nm_dose_tally_noalloc(torch.from_numpy(den).cuda(), torch.from_numpy(mat).cuda(), ph.spacing, pm,
                                 out, 400_000, 9, activity=torch.from_numpy(ph.activity).cuda())
    assert np.array_equal(out.cpu().numpy(), ref)
    assert c["device_status"] == 0 and int(out.sum().item()) == c["deposited"]


def _raw_call(nm, shape, spacing, m, density_ptr, material_ptr, activity_ptr, tally_ptr, opts=None):
    """nm_dose_tally_noalloc through the C ABI directly, past the binding's own
    checks, so that the library's checks are the ones exercised."""
    import ctypes as C
    nz, ny, nx = shape
    g = nm.nm_grid(nx, ny, nz, *map(float, spacing), density_ptr, material_ptr)
    mc = m.c()
    c = nm.nm_counters()
    return nm.load().nm_dose_tally_noalloc(C.byref(g), C.byref(mc), activity_ptr,
                                           C.byref(opts) if opts is not None else None, 1000, 1, tally_ptr,
                                           C.byref(c))


def test_noalloc_rejects_oversized_grids_host_pointers_and_bad_options(nm):
    import torch
    from paper_2111_11687_gb300 import inputs

    wm = nm.Materials(inputs.WATER_Z_OVER_A, inputs.WATER_ZEFF)
    big = torch.ones((65, 64, 64), dtype=torch.float32, device="cuda")   # 266240 > 2^18 voxels
    bm = torch.zeros((65, 64, 64), dtype=torch.uint8, device="cuda")
    out = torch.zeros((65, 64, 64), dtype=torch.int64, device="cuda")
    o = nm.options(source_mode=nm.NM_SOURCE_POINT, point=(1.0, 1.0, 1.0))
    with pytest.raises(nm.NmError) as e:
        nm.nm_dose_tally_noalloc(big, bm, (0.5, 0.5, 0.5), wm, out, 1000, 1, opts=o)
    assert e.value.status == nm.NM_ERR_ARG and "limit" in nm.nm_last_error()

    shape = (8, 8, 8)
    host_den = np.ones(shape, np.float32)
    host_mat = np.zeros(shape, np.uint8)
    dev_tally = torch.zeros(shape, dtype=torch.int64, device="cuda")
    st = _raw_call(nm, shape, (0.5, 0.5, 0.5), wm, host_den.ctypes.data, host_mat.ctypes.data, None,
                   dev_tally.data_ptr(), o)
    assert st == nm.NM_ERR_ARG and "device" in nm.nm_last_error()

    # Options and spacing that nm_dose_create refuses are refused here too,
    # on the host, before any fixed-point unit is derived from them.
    den = torch.ones(shape, dtype=torch.float32, device="cuda")
    mat = torch.zeros(shape, dtype=torch.uint8, device="cuda")
    act = torch.ones(shape, dtype=torch.float32, device="cuda")
    for bad in (-1.022, float("nan"), 2.0):
        with pytest.raises(nm.NmError) as e:
            nm.nm_dose_tally_noalloc(den, mat, (0.5, 0.5, 0.5), wm, dev_tally, 1000, 1, activity=act,
                                     opts=nm.options(positron_mev=bad))
        assert e.value.status == nm.NM_ERR_ARG and "positron" in nm.nm_last_error()
    with pytest.raises(nm.NmError) as e:
        nm.nm_dose_tally_noalloc(den, mat, (float("inf"), 0.5, 0.5), wm, dev_tally, 1000, 1, activity=act)
    assert e.value.status == nm.NM_ERR_ARG and "voxel sizes" in nm.nm_last_error()
    with pytest.raises(nm.NmError) as e:
        nm.nm_dose_tally_noalloc(den, mat, (0.5, 0.5, 0.5), nm.Materials([-0.5], [7.42]), dev_tally, 1000, 1,
                                 activity=act)
    assert e.value.status == nm.NM_ERR_ARG
    # the array is still usable after the refusals
    nm.nm_dose_tally_noalloc(den, mat, (0.5, 0.5, 0.5), wm, dev_tally, 1000, 1, activity=act)
    assert int(dev_tally.sum().item()) > 0
