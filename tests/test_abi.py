"""CPU checks of the C ABI boundary: the library builds and exports every entry
point that include/nm_dose.h declares, the binding covers them, the product
never touches the oracle, and the oracle never touches the product."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "nm_dose.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nm_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2111_11687_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header(lib_path):
    from paper_2111_11687_gb300 import nmdose
    assert sorted(nmdose.symbols()) == declared_functions()
    nmdose.load()


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2111_11687_gb300 import nmdose
    monkeypatch.setattr(nmdose, "_lib", None)
    monkeypatch.setattr(nmdose, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        nmdose.load()


def test_options_default_without_gpu(lib_path):
    from paper_2111_11687_gb300 import nmdose
    o = nmdose.options()
    assert o.batches == 10 and o.source_mode == nmdose.NM_SOURCE_DECAY
    assert abs(o.photon_mev - 0.511) < 1e-12 and abs(o.positron_mev - 0.25) < 1e-12
    # A(t_s): 8.0 mCi after 60 min of decay with T1/2 = 109.77 min.
    assert abs(o.activity_bq / (8e-3 * 3.7e10 * 2 ** (-60 / 109.77)) - 1) < 1e-12


def test_product_and_oracle_share_nothing():
    pkg = os.path.join(ROOT, "paper_2111_11687_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, flags=re.M), f
                assert "nm_oracle" not in text and "liboracle" not in text, f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".cpp")):
            text = open(os.path.join(ROOT, "oracle", f)).read()
            assert not re.search(r"^\s*(import|from)\s+paper_2111_11687_gb300\b", text, flags=re.M), f
            assert "nm_dose.h" not in text and "libnmdose" not in text, f
            assert "nm_internal" not in text, f


class _NoCalls:
    """Stands in for the library: any entry point that is reached fails the test."""

    def __getattr__(self, name):
        raise AssertionError(f"{name} was called with mismatched buffers")


def test_binding_rejects_mismatched_buffers_before_the_call(monkeypatch):
    """The C side cannot see the size or element type of a device buffer, so
    the binding checks both before a pointer crosses the ABI."""
    import numpy as np

    from paper_2111_11687_gb300 import nmdose
    monkeypatch.setattr(nmdose, "_lib", _NoCalls())
    shape = (4, 5, 6)
    den = np.ones(shape, np.float32)
    mat = np.zeros(shape, np.uint8)
    act = np.ones(shape, np.float32)
    m = nmdose.Materials([0.5551], [7.42])
    bad = [
        dict(density=den.astype(np.float64)),          # wrong element type
        dict(material=np.zeros(shape, np.int32)),
        dict(activity=np.ones((4, 5, 5), np.float32)),  # wrong size
        dict(labels=np.zeros(shape, np.int8)),
    ]
    for kw in bad:
        args = dict(density=den, material=mat, activity=act, labels=None)
        args.update(kw)
        with pytest.raises(ValueError):
            nmdose.nm_dose_create(args["density"], args["material"], (0.5, 0.5, 0.5), m, args["activity"],
                                  args["labels"])
    with pytest.raises(ValueError):
        nmdose.nm_ct_to_phantom(np.zeros(shape, np.int16), den, np.zeros(shape[:2], np.uint8))
    # The allocation-free tally writes 8 bytes per voxel into `tally`: host
    # arrays, an int32 tally or a short one never reach the library.
    for tally in (np.zeros(shape, np.int64), np.zeros(shape, np.int32), np.zeros(10, np.int64)):
        with pytest.raises(ValueError):
            nmdose.nm_dose_tally_noalloc(den, mat, (0.5, 0.5, 0.5), m, tally, 1000, 1, activity=act)


def test_raw_getters_check_buffers_against_the_handle(monkeypatch):
    """nm_dose_get and nm_dose_get_tally write V values (and n_labels + 1 organ
    means) through raw pointers: for a handle made by the binding, buffers of
    another size or type, or non-contiguous ones, are refused before the call."""
    import numpy as np

    from paper_2111_11687_gb300 import nmdose
    monkeypatch.setattr(nmdose, "_lib", _NoCalls())
    fake = 0x1234
    monkeypatch.setitem(nmdose._HANDLE_GRID, fake, (120, 27))
    good = np.empty(120, np.float32)
    for kw in (dict(dose=np.empty(119, np.float32)), dict(dose=np.empty(120, np.float64)),
               dict(sigma=np.empty(121, np.float32)), dict(organ_dose=np.empty(27))):
        args = dict(dose=good, sigma=None, organ_dose=None)
        args.update(kw)
        with pytest.raises(ValueError):
            nmdose.nm_dose_get(fake, **args)
    for tally in (np.empty(120, np.int32), np.empty(100, np.int64)):
        with pytest.raises(ValueError):
            nmdose.nm_dose_get_tally(fake, tally)
    with pytest.raises(ValueError):
        nmdose.nm_dose_get(fake, np.empty((240,), np.float32)[::2], None, None)   # not contiguous
