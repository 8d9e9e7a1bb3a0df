"""The recorder of agreement figures: silent unless NM_PARITY_REPORT is set,
one JSON line per call otherwise, with NumPy values made plain; the voxel-map
figures on a case whose answer is known by construction."""
import json

import numpy as np

from tests.parity_record import map_figures, record


def test_record_is_silent_without_the_variable(tmp_path, monkeypatch):
    monkeypatch.delenv("NM_PARITY_REPORT", raising=False)
    monkeypatch.chdir(tmp_path)
    record("x", a=1.0)
    assert list(tmp_path.iterdir()) == []


def test_record_appends_plain_json(tmp_path, monkeypatch):
    out = tmp_path / "r.jsonl"
    monkeypatch.setenv("NM_PARITY_REPORT", str(out))
    record("a", f=np.float32(0.5), i=np.int64(3), b=np.bool_(True), v=np.arange(3), t=(1, 2.5), n=None)
    record("b", f=1.0)
    lines = [json.loads(l) for l in out.read_text().splitlines()]
    assert [l["kind"] for l in lines] == ["a", "b"]
    assert lines[0]["f"] == 0.5 and lines[0]["i"] == 3 and lines[0]["b"] is True
    assert lines[0]["v"] == [0, 1, 2] and lines[0]["t"] == [1, 2.5] and lines[0]["n"] is None
    assert "test_record_appends_plain_json" in lines[0]["test"]


def test_map_figures_on_a_known_offset():
    rng = np.random.default_rng(1)
    o = rng.uniform(1.0, 2.0, (6, 7, 8))
    g = o * 1.02                       # every selected voxel 2 % high
    so = 0.01 * o                      # the oracle's relative sigma: 1 %
    sg = 0.01 * g
    comb = np.sqrt(sg ** 2 + so ** 2)
    sel = np.zeros(o.shape, bool)
    sel[1:5, 2:6, 3:7] = True
    f = map_figures(g, o, so, sel, comb)
    assert f["voxels"] == 64
    assert np.isclose(f["median_abs_rel"], 0.02) and np.isclose(f["p95_abs_rel"], 0.02)
    assert np.isclose(f["mean_rel"], 0.02) and np.isclose(f["median_oracle_rel_sigma"], 0.01)
    # |g - o| = 0.02 o against 3 x 0.0143 o: every voxel within three sigma
    assert f["frac_within_3sigma"] == 1.0
    assert np.isclose(f["z_mean"], 0.02 / np.sqrt(0.01 ** 2 + 0.0102 ** 2))
    assert map_figures(g, o, so, np.zeros(o.shape, bool), comb) == {"voxels": 0}
