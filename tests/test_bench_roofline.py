"""The transport roofline that bench.py reports, on made-up counters (CPU):
algorithmic bytes per decay (5 B per voxel read, 8 B per tally atomic, 12 B per
alias entry), the fraction of the peak, and the further ceilings (L2 sectors,
atomics, instruction issue)."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_transport_roofline_arithmetic(monkeypatch):
    import bench
    monkeypatch.setattr(bench, "_peaks", lambda: {"hbm_gbs": 6000.0})
    monkeypatch.setattr(bench, "_profile_figures", lambda: {"dram_bytes_per_decay": 40.0, "lts_sectors_per_decay": 25.0,
                                                            "warp_inst_per_decay": 250.0, "lane_efficiency_pct": 50.0})
    per = {"flight_steps": 14.0, "interactions": 3.5, "positron_deposits": 1.0, "escapes": 2.0}
    r = bench.transport_roofline(per, 1e8, 25.0, {"sm_mhz": 2000.0}, {"l2_read_gbs": 20000.0,
                                                                        "atomic_add_u64_per_s": 2e11})
    bpd = 5 * 14.0 + 8 * 4.5 + 12
    assert r["bytes_per_decay"] == pytest.approx(bpd)
    rate = 1e8 / 25e-3
    assert r["achieved"] == pytest.approx(bpd * rate / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6000.0) and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["traffic"] == pytest.approx(40.0 * 1e8)
    c = r["ceilings"]
    assert c["l2_sectors"]["achieved"] == pytest.approx(25 * 32 * rate / 1e9)
    assert c["atomics"]["frac"] == pytest.approx(4.5 * rate / 2e11)
    assert c["issue"]["peak"] == pytest.approx(152 * 4 * 2e9 / 250.0)
    assert c["issue"]["frac"] == pytest.approx(rate / (152 * 4 * 2e9 / 250.0))
    json.dumps(r)                                   # the line stays JSON


def test_roofline_without_profile_leaves_traffic_null(monkeypatch):
    import bench
    monkeypatch.setattr(bench, "_peaks", lambda: None)
    monkeypatch.setattr(bench, "_profile_figures", lambda: None)
    per = {"flight_steps": 10.0, "interactions": 3.0, "positron_deposits": 1.0, "escapes": 2.0}
    r = bench.transport_roofline(per, 1e8, 20.0, None, None)
    assert r["traffic"] is None and r["traffic_source"] is None and r["peak_source"] == "fallback"
    assert "issue" not in r["ceilings"]


def test_committed_transport_profile_describes_the_current_kernel():
    """The ncu figures bench.py quotes (traffic, L2 sectors, instructions per
    decay) are read from the committed transport summary only while it was
    captured on the current kernel source; a kernel change must come with a
    new capture, else the benchmark line loses those figures."""
    import bench
    prof = bench._profile_figures()
    assert prof is not None, "profiles/transport_kernel_adult_phantom.md was captured on another kernel source"
    for k in ("dram_bytes_per_decay", "lts_sectors_per_decay", "warp_inst_per_decay", "lane_efficiency_pct"):
        assert prof[k] > 0, k
