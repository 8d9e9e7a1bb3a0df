"""Measured agreement of the GPU path with the FP64 oracle, written down.

The parity tests assert their criteria whether or not anything is recorded.
When the environment variable NM_PARITY_REPORT names a file, record() also
appends one JSON line per call to it: the pytest id of the running test and
the figures passed (the error of a result against the oracle, the margin a
criterion passed with).  Unset, record() does nothing.  No figure recorded
here feeds back into any test or expected value."""
import json
import os

import numpy as np


def _plain(v):
    if isinstance(v, (np.floating, float)):
        return float(v)
    if isinstance(v, (np.integer, int, bool, np.bool_)):
        return v.item() if hasattr(v, "item") else v
    if isinstance(v, np.ndarray):
        return [_plain(x) for x in v.tolist()]
    if isinstance(v, (list, tuple)):
        return [_plain(x) for x in v]
    if isinstance(v, dict):
        return {str(k): _plain(x) for k, x in v.items()}
    return v


def record(kind, **figures):
    path = os.environ.get("NM_PARITY_REPORT")
    if not path:
        return
    test = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" (")[0]
    line = {"test": test, "kind": kind}
    line.update({k: _plain(v) for k, v in figures.items()})
    try:
        with open(path, "a") as f:
            f.write(json.dumps(line) + "\n")
    except OSError:
        pass


def map_figures(g, o, so, sel, comb):
    """Voxel-map agreement over the selected voxels: the fraction within three
    combined sigma, the relative difference gpu/oracle - 1 (median of its
    magnitude, 95th percentile, mean), and the oracle's own relative sigma
    there, which sets the scale those differences are expected at."""
    g = np.asarray(g, np.float64)[sel]
    o = np.asarray(o, np.float64)[sel]
    so = np.asarray(so, np.float64)[sel]
    c = np.asarray(comb, np.float64)[sel]
    if g.size == 0:
        return {"voxels": 0}
    rel = g / o - 1
    return {"voxels": int(g.size),
            "frac_within_3sigma": float((np.abs(g - o) <= 3 * c).mean()),
            "median_abs_rel": float(np.median(np.abs(rel))),
            "p95_abs_rel": float(np.percentile(np.abs(rel), 95)),
            "mean_rel": float(rel.mean()),
            "median_oracle_rel_sigma": float(np.median(so / o)),
            "z_mean": float(((g - o) / c).mean()),
            "z_std": float(((g - o) / c).std())}
