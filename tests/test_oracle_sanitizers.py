"""The oracle under AddressSanitizer + UndefinedBehaviorSanitizer (fatal) and
under ThreadSanitizer (its worker threads share atomic tallies and
histories-by-chunk): every entry point the tests use, on small cases, in a
subprocess that preloads the sanitizer runtime.  CPU only."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "nm_oracle.cpp")

SCRIPT = r"""
import numpy as np, oracle
from paper_2111_11687_gb300 import inputs
oracle.build()
ph = inputs.adult_phantom(shape=(20, 16, 16), spacing=(3.0, 3.0, 4.5), seed=3)
den, mt = oracle.hu_to_phantom(ph.hu)
mat = oracle.Materials(z_over_a=inputs.MATERIAL_Z_OVER_A, zeff=inputs.MATERIAL_ZEFF)
r = oracle.run(den, mt, mat, activity=ph.activity, labels=ph.labels, n_labels=27, spacing=ph.spacing,
               n_hist=4000, seed=1, batches=4, threads=2, history_sigma=True, beta_max_mev=0.6335, beta_z=8)
assert r.counters["deposited"] + r.counters["escaped"] == r.counters["emitted"]
water = oracle.Materials(z_over_a=[0.5551], zeff=[7.42], rayleigh=1)
oracle.run(np.ones((6, 6, 6)), np.zeros((6, 6, 6), np.uint8), water, point=(1.5, 1.5, 1.5),
           spacing=(0.5,) * 3, n_hist=2000, seed=2, batches=2, threads=2)
oracle.trace((4, 5, 6), (0.3, 0.4, 0.5), np.array([0.1, 0.2, 0.3]), np.array([0.6, 0.0, 0.8]))
oracle.first_flight(np.full((4, 4, 4), 0.2), (0.5,) * 3, np.array([0.1, 1.0, 1.0]), np.array([1.0, 0.0, 0.0]),
                    1000, 6)
oracle.sample_kn_cos(0.2, 1000, 3)
oracle.sample_dirs(1000, 4)
oracle.sample_beta(0.6335, 8, 1000, 5)
print("sanitized run ok")
"""


def _runtime(name):
    path = subprocess.run(["gcc", f"-print-file-name={name}"], capture_output=True, text=True).stdout.strip()
    return path if os.path.isabs(path) and os.path.exists(path) else None


@pytest.mark.parametrize("kind", ["address,undefined", "thread"])
def test_oracle_is_clean_under_sanitizers(tmp_path, kind):
    rt = _runtime("libasan.so" if kind.startswith("address") else "libtsan.so")
    if rt is None:
        pytest.skip(f"no {kind} sanitizer runtime in this toolchain")
    lib = str(tmp_path / "liboracle_san.so")
    flags = ["-O1", "-g", "-std=c++17", "-fPIC", "-shared", f"-fsanitize={kind}", "-fno-omit-frame-pointer"]
    if "undefined" in kind:
        flags.append("-fno-sanitize-recover=undefined")
    subprocess.check_call(["g++", *flags, "-o", lib, SRC, "-lpthread"])
    env = dict(os.environ, PYTHONPATH=ROOT, NM_ORACLE_LIB=lib, LD_PRELOAD=rt,
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=0", TSAN_OPTIONS="halt_on_error=1 report_signal_unsafe=0")
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    assert "sanitized run ok" in r.stdout
    for marker in ("ERROR: AddressSanitizer", "runtime error:", "WARNING: ThreadSanitizer"):
        assert marker not in r.stderr, r.stderr[-3000:]
