"""FP64 CPU oracle for the ARCHER-NM Monte Carlo (paper §2.1, Eq. 1-4).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product (``paper_2111_11687_gb300``) never imports it and shares no
code with it.

The C++ part (``nm_oracle.cpp``) is compiled by :func:`build` into
``liboracle.so`` next to this file; this module is a ctypes wrapper around it
plus Eq. 4, which is a plain comparison formula.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nm_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (plain g++, -O2).  With
    NM_ORACLE_LIB set (the sanitizer test) that prebuilt library is used."""
    global _LIB_PATH
    if os.environ.get("NM_ORACLE_LIB"):
        _LIB_PATH = os.environ["NM_ORACLE_LIB"]
        return _LIB_PATH
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", tmp, _SRC, "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Materials(C.Structure):
    _fields_ = [
        ("n", C.c_int32),
        ("z_over_a", C.POINTER(C.c_double)),
        ("zeff", C.POINTER(C.c_double)),
        ("pe_coeff", C.c_double),
        ("pe_exp", C.c_double),
        ("rayleigh_coeff", C.c_double),
        ("rayleigh", C.c_int32),
        ("photon_cut_mev", C.c_double),
    ]


class _Problem(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
        ("density", C.POINTER(C.c_double)),
        ("material", C.POINTER(C.c_uint8)),
        ("activity", C.POINTER(C.c_double)),
        ("labels", C.POINTER(C.c_uint8)),
        ("n_labels", C.c_int32),
        ("mat", _Materials),
        ("point_mode", C.c_int32),
        ("point", C.c_double * 3),
        ("photon_mev", C.c_double),
        ("positron_mev", C.c_double),
        ("n_hist", C.c_uint64),
        ("first_history", C.c_uint64),
        ("seed", C.c_uint64),
        ("batches", C.c_int32),
        ("threads", C.c_int32),
        ("activity_bq", C.c_double),
        ("beta_max_mev", C.c_double),
        ("beta_z", C.c_int32),
        ("annihilation", C.c_int32),
        ("beta_sign", C.c_int32),
        ("n_beta", C.c_int32),
        ("beta_endpoint_mev", C.POINTER(C.c_double)),
        ("beta_intensity", C.POINTER(C.c_double)),
        ("n_gamma", C.c_int32),
        ("gamma_mev", C.POINTER(C.c_double)),
        ("gamma_yield", C.POINTER(C.c_double)),
    ]


class _Counters(C.Structure):
    _fields_ = [(n, C.c_int64) for n in (
        "emitted", "deposited", "escaped", "crossings", "flights",
        "compton", "photo", "rayleigh", "cutoff", "escapes")] + [("threads_used", C.c_int32)]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB_PATH)
        d, p = C.c_double, C.POINTER
        lib.orc_sigma_kn.restype = d
        lib.orc_sigma_kn.argtypes = [d]
        lib.orc_dsigma_kn.restype = d
        lib.orc_dsigma_kn.argtypes = [d, d]
        lib.orc_mu.restype = None
        lib.orc_mu.argtypes = [p(_Materials), C.c_int, d, d, p(d), p(d), p(d)]
        lib.orc_hu_to_phantom.restype = None
        lib.orc_hu_to_phantom.argtypes = [p(C.c_int16), C.c_int64, p(d), p(C.c_uint8)]
        lib.orc_trace.restype = C.c_int64
        lib.orc_trace.argtypes = [C.c_int32] * 3 + [d] * 3 + [p(d), p(d), C.c_int64, p(C.c_int64), p(d)]
        lib.orc_first_flight.restype = None
        lib.orc_first_flight.argtypes = [C.c_int32] * 3 + [d] * 3 + [p(d), p(d), p(d), C.c_int64, C.c_uint64, p(d)]
        lib.orc_sample_kn_cos.restype = None
        lib.orc_sample_kn_cos.argtypes = [d, C.c_int64, C.c_uint64, p(d)]
        lib.orc_sample_dirs.restype = None
        lib.orc_sample_dirs.argtypes = [C.c_int64, C.c_uint64, p(d)]
        lib.orc_rotate.restype = None
        lib.orc_rotate.argtypes = [p(d), d, d]
        lib.orc_sample_thomson_cos.restype = None
        lib.orc_sample_thomson_cos.argtypes = [C.c_int64, C.c_uint64, p(d)]
        lib.orc_interactions.restype = None
        lib.orc_interactions.argtypes = [p(_Materials), C.c_int32, d, d, C.c_int64, C.c_uint64, p(C.c_int32),
                                         p(d), p(d)]
        lib.orc_beta_density.restype = d
        lib.orc_beta_density.argtypes = [d, d, C.c_int32]
        lib.orc_beta_density_signed.restype = d
        lib.orc_beta_density_signed.argtypes = [d, d, C.c_int32, C.c_int32]
        lib.orc_sample_beta_branches.restype = None
        lib.orc_sample_beta_branches.argtypes = [p(d), p(d), C.c_int32, C.c_int32, C.c_int32, C.c_int64, C.c_uint64,
                                                 p(d)]
        lib.orc_sample_beta.restype = None
        lib.orc_sample_beta.argtypes = [d, C.c_int32, C.c_int64, C.c_uint64, p(d)]
        lib.orc_range_kp.restype = d
        lib.orc_range_kp.argtypes = [d]
        lib.orc_energy_at_range.restype = d
        lib.orc_energy_at_range.argtypes = [d]
        lib.orc_run.restype = C.c_int
        lib.orc_run.argtypes = [p(_Problem), p(C.c_int64), p(d), p(d), p(d), p(d), p(d), p(_Counters), p(d)]
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


# ---------------------------------------------------------------------------
# Materials (config values; the paper names its materials but prints no
# constants, §2.1).
# ---------------------------------------------------------------------------
@dataclass
class Materials:
    z_over_a: list
    zeff: list
    pe_coeff: float = 2.0e-9
    pe_exp: float = 3.8
    rayleigh_coeff: float = 1.0e-6
    rayleigh: int = 0
    photon_cut_mev: float = 0.010
    _keep: list = field(default_factory=list, repr=False)

    def c(self) -> _Materials:
        za = np.ascontiguousarray(self.z_over_a, dtype=np.float64)
        ze = np.ascontiguousarray(self.zeff, dtype=np.float64)
        self._keep = [za, ze]
        return _Materials(len(za), _dp(za), _dp(ze), self.pe_coeff, self.pe_exp,
                          self.rayleigh_coeff, self.rayleigh, self.photon_cut_mev)


def sigma_kn(e_mev: float) -> float:
    """Klein-Nishina total cross section per electron (cm^2)."""
    return _load().orc_sigma_kn(float(e_mev))


def dsigma_kn(e_mev: float, cos_theta: float) -> float:
    """Klein-Nishina dσ/dΩ per electron (cm^2/sr)."""
    return _load().orc_dsigma_kn(float(e_mev), float(cos_theta))


def mu(mat: Materials, m: int, rho: float, e_mev: float):
    """(mu_compton, mu_photo, mu_rayleigh) in 1/cm."""
    a, b, c = C.c_double(), C.c_double(), C.c_double()
    cm = mat.c()
    _load().orc_mu(C.byref(cm), m, rho, e_mev, C.byref(a), C.byref(b), C.byref(c))
    return a.value, b.value, c.value


def hu_to_phantom(hu: np.ndarray):
    """HU (int16) -> (density float64, material uint8), §2.1."""
    hu = np.ascontiguousarray(hu, dtype=np.int16)
    den = np.empty(hu.shape, np.float64)
    mat = np.empty(hu.shape, np.uint8)
    _load().orc_hu_to_phantom(hu.ctypes.data_as(C.POINTER(C.c_int16)), hu.size, _dp(den),
                              mat.ctypes.data_as(C.POINTER(C.c_uint8)))
    return den, mat


def trace(shape_zyx, spacing_xyz, p, d):
    """Voxel path lengths of a ray: returns (flat voxel ids, lengths)."""
    nz, ny, nx = shape_zyx
    p = np.ascontiguousarray(p, np.float64)
    d = np.ascontiguousarray(d, np.float64)
    cap = 4 * (nx + ny + nz) + 8
    vox = np.empty(cap, np.int64)
    ln = np.empty(cap, np.float64)
    n = _load().orc_trace(nx, ny, nz, *map(float, spacing_xyz), _dp(p), _dp(d), cap,
                          vox.ctypes.data_as(C.POINTER(C.c_int64)), _dp(ln))
    assert n <= cap
    return vox[:n], ln[:n]


def first_flight(mu_zyx: np.ndarray, spacing_xyz, p, d, n: int, seed: int):
    mu_zyx = np.ascontiguousarray(mu_zyx, np.float64)
    nz, ny, nx = mu_zyx.shape
    p = np.ascontiguousarray(p, np.float64)
    d = np.ascontiguousarray(d, np.float64)
    out = np.empty(n, np.float64)
    _load().orc_first_flight(nx, ny, nz, *map(float, spacing_xyz), _dp(mu_zyx), _dp(p), _dp(d), n, seed, _dp(out))
    return out


def sample_kn_cos(e_mev: float, n: int, seed: int) -> np.ndarray:
    out = np.empty(n, np.float64)
    _load().orc_sample_kn_cos(float(e_mev), n, seed, _dp(out))
    return out


def sample_dirs(n: int, seed: int) -> np.ndarray:
    out = np.empty((n, 3), np.float64)
    _load().orc_sample_dirs(n, seed, _dp(out))
    return out


def sample_thomson_cos(n: int, seed: int) -> np.ndarray:
    """Rayleigh scattering cosines (Thomson shape) as the transport draws them."""
    out = np.empty(n, np.float64)
    _load().orc_sample_thomson_cos(n, seed, _dp(out))
    return out


def interactions(mat: Materials, m: int, rho: float, e_mev: float, n: int, seed: int):
    """n real interactions at energy e_mev in material m (density rho) drawn by
    the function the full simulation uses: (type 0 Compton / 1 photoelectric /
    2 Rayleigh, photon energy after the event, scattering cosine)."""
    t = np.empty(n, np.int32)
    e2 = np.empty(n, np.float64)
    c = np.empty(n, np.float64)
    cm = mat.c()
    _load().orc_interactions(C.byref(cm), int(m), float(rho), float(e_mev), n, seed,
                             t.ctypes.data_as(C.POINTER(C.c_int32)), _dp(e2), _dp(c))
    return t, e2, c


def rotate(d, cos_theta: float, phi: float) -> np.ndarray:
    v = np.ascontiguousarray(d, np.float64).copy()
    _load().orc_rotate(_dp(v), float(cos_theta), float(phi))
    return v


@dataclass
class Result:
    tally: np.ndarray        # int64 [nz,ny,nx] energy units (2^-6 eV)
    dose_rate: np.ndarray    # Gy/s, Eq. 1
    sigma: np.ndarray        # Gy/s, batch sigma of the mean
    organ_mean: np.ndarray   # [n_labels+1] Gy/s, Eq. 2
    organ_eps: np.ndarray    # [n_labels+1] relative, Eq. 3
    organ_sigma: np.ndarray  # [n_labels+1] Gy/s, batch sigma of the organ mean
    counters: dict
    sigma_history: np.ndarray = None  # Gy/s, history-by-history sigma of the mean (if asked for)


def beta_density(t: float, t_max: float, z: int) -> float:
    """Unnormalised allowed beta+ spectrum N(T) with the Fermi function (daughter Z)."""
    return _load().orc_beta_density(float(t), float(t_max), int(z))


def beta_density_signed(t: float, t_max: float, z: int, sign: int) -> float:
    """Unnormalised allowed beta spectrum of a positron (sign +1) or an electron (-1)."""
    return _load().orc_beta_density_signed(float(t), float(t_max), int(z), int(sign))


def sample_beta_branches(endpoints, intensities, z: int, sign: int, n: int, seed: int) -> np.ndarray:
    """Kinetic energies (MeV) from a spectrum of several branches."""
    e = np.ascontiguousarray(endpoints, np.float64)
    i = np.ascontiguousarray(intensities, np.float64)
    out = np.empty(n)
    _load().orc_sample_beta_branches(_dp(e), _dp(i), len(e), int(z), int(sign), n, seed, _dp(out))
    return out


def sample_beta(t_max: float, z: int, n: int, seed: int) -> np.ndarray:
    """Positron kinetic energies (MeV) drawn from N(T) by rejection."""
    out = np.empty(n)
    _load().orc_sample_beta(float(t_max), int(z), n, seed, _dp(out))
    return out


def range_kp(t_mev: float) -> float:
    """Katz-Penfold range (g/cm^2) of an electron or positron of kinetic energy T."""
    return _load().orc_range_kp(float(t_mev))


def energy_at_range(r_gcm2: float) -> float:
    """Inverse of range_kp: the kinetic energy whose range is R."""
    return _load().orc_energy_at_range(float(r_gcm2))


def run(density, material, mat: Materials, *, activity=None, labels=None, n_labels: int = 0,
        spacing=(1.0, 1.0, 1.0), point=None, photon_mev: float = 0.511, positron_mev: float = 0.25,
        n_hist: int, seed: int = 1, batches: int = 10, threads: int = 0, first_history: int = 0,
        activity_bq: float = 1.0, history_sigma: bool = False, beta_max_mev: float = 0.0,
        beta_z: int = 8, annihilation: bool = True, beta_sign: int = 1, beta_branches=None,
        gamma_lines=None) -> Result:
    """Run the oracle MC.  Arrays are [nz, ny, nx] (x fastest); spacing (dx, dy, dz) in cm.

    ``point`` (cm, xyz) selects point-photon mode (one photon per history);
    otherwise decays are drawn from ``activity``.  ``beta_max_mev`` > 0 draws
    each positron's energy from the allowed beta+ spectrum with that endpoint
    (daughter atomic number ``beta_z``) and follows it along a straight track
    of Katz-Penfold range; else ``positron_mev`` is deposited at the decay.
    Other radionuclides: ``annihilation=False`` drops the two 0.511 MeV
    photons (a beta- emitter), ``beta_sign`` -1 makes the tracked particle an
    electron, ``beta_branches`` [(endpoint MeV, intensity), ...] replaces the
    single endpoint, ``gamma_lines`` [(MeV, yield per decay), ...] adds photons
    from the decay site (each line independently).  ``history_sigma`` also
    returns the history-by-history sigma of the mean dose rate (Walters et al.
    2002: the spread of each history's total deposit per voxel).
    """
    lib = _load()
    density = np.ascontiguousarray(density, np.float64)
    material = np.ascontiguousarray(material, np.uint8)
    nz, ny, nx = density.shape
    V = density.size
    act = None if activity is None else np.ascontiguousarray(activity, np.float64)
    lab = None if labels is None else np.ascontiguousarray(labels, np.uint8)
    pr = _Problem()
    pr.nx, pr.ny, pr.nz = nx, ny, nz
    pr.dx, pr.dy, pr.dz = map(float, spacing)
    pr.density = _dp(density)
    pr.material = material.ctypes.data_as(C.POINTER(C.c_uint8))
    pr.activity = _dp(act) if act is not None else None
    pr.labels = lab.ctypes.data_as(C.POINTER(C.c_uint8)) if lab is not None else None
    pr.n_labels = n_labels
    pr.mat = mat.c()
    pr.point_mode = 1 if point is not None else 0
    if point is not None:
        pr.point[:] = [float(x) for x in point]
    pr.photon_mev = photon_mev
    pr.positron_mev = positron_mev
    pr.n_hist = n_hist
    pr.first_history = first_history
    pr.seed = seed
    pr.batches = batches
    pr.threads = threads
    pr.activity_bq = activity_bq
    pr.beta_max_mev = beta_max_mev
    pr.beta_z = beta_z
    pr.annihilation = 1 if annihilation else 0
    pr.beta_sign = -1 if beta_sign < 0 else 1
    keep = []
    if beta_branches:
        be = np.ascontiguousarray([b[0] for b in beta_branches], np.float64)
        bi = np.ascontiguousarray([b[1] for b in beta_branches], np.float64)
        keep += [be, bi]
        pr.n_beta, pr.beta_endpoint_mev, pr.beta_intensity = len(be), _dp(be), _dp(bi)
    if gamma_lines:
        ge = np.ascontiguousarray([g[0] for g in gamma_lines], np.float64)
        gy = np.ascontiguousarray([g[1] for g in gamma_lines], np.float64)
        keep += [ge, gy]
        pr.n_gamma, pr.gamma_mev, pr.gamma_yield = len(ge), _dp(ge), _dp(gy)
    tally = np.empty(density.shape, np.int64)
    dr = np.empty(density.shape, np.float64)
    sg = np.empty(density.shape, np.float64)
    nl = n_labels + 1
    om, oe, os_ = (np.zeros(nl), np.zeros(nl), np.zeros(nl))
    cnt = _Counters()
    sh = np.empty(density.shape, np.float64) if history_sigma else None
    rc = lib.orc_run(C.byref(pr), tally.ctypes.data_as(C.POINTER(C.c_int64)), _dp(dr), _dp(sg),
                     _dp(om), _dp(oe), _dp(os_), C.byref(cnt), _dp(sh) if sh is not None else None)
    if rc != 0:
        raise ValueError(f"orc_run failed with code {rc}")
    counters = {n: getattr(cnt, n) for n, _ in _Counters._fields_}
    return Result(tally, dr, sg, om, oe, os_, counters, sh)


def rel_diff_percent(test, ref):
    """Eq. 4: relative percent difference of ``test`` against ``ref``."""
    test = np.asarray(test, np.float64)
    ref = np.asarray(ref, np.float64)
    return 100.0 * (test - ref) / ref


def time_integrated_activity(maps, t_h, half_life_h: float) -> np.ndarray:
    """Decays per voxel from injection on (Bq s), from activity maps (Bq per
    voxel) measured at increasing times t_h (hours): a linear rise from zero
    before the first time point, the trapezoid rule between time points, and
    physical decay alone after the last one (its integral A_n T_1/2 / ln 2).
    This is the multi-time-point reading of the paper's outlook (§4), written
    out in FP64."""
    t = [3600.0 * float(x) for x in t_h]
    a = [np.asarray(m, np.float64) for m in maps]
    out = 0.5 * a[0] * t[0]
    for k in range(1, len(a)):
        out = out + 0.5 * (a[k - 1] + a[k]) * (t[k] - t[k - 1])
    return out + a[-1] * (3600.0 * half_life_h / np.log(2.0))
