"""Thin Python binding of libnmdose (include/nm_dose.h).

Argument marshalling only: every step of the simulation runs in the CUDA
library.  Functions keep the C names; arrays may be numpy arrays (host) or
torch tensors (host or CUDA), passed by pointer.  If the library has not been
built, the first call raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnmdose.so")
_lib = None

NM_OK, NM_ERR_ARG, NM_ERR_CUDA, NM_ERR_OOM, NM_ERR_OVERFLOW, NM_ERR_TIMEOUT, NM_ERR_STATE, NM_ERR_DEVICE = range(8)
NM_SOURCE_DECAY, NM_SOURCE_POINT = 0, 1
NM_MAX_MATERIALS = 8
NM_MAX_LABELS = 31
UNITS_PER_MEV = 64.0e6
STATUS_NAMES = ["NM_OK", "NM_ERR_ARG", "NM_ERR_CUDA", "NM_ERR_OOM", "NM_ERR_OVERFLOW",
                "NM_ERR_TIMEOUT", "NM_ERR_STATE", "NM_ERR_DEVICE"]


class NmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class nm_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
                ("dx", C.c_float), ("dy", C.c_float), ("dz", C.c_float),
                ("density", C.c_void_p), ("material", C.c_void_p)]


class nm_materials(C.Structure):
    _fields_ = [("n", C.c_int32), ("z_over_a", C.POINTER(C.c_double)), ("zeff", C.POINTER(C.c_double)),
                ("pe_coeff", C.c_double), ("pe_exp", C.c_double), ("rayleigh_coeff", C.c_double),
                ("rayleigh", C.c_int32), ("photon_cut_mev", C.c_double), ("electron_cut_mev", C.c_double)]


class nm_options(C.Structure):
    _fields_ = [("source_mode", C.c_int32), ("point", C.c_float * 3), ("photon_mev", C.c_double),
                ("positron_mev", C.c_double), ("batches", C.c_int32), ("activity_bq", C.c_double),
                ("n_labels", C.c_int32), ("block_threads", C.c_int32), ("chunk", C.c_int32),
                ("warp_aggregate", C.c_int32), ("regroup", C.c_int32), ("regroup_lanes", C.c_int32),
                ("max_steps", C.c_int32),
                ("stream", C.c_void_p), ("history_sigma", C.c_int32), ("beta_max_mev", C.c_double),
                ("beta_z", C.c_int32), ("kn_sampler", C.c_int32), ("no_annihilation", C.c_int32),
                ("beta_electron", C.c_int32), ("n_beta", C.c_int32),
                ("beta_endpoint_mev", C.POINTER(C.c_double)), ("beta_intensity", C.POINTER(C.c_double)),
                ("n_gamma", C.c_int32), ("gamma_mev", C.POINTER(C.c_double)),
                ("gamma_yield", C.POINTER(C.c_double))]


class nm_counters(C.Structure):
    _fields_ = [("histories", C.c_uint64), ("batches", C.c_uint64), ("emitted", C.c_int64),
                ("deposited", C.c_int64), ("escaped", C.c_int64), ("killed", C.c_int64),
                ("steps", C.c_uint64), ("compton", C.c_uint64), ("photo", C.c_uint64),
                ("rayleigh", C.c_uint64), ("cutoff", C.c_uint64), ("escapes", C.c_uint64),
                ("transport_ms", C.c_double), ("fold_ms", C.c_double), ("device_status", C.c_uint32),
                ("block_threads", C.c_int32), ("chunk", C.c_int32), ("warp_aggregate", C.c_int32),
                ("regroup", C.c_int32), ("regroup_lanes", C.c_int32), ("grid_blocks", C.c_int32), ("history_splits", C.c_uint64)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class nm_conv3d_desc(C.Structure):
    _fields_ = [(k, C.c_int32) for k in ("n", "d", "h", "w", "c0", "c1", "src0_coarse", "cout")]


class nm_denoise_options(C.Structure):
    _fields_ = [("patch", C.c_int32), ("batch", C.c_int32), ("levels", C.c_int32), ("base_width", C.c_int32),
                ("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("seed", C.c_uint64), ("stream", C.c_void_p), ("infer_voxels", C.c_int64)]


# Every entry point declared in include/nm_dose.h, with its ctypes signature.
_SIGS = {
    "nm_options_default": (None, [C.POINTER(nm_options)]),
    "nm_last_error": (C.c_char_p, []),
    "nm_ct_to_phantom": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "nm_dose_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(nm_grid), C.POINTER(nm_materials),
                                 C.c_void_p, C.c_void_p, C.POINTER(nm_options)]),
    "nm_dose_run": (C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64]),
    "nm_dose_run_batch": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(C.c_uint64), C.c_uint64]),
    "nm_dose_get": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "nm_dose_get_organs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "nm_dose_get_tally": (C.c_int, [C.c_void_p, C.c_void_p]),
    "nm_time_integrated_activity": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(C.c_double), C.c_int32, C.c_int64,
                                              C.c_double, C.c_void_p, C.POINTER(C.c_double), C.c_void_p]),
    "nm_dose_get_history_sigma": (C.c_int, [C.c_void_p, C.c_void_p]),
    "nm_dose_map_organs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "nm_dose_counters": (C.c_int, [C.c_void_p, C.POINTER(nm_counters)]),
    "nm_dose_reset": (C.c_int, [C.c_void_p]),
    "nm_dose_seek": (C.c_int, [C.c_void_p, C.c_uint64]),
    "nm_dose_checkpoint_size": (C.c_int, [C.c_void_p, C.POINTER(C.c_uint64)]),
    "nm_dose_checkpoint": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64]),
    "nm_dose_restore": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64]),
    "nm_dose_merge": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64]),
    "nm_dose_destroy": (None, [C.c_void_p]),
    "nm_check_philox": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "nm_check_kahn": (C.c_int, [C.c_double, C.c_int64, C.c_uint64, C.c_void_p]),
    "nm_check_beta": (C.c_int, [C.c_double, C.c_int32, C.c_int64, C.c_uint64, C.c_void_p]),
    "nm_debug_fail_alloc": (None, [C.c_int32]),
    "nm_release_cached_memory": (None, []),
    "nm_check_kn_table": (C.c_int, [C.c_double, C.c_double, C.c_double, C.c_int64, C.c_uint64, C.c_void_p]),
    "nm_check_wait_timeout": (C.c_int, [C.c_int64]),
    "nm_dose_alias_table": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.c_void_p, C.c_void_p, C.c_void_p]),
    "nm_check_source": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int64, C.c_uint64, C.c_void_p, C.c_void_p, C.c_void_p]),
    "nm_probe_l2_read": (C.c_int, [C.c_int64, C.c_int32, C.POINTER(C.c_double)]),
    "nm_probe_atomic_add_u64": (C.c_int, [C.c_int64, C.c_int64, C.POINTER(C.c_double)]),
    "nm_conv3d_kpad": (C.c_int32, [C.c_int32]),
    "nm_conv3d_fwd": (C.c_int, [C.POINTER(nm_conv3d_desc), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_void_p, C.c_int32, C.c_void_p]),
    "nm_conv3d_dgrad": (C.c_int, [C.POINTER(nm_conv3d_desc), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "nm_conv3d_wgrad": (C.c_int, [C.POINTER(nm_conv3d_desc), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p]),
    "nm_denoise_options_default": (None, [C.POINTER(nm_denoise_options)]),
    "nm_denoise_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(nm_denoise_options)]),
    "nm_denoise_destroy": (None, [C.c_void_p]),
    "nm_denoise_param_count": (C.c_int64, [C.c_void_p]),
    "nm_denoise_layer": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                   C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "nm_denoise_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "nm_denoise_adam_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int64)]),
    "nm_denoise_capture": (C.c_int, [C.c_void_p, C.c_int32]),
    "nm_denoise_captured": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_int64]),
    "nm_denoise_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_float,
                                        C.POINTER(C.c_float)]),
    "nm_denoise_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "nm_denoise_make_patches": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32,
                                          C.c_int32, C.c_float, C.c_float, C.c_void_p, C.c_int32, C.c_int32,
                                          C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "nm_denoise_scales": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_float),
                                    C.POINTER(C.c_float), C.c_void_p]),
    "nm_denoise_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32,
                                   C.c_int32, C.c_void_p]),
    "nm_denoise_apply_roi": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                                       C.c_int32, C.c_int32, C.c_void_p]),
    "nm_dose_tally_noalloc": (C.c_int, [C.POINTER(nm_grid), C.POINTER(nm_materials), C.c_void_p,
                                        C.POINTER(nm_options), C.c_uint64, C.c_uint64, C.c_void_p,
                                        C.POINTER(nm_counters)]),
}


def load():
    """Load libnmdose.so; raises if it was not built (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2111_11687_gb300.build.build()")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def symbols():
    return list(_SIGS)


def _check(st):
    if st != NM_OK:
        raise NmError(st, load().nm_last_error().decode())


def ptr(x):
    """Pointer of a numpy array or torch tensor (host or device), or None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array arguments must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor arguments must be contiguous")
        return x.data_ptr()
    raise TypeError(type(x))


def _dtype(x) -> str:
    """Element type name of a numpy array or torch tensor ('float32', 'int64', ...)."""
    return x.dtype.name if isinstance(x, np.ndarray) else str(x.dtype).replace("torch.", "")


def _cuda_device(x):
    """CUDA device index of a torch tensor, or None for host memory."""
    return x.device.index if getattr(x, "is_cuda", False) else None


def _want(name, x, dtype, numel, cuda=None):
    """Checks an array argument before its pointer crosses the C ABI, which
    cannot see the size or type of a device buffer: ``dtype`` and ``numel``
    must match, and with ``cuda`` = a device index the tensor must live on
    that CUDA device.  Raises ValueError; None passes (the C side decides
    whether it is allowed)."""
    if x is None:
        return
    if _dtype(x) != dtype:
        raise ValueError(f"{name}: expected {dtype}, got {_dtype(x)}")
    n = int(np.prod(x.shape))
    if n != numel:
        raise ValueError(f"{name}: expected {numel} elements, got {n}")
    if cuda is not None and _cuda_device(x) != cuda:
        raise ValueError(f"{name}: must be a CUDA tensor on device {cuda}")


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def options(**kw) -> nm_options:
    """nm_options from keyword arguments.  ``beta_branches`` [(endpoint MeV,
    intensity), ...] and ``gamma_lines`` [(MeV, yield per decay), ...] fill the
    radionuclide arrays (kept alive by the returned struct)."""
    o = nm_options()
    load().nm_options_default(C.byref(o))
    o._keep = []
    for k, v in kw.items():
        if k == "point":
            o.point[:] = [float(a) for a in v]
        elif k == "stream":
            o.stream = _stream_ptr(v)
        elif k == "beta_branches":
            e = np.ascontiguousarray([b[0] for b in v], np.float64)
            i = np.ascontiguousarray([b[1] for b in v], np.float64)
            o._keep += [e, i]
            o.n_beta = len(e)
            o.beta_endpoint_mev = e.ctypes.data_as(C.POINTER(C.c_double))
            o.beta_intensity = i.ctypes.data_as(C.POINTER(C.c_double))
        elif k == "gamma_lines":
            e = np.ascontiguousarray([g[0] for g in v], np.float64)
            y = np.ascontiguousarray([g[1] for g in v], np.float64)
            o._keep += [e, y]
            o.n_gamma = len(e)
            o.gamma_mev = e.ctypes.data_as(C.POINTER(C.c_double))
            o.gamma_yield = y.ctypes.data_as(C.POINTER(C.c_double))
        else:
            setattr(o, k, v)
    return o


@dataclass
class Materials:
    z_over_a: list
    zeff: list
    pe_coeff: float = 2.0e-9
    pe_exp: float = 3.8
    rayleigh_coeff: float = 1.0e-6
    rayleigh: int = 0
    photon_cut_mev: float = 0.010
    electron_cut_mev: float = 0.200

    def c(self):
        za = np.ascontiguousarray(self.z_over_a, np.float64)
        ze = np.ascontiguousarray(self.zeff, np.float64)
        m = nm_materials(len(za), za.ctypes.data_as(C.POINTER(C.c_double)), ze.ctypes.data_as(C.POINTER(C.c_double)),
                         self.pe_coeff, self.pe_exp, self.rayleigh_coeff, self.rayleigh,
                         self.photon_cut_mev, self.electron_cut_mev)
        m._keep = (za, ze)
        return m


def nm_ct_to_phantom(hu, density, material, stream=None):
    n = int(np.prod(hu.shape))
    _want("hu", hu, "int16", n)
    _want("density", density, "float32", n)
    _want("material", material, "uint8", n)
    _check(load().nm_ct_to_phantom(ptr(hu), n, ptr(density), ptr(material), _stream_ptr(stream)))


# Voxel and label counts of the handles nm_dose_create returned, so that the
# raw wrappers below can check the buffers they hand over: the C side cannot
# see the size of a device buffer.
_HANDLE_GRID = {}


def _handle_key(h):
    return h.value if isinstance(h, C.c_void_p) else int(h)


def _grid_of(h):
    """(voxels, labels) of a handle made here, or None for one made elsewhere."""
    return _HANDLE_GRID.get(_handle_key(h)) if h is not None else None


def nm_dose_create(density, material, spacing, materials: Materials, activity=None, labels=None,
                   opts: nm_options | None = None):
    """density/material/activity/labels are [nz, ny, nx] (x fastest); spacing (dx, dy, dz) cm."""
    nz, ny, nx = density.shape
    V = nx * ny * nz
    _want("density", density, "float32", V)
    _want("material", material, "uint8", V)
    _want("activity", activity, "float32", V)
    _want("labels", labels, "uint8", V)
    g = nm_grid(nx, ny, nz, float(spacing[0]), float(spacing[1]), float(spacing[2]), ptr(density), ptr(material))
    m = materials.c()
    h = C.c_void_p()
    _check(load().nm_dose_create(C.byref(h), C.byref(g), C.byref(m), ptr(activity), ptr(labels),
                                 C.byref(opts) if opts is not None else None))
    _HANDLE_GRID[h.value] = (V, int(opts.n_labels) if opts is not None else 0)
    return h


def nm_dose_run(h, n_decays: int, seed: int):
    _check(load().nm_dose_run(h, int(n_decays), int(seed)))


def nm_dose_run_batch(handles, n_decays, seed: int):
    """handles: list of handles (or Dose objects); n_decays: one count per handle."""
    hs = [h.h if isinstance(h, Dose) else h for h in handles]
    arr = (C.c_void_p * len(hs))(*[h.value if isinstance(h, C.c_void_p) else h for h in hs])
    nd = (C.c_uint64 * len(hs))(*[int(x) for x in n_decays])
    _check(load().nm_dose_run_batch(arr, len(hs), nd, int(seed)))


def nm_dose_get(h, dose=None, sigma=None, organ_dose=None):
    grid = _grid_of(h)
    if grid is not None:
        V, n_labels = grid
        _want("dose", dose, "float32", V)
        _want("sigma", sigma, "float32", V)
        _want("organ_dose", organ_dose, "float64", n_labels + 1)
    pointers = ptr(dose), ptr(sigma), ptr(organ_dose)
    _check(load().nm_dose_get(h, *pointers))


def nm_dose_get_organs(h, n_labels: int, eps: bool = True, sigma: bool = True):
    """(mean, eps_rms, sigma_mean, voxels) per label; eps=False skips Eq. 3 and
    with it the pass over the voxels (eps_rms is then None); sigma=False skips
    the batch sigma (None), which needs two batches."""
    n = n_labels + 1
    mean = np.zeros(n)
    sig = np.zeros(n) if sigma else None
    e = np.zeros(n) if eps else None
    cnt = np.zeros(n, np.int64)
    _check(load().nm_dose_get_organs(h, ptr(mean), ptr(e), ptr(sig), ptr(cnt)))
    return mean, e, sig, cnt


def nm_dose_get_tally(h, tally):
    grid = _grid_of(h)
    if grid is not None:
        _want("tally", tally, "int64", grid[0])
    p = ptr(tally)
    _check(load().nm_dose_get_tally(h, p))


def nm_time_integrated_activity(maps, t_h, half_life_h: float, out, stream=None) -> float:
    """Time-integrated activity (Bq s per voxel) of activity maps measured at
    times t_h (hours) into ``out``; returns the total over voxels."""
    V = int(np.prod(maps[0].shape))
    for k, m in enumerate(maps):
        _want(f"maps[{k}]", m, "float32", V)
    _want("out", out, "float32", V)
    arr = (C.c_void_p * len(maps))(*[ptr(m) for m in maps])
    t = (C.c_double * len(maps))(*[float(x) for x in t_h])
    total = C.c_double()
    _check(load().nm_time_integrated_activity(arr, t, len(maps), V, float(half_life_h), ptr(out), C.byref(total),
                                              _stream_ptr(stream)))
    return total.value


def nm_dose_counters(h) -> dict:
    c = nm_counters()
    _check(load().nm_dose_counters(h, C.byref(c)))
    return c.as_dict()


def nm_dose_reset(h):
    _check(load().nm_dose_reset(h))


def nm_dose_destroy(h):
    load().nm_dose_destroy(h)
    if h is not None:
        _HANDLE_GRID.pop(_handle_key(h), None)


def nm_release_cached_memory() -> None:
    """Return the device buffers the library keeps for reuse (from destroyed
    handles and per-call temporaries) to the device."""
    load().nm_release_cached_memory()


def nm_last_error() -> str:
    return load().nm_last_error().decode()


def nm_check_philox(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    ctr = np.ascontiguousarray(ctr, np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, np.uint32).reshape(-1, 2)
    out = np.empty_like(ctr)
    _check(load().nm_check_philox(ptr(ctr), ptr(key), len(ctr), ptr(out)))
    return out


def nm_check_kahn(e_mev: float, n: int, seed: int) -> np.ndarray:
    out = np.empty(n, np.float32)
    _check(load().nm_check_kahn(float(e_mev), n, seed, ptr(out)))
    return out


def nm_check_kn_table(e_mev: float, cut_mev: float, e0_mev: float, n: int, seed: int) -> np.ndarray:
    out = np.empty(n, np.float32)
    _check(load().nm_check_kn_table(float(e_mev), float(cut_mev), float(e0_mev), n, seed, ptr(out)))
    return out


def nm_check_beta(t_max_mev: float, z: int, n: int, seed: int) -> np.ndarray:
    out = np.empty(n, np.float32)
    _check(load().nm_check_beta(float(t_max_mev), int(z), n, seed, ptr(out)))
    return out


def nm_dose_alias_table(h):
    n = C.c_int64()
    _check(load().nm_dose_alias_table(h, C.byref(n), None, None, None))
    prob = np.empty(n.value, np.float32)
    vox = np.empty(n.value, np.int32)
    ali = np.empty(n.value, np.int32)
    _check(load().nm_dose_alias_table(h, C.byref(n), ptr(prob), ptr(vox), ptr(ali)))
    return prob, vox, ali


def nm_check_source(h, first: int, n: int, seed: int):
    vox = np.empty(n, np.int32)
    pos = np.empty((n, 3), np.float32)
    d = np.empty((n, 3), np.float32)
    _check(load().nm_check_source(h, first, n, seed, ptr(vox), ptr(pos), ptr(d)))
    return vox, pos, d


def nm_dose_tally_noalloc(density, material, spacing, materials: Materials, tally, n_decays: int, seed: int,
                          activity=None, opts: nm_options | None = None) -> dict:
    """Tally without device allocation; density, material, activity and tally must
    be CUDA tensors on one device (float32, uint8, float32, int64, all with the
    grid's voxel count): the C side writes 8 bytes per voxel into tally and
    cannot check its size.  Returns the counters."""
    nz, ny, nx = density.shape
    V = nx * ny * nz
    dev = _cuda_device(density)
    if dev is None:
        raise ValueError("density: must be a CUDA tensor")
    _want("density", density, "float32", V, dev)
    _want("material", material, "uint8", V, dev)
    _want("tally", tally, "int64", V, dev)
    if activity is not None or opts is None or opts.source_mode == NM_SOURCE_DECAY:
        if activity is None:
            raise ValueError("activity: decay mode needs an activity map")
        _want("activity", activity, "float32", V, dev)
    g = nm_grid(nx, ny, nz, float(spacing[0]), float(spacing[1]), float(spacing[2]), ptr(density), ptr(material))
    m = materials.c()
    c = nm_counters()
    _check(load().nm_dose_tally_noalloc(C.byref(g), C.byref(m), ptr(activity),
                                        C.byref(opts) if opts is not None else None,
                                        int(n_decays), int(seed), ptr(tally), C.byref(c)))
    return c.as_dict()


def nm_probe_l2_read(nbytes: int, reps: int) -> float:
    """L2 read bandwidth (GB/s) over an nbytes buffer read reps times."""
    out = C.c_double()
    _check(load().nm_probe_l2_read(int(nbytes), int(reps), C.byref(out)))
    return out.value


def nm_probe_atomic_add_u64(slots: int, ops: int) -> float:
    """Scattered 64-bit atomic adds per second into `slots` 8-byte words."""
    out = C.c_double()
    _check(load().nm_probe_atomic_add_u64(int(slots), int(ops), C.byref(out)))
    return out.value


def nm_conv3d_kpad(cin: int) -> int:
    return int(load().nm_conv3d_kpad(int(cin)))


def _desc(n, d, h, w, c0, c1=0, coarse=0, cout=16):
    return nm_conv3d_desc(n, d, h, w, c0, c1, coarse, cout)


def nm_conv3d_fwd(desc, x0, x1, w, bias, y, relu: bool, stream=None):
    _check(load().nm_conv3d_fwd(C.byref(desc), ptr(x0), ptr(x1), ptr(w), ptr(bias), ptr(y), int(relu),
                                _stream_ptr(stream)))


def nm_conv3d_dgrad(desc, dy, w, dx, stream=None):
    _check(load().nm_conv3d_dgrad(C.byref(desc), ptr(dy), ptr(w), ptr(dx), _stream_ptr(stream)))


def nm_conv3d_wgrad(desc, x0, x1, dy, dw, db=None, stream=None):
    _check(load().nm_conv3d_wgrad(C.byref(desc), ptr(x0), ptr(x1), ptr(dy), ptr(dw), ptr(db), _stream_ptr(stream)))


class Denoiser:
    """Owning wrapper of an nm_denoiser handle (all arrays are device tensors)."""

    def __init__(self, **kw):
        o = nm_denoise_options()
        load().nm_denoise_options_default(C.byref(o))
        for k, v in kw.items():
            setattr(o, k, _stream_ptr(v) if k == "stream" else v)
        self.opts = o
        self.h = C.c_void_p()
        _check(load().nm_denoise_create(C.byref(self.h), C.byref(o)))
        self.n_params = int(load().nm_denoise_param_count(self.h))

    def layers(self):
        out = []
        i = 0
        while True:
            ci, co, kp = C.c_int32(), C.c_int32(), C.c_int32()
            wo, bo = C.c_int64(), C.c_int64()
            if load().nm_denoise_layer(self.h, i, C.byref(ci), C.byref(co), C.byref(kp), C.byref(wo), C.byref(bo)) != NM_OK:
                break
            out.append(dict(cin=ci.value, cout=co.value, kpad=kp.value, w_off=wo.value, b_off=bo.value))
            i += 1
        return out

    def params(self, get=None, set=None, grads=None):
        _check(load().nm_denoise_params(self.h, ptr(get), ptr(set), ptr(grads)))

    def adam_state(self):
        """(first moments, second moments, updates made) of Adam, host copies."""
        m1 = np.empty(self.n_params, np.float32)
        m2 = np.empty(self.n_params, np.float32)
        t = C.c_int64()
        _check(load().nm_denoise_adam_state(self.h, ptr(m1), ptr(m2), C.byref(t)))
        return m1, m2, t.value

    def capture(self, on: bool = True):
        """Keep every layer's input, output activation and masked output
        gradient on later train steps (test support)."""
        _check(load().nm_denoise_capture(self.h, 1 if on else 0))

    def captured(self, layer: int, kind: int, shape):
        """Layer `layer`'s captured tensor (kind 0 input, 1 output activation,
        2 masked output gradient) as a host BF16 bit-pattern array of `shape`."""
        out = np.empty(shape, np.uint16)
        _check(load().nm_denoise_captured(self.h, int(layer), int(kind), ptr(out), out.nbytes))
        return out

    def train_step(self, x, target, weight=None, lr=None) -> float:
        loss = C.c_float()
        _check(load().nm_denoise_train_step(self.h, ptr(x), ptr(target), ptr(weight),
                                            float(self.opts.lr if lr is None else lr), C.byref(loss)))
        return loss.value

    def forward(self, x, y):
        _check(load().nm_denoise_forward(self.h, ptr(x), ptr(y)))

    def apply(self, dose, density, activity, out, roi=None):
        nz, ny, nx = dose.shape
        if roi is None:
            _check(load().nm_denoise_apply(self.h, ptr(dose), ptr(density), ptr(activity), nx, ny, nz, ptr(out)))
        else:
            _check(load().nm_denoise_apply_roi(self.h, ptr(dose), ptr(density), ptr(activity), ptr(roi), nx, ny, nz,
                                               ptr(out)))

    def close(self):
        if self.h:
            load().nm_denoise_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def nm_denoise_make_patches(dose, density, activity, dose_high, dose_scale, act_scale, corners, patch, x,
                            target=None, weight=None, stream=None):
    nz, ny, nx = dose.shape
    _check(load().nm_denoise_make_patches(ptr(dose), ptr(density), ptr(activity), ptr(dose_high), nx, ny, nz,
                                          float(dose_scale), float(act_scale), ptr(corners), int(corners.shape[0]),
                                          int(patch), ptr(x), ptr(target), ptr(weight), _stream_ptr(stream)))


def nm_denoise_scales(dose, activity, density, stream=None):
    ds, as_ = C.c_float(), C.c_float()
    _check(load().nm_denoise_scales(ptr(dose), ptr(activity), ptr(density), int(dose.numel()), C.byref(ds),
                                    C.byref(as_), _stream_ptr(stream)))
    return ds.value, as_.value


def _nbytes(buf) -> int:
    if isinstance(buf, np.ndarray):
        return int(buf.nbytes)
    return int(buf.numel() * buf.element_size())


class Dose:
    """Owning wrapper of an nm_dose handle."""

    def __init__(self, density, material, spacing, materials: Materials, activity=None, labels=None, **opts):
        self.shape = tuple(density.shape)
        self.n_labels = int(opts.get("n_labels", 0))
        self.h = nm_dose_create(density, material, spacing, materials, activity, labels, options(**opts))

    def run(self, n_decays: int, seed: int = 1):
        nm_dose_run(self.h, n_decays, seed)

    def get(self, dose=None, sigma=None):
        V = int(np.prod(self.shape))
        if dose is None:
            dose = np.empty(self.shape, np.float32)
        if sigma is None:
            sigma = np.empty(self.shape, np.float32)
        _want("dose", dose, "float32", V)
        _want("sigma", sigma, "float32", V)
        nm_dose_get(self.h, dose, sigma, None)
        return dose, sigma

    def organs(self, eps: bool = True, sigma: bool = True):
        return nm_dose_get_organs(self.h, self.n_labels, eps, sigma)

    def map_organs(self, dose):
        _want("dose", dose, "float32", int(np.prod(self.shape)))
        out = np.zeros(self.n_labels + 1)
        _check(load().nm_dose_map_organs(self.h, ptr(dose), ptr(out)))
        return out

    def tally(self):
        t = np.empty(self.shape, np.int64)
        nm_dose_get_tally(self.h, t)
        return t

    def counters(self):
        return nm_dose_counters(self.h)

    def history_sigma(self, out=None):
        """History-by-history sigma of the mean dose rate (Gy/s)."""
        if out is None:
            out = np.empty(self.shape, np.float32)
        _want("out", out, "float32", int(np.prod(self.shape)))
        _check(load().nm_dose_get_history_sigma(self.h, ptr(out)))
        return out

    def reset(self):
        nm_dose_reset(self.h)

    def seek(self, next_history_id: int):
        """Id of the next history (shards of one run take disjoint ranges)."""
        _check(load().nm_dose_seek(self.h, int(next_history_id)))

    def checkpoint_size(self) -> int:
        n = C.c_uint64()
        _check(load().nm_dose_checkpoint_size(self.h, C.byref(n)))
        return n.value

    def checkpoint(self, out=None):
        """The statistics as a byte image (numpy uint8 by default, or into
        ``out``: any host or device buffer of at least checkpoint_size() bytes)."""
        if out is None:
            out = np.empty(self.checkpoint_size(), np.uint8)
        _check(load().nm_dose_checkpoint(self.h, ptr(out), _nbytes(out)))
        return out

    def restore(self, image):
        _check(load().nm_dose_restore(self.h, ptr(image), _nbytes(image)))

    def merge(self, image):
        """Adds another shard's image (disjoint history ids) to these statistics."""
        _check(load().nm_dose_merge(self.h, ptr(image), _nbytes(image)))

    def close(self):
        if self.h:
            nm_dose_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
