"""Seeded synthetic inputs: CT (HU), PET activity and organ labels.

This module holds none of the method's arithmetic: it only draws the raw
inputs a PET/CT study provides (§2.1, §2.2 of the paper -- CT numbers, a PET
activity map and 27 organ masks), plus the material constants the physics is
configured with.  The HU -> density/material conversion, the decay sampling and
everything after it live in the CUDA path and, independently, in the oracle.
Both sides draw their inputs from here and from nowhere else.

Geometry: arrays are indexed [z, y, x] with x fastest; spacing is (dx, dy, dz)
in cm; the grid origin is its corner.  Body coordinates are in cm, x across the
body, y front (-) to back (+), z from the feet up.

Every generator is a pure function of its arguments and its seed
(numpy PCG64), so the same call gives the same arrays on any machine.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# Organ labels 1..27, in the order of the paper's Table 1; 0 = no organ.
ORGANS = [
    "Bladder", "Bowel", "Brain", "Brain_Stem", "Esophagus", "Eye_Left", "Eye_Right",
    "Heart", "Kidney_Left", "Kidney_Right", "Larynx", "Liver", "Lung_Left", "Lung_Right",
    "Optic_Chiasm", "Optical_Nerve_Left", "Optical_Nerve_Right", "Pancreas",
    "Parotid_Left", "Parotid_Right", "Pelvis", "Pituitary", "Rectum", "Spinal_Cord",
    "Spleen", "Stomach", "Thyroid_Gland",
]
N_LABELS = len(ORGANS)
LABEL = {name: i + 1 for i, name in enumerate(ORGANS)}

# The five phantom materials (index = material id) with their configured
# electron fraction Z/A and photoelectric effective Z.  The paper names its
# materials without constants (§2.1); these are configuration values that both
# the oracle and the CUDA path read.
MATERIAL_NAMES = ["air", "lung", "adipose", "soft_tissue", "bone"]
MATERIAL_Z_OVER_A = [0.4992, 0.5497, 0.5558, 0.5500, 0.5300]
MATERIAL_ZEFF = [7.6, 7.5, 6.4, 7.4, 13.0]
# Water for the point-source cube.
WATER_Z_OVER_A = [0.5551]
WATER_ZEFF = [7.42]
# mu_pe/rho = PE_COEFF * Zeff^PE_EXP / E^3 (cm^2/g, E in MeV): water at 30 keV
# gets about 0.15 cm^2/g.
PE_COEFF = 2.0e-9
PE_EXP = 3.8
# mu_R/rho = RAYLEIGH_COEFF * Zeff^2 / E^2 (optional, off by default).
RAYLEIGH_COEFF = 1.0e-6
PHOTON_CUT_MEV = 0.010
ELECTRON_CUT_MEV = 0.200
PHOTON_MEV = 0.511
POSITRON_MEV = 0.25
# A(t_s): 8.0 mCi decayed for 60 min with T1/2 = 109.77 min (§2.2).
ACTIVITY_BQ = 8.0e-3 * 3.7e10 * 2.0 ** (-60.0 / 109.77)

# Uptake ratios (organ activity concentration relative to the rest of the body).
UPTAKE = {"Brain": 8.0, "Bladder": 20.0, "Heart": 5.0, "Liver": 3.0}


@dataclass
class WaterCube:
    density: np.ndarray     # float32 [n,n,n] g/cm^3
    material: np.ndarray    # uint8   [n,n,n]
    spacing: tuple          # cm
    point: tuple            # cm, source position


def water_cube(n: int = 64, voxel_cm: float = 0.5) -> WaterCube:
    """Uniform water (1.0 g/cm^3) cube with a point source at its centre."""
    den = np.ones((n, n, n), np.float32)
    mat = np.zeros((n, n, n), np.uint8)
    c = n * voxel_cm / 2.0
    return WaterCube(den, mat, (voxel_cm,) * 3, (c, c, c))


def paper_point_source(n: int = 101, voxel_cm: float = 0.05) -> "Phantom":
    """The paper's point-source check (§2.2): CT of n^3 voxels all at 0 HU
    (water), PET zero except the central voxel (default 101^3 voxels of
    0.5 mm); every decay starts in that voxel."""
    hu = np.zeros((n, n, n), np.int16)
    act = np.zeros((n, n, n), np.float32)
    act[n // 2, n // 2, n // 2] = 1.0
    lab = np.zeros((n, n, n), np.uint8)
    return Phantom(hu, act, lab, (voxel_cm,) * 3)


@dataclass
class Phantom:
    hu: np.ndarray          # int16 [nz,ny,nx]
    activity: np.ndarray    # float32 [nz,ny,nx], PET concentration (arbitrary Bq/mL scale)
    labels: np.ndarray      # uint8 [nz,ny,nx], 0..27
    spacing: tuple          # (dx, dy, dz) cm

    @property
    def shape(self):
        return self.hu.shape


class _Raster:
    """Voxel-centre coordinates of a grid placed in body coordinates."""

    def __init__(self, shape, spacing, origin, scale):
        self.nz, self.ny, self.nx = shape
        self.dx, self.dy, self.dz = spacing
        self.ox, self.oy, self.oz = origin     # body coords of the grid corner
        self.s = scale                        # body-cm per phantom-cm

    def _axis(self, n, d, o, lo, hi):
        # index range whose voxel centres may fall in [lo, hi] (body cm)
        i0 = int(np.floor((lo - o) / d - 0.5))
        i1 = int(np.ceil((hi - o) / d + 0.5))
        i0, i1 = max(i0, 0), min(i1, n)
        return i0, i1

    def box(self, c, r):
        """Slices and centre coordinates (relative to c, in units of r) of the
        bounding box of an axis-aligned ellipsoid with centre c and radii r."""
        s = self.s
        c = [ci * s for ci in c]
        r = [ri * s for ri in r]
        x0, x1 = self._axis(self.nx, self.dx, self.ox, c[0] - r[0], c[0] + r[0])
        y0, y1 = self._axis(self.ny, self.dy, self.oy, c[1] - r[1], c[1] + r[1])
        z0, z1 = self._axis(self.nz, self.dz, self.oz, c[2] - r[2], c[2] + r[2])
        if x0 >= x1 or y0 >= y1 or z0 >= z1:
            return None
        X = (self.ox + (np.arange(x0, x1) + 0.5) * self.dx - c[0]) / r[0]
        Y = (self.oy + (np.arange(y0, y1) + 0.5) * self.dy - c[1]) / r[1]
        Z = (self.oz + (np.arange(z0, z1) + 0.5) * self.dz - c[2]) / r[2]
        return (slice(z0, z1), slice(y0, y1), slice(x0, x1)), X[None, None, :], Y[None, :, None], Z[:, None, None]

    def ellipsoid(self, c, r):
        b = self.box(c, r)
        if b is None:
            return None, None
        sl, X, Y, Z = b
        return sl, (X * X + Y * Y + Z * Z) <= 1.0

    def shell(self, c, r_out, r_in):
        """Voxels inside the ellipsoid (c, r_out) but outside (c, r_in)."""
        b = self.box(c, r_out)
        if b is None:
            return None, None
        sl, X, Y, Z = b
        outer = (X * X + Y * Y + Z * Z) <= 1.0
        Xi, Yi, Zi = X * (r_out[0] / r_in[0]), Y * (r_out[1] / r_in[1]), Z * (r_out[2] / r_in[2])
        inner = (Xi * Xi + Yi * Yi + Zi * Zi) <= 1.0
        return sl, outer & ~inner

    def cylinder_z(self, cx, cy, rx, ry, z0, z1):
        zc, hz = (z0 + z1) / 2.0, (z1 - z0) / 2.0
        b = self.box((cx, cy, zc), (rx, ry, hz))
        if b is None:
            return None, None
        sl, X, Y, Z = b
        return sl, ((X * X + Y * Y) <= 1.0) & (np.abs(Z) <= 1.0)


# Whole-body geometry in body cm (z from the feet).  Each entry: label name or
# None, HU, shape.  Later entries overwrite earlier ones.
_ZH = 88.0  # body z of the pelvis-to-head field of view's lower edge


def _organ_table():
    z = _ZH
    E = "ell"
    return [
        # name, HU, kind, params
        ("Lung_Left", -780, E, ((7.5, 1.0, z + 50), (5.5, 7.5, 11.0))),
        ("Lung_Right", -780, E, ((-7.5, 1.0, z + 50), (5.5, 7.5, 11.0))),
        ("Heart", 45, E, ((1.5, -2.5, z + 46), (4.5, 4.0, 5.0))),
        ("Liver", 55, E, ((-7.0, 0.0, z + 36), (7.5, 6.5, 5.5))),
        ("Spleen", 50, E, ((10.0, 3.0, z + 37), (3.0, 2.5, 4.5))),
        ("Stomach", 30, E, ((5.0, -3.0, z + 36), (4.0, 3.0, 4.0))),
        ("Pancreas", 40, E, ((1.0, 1.0, z + 32), (5.0, 1.5, 1.5))),
        ("Kidney_Left", 35, E, ((6.5, 5.0, z + 30), (2.5, 2.2, 5.0))),
        ("Kidney_Right", 35, E, ((-6.5, 5.0, z + 30), (2.5, 2.2, 5.0))),
        ("Bowel", 20, E, ((0.0, -2.0, z + 22), (9.0, 5.5, 6.0))),
        ("Rectum", 25, E, ((0.0, 3.5, z + 12), (1.5, 1.5, 3.0))),
        ("Bladder", 10, E, ((0.0, -4.0, z + 12), (4.0, 3.5, 3.5))),
        ("Esophagus", 35, "cyl", (0.0, 4.5, 0.8, 0.8, z + 40, z + 64)),
        ("Thyroid_Gland", 60, E, ((0.0, -2.5, z + 62), (2.2, 1.0, 1.8))),
        ("Larynx", 30, E, ((0.0, -3.0, z + 65.5), (1.5, 1.5, 2.0))),
        ("Brain", 35, E, ((0.0, 0.3, z + 79.5), (7.2, 8.6, 7.5))),
        ("Brain_Stem", 35, E, ((0.0, 2.5, z + 72.5), (1.3, 1.3, 3.0))),
        ("Parotid_Left", 25, E, ((6.3, 0.5, z + 71), (1.6, 2.2, 2.6))),
        ("Parotid_Right", 25, E, ((-6.3, 0.5, z + 71), (1.6, 2.2, 2.6))),
        ("Eye_Left", 20, E, ((3.2, -8.3, z + 78), (1.2, 1.2, 1.2))),
        ("Eye_Right", 20, E, ((-3.2, -8.3, z + 78), (1.2, 1.2, 1.2))),
        ("Optical_Nerve_Left", 35, E, ((1.9, -5.6, z + 78), (0.45, 1.8, 0.45))),
        ("Optical_Nerve_Right", 35, E, ((-1.9, -5.6, z + 78), (0.45, 1.8, 0.45))),
        ("Optic_Chiasm", 35, E, ((0.0, -3.6, z + 78), (1.0, 0.6, 0.45))),
        ("Pituitary", 35, E, ((0.0, -2.5, z + 76.5), (0.6, 0.6, 0.5))),
        ("Spinal_Cord", 30, "cyl", (0.0, 7.2, 0.6, 0.6, z + 8, z + 66)),
    ]


def _draw(shape, spacing, z_bottom, rng, uptake_jitter=0.0, lesions=0, body_scale=1.0):
    nz, ny, nx = shape
    dx, dy, dz = spacing
    s = body_scale
    # Grid centred across the body; z_bottom = body z of the grid's lower edge.
    origin = (-nx * dx / 2.0, -ny * dy / 2.0, z_bottom * s)
    R = _Raster(shape, spacing, origin, s)
    hu = np.full(shape, -1000, np.int16)
    lab = np.zeros(shape, np.uint8)
    body = np.zeros(shape, bool)

    def put(sl_mask, value, label=None, where=None):
        sl, m = sl_mask
        if sl is None:
            return
        if where is not None:
            m = m & where[sl]
        hu[sl][m] = value
        if label is not None:
            lab[sl][m] = label

    def mark_body(sl_mask):
        sl, m = sl_mask
        if sl is not None:
            body[sl] |= m

    z = _ZH
    # Body envelope: torso, neck, head, thighs -- adipose shell, soft tissue core.
    parts = [((0.0, 0.0, z + 38), (17.0, 11.5, 32.0)),
             ((0.0, 1.0, z + 67), (6.0, 6.0, 6.0)),
             ((0.0, 0.0, z + 78.5), (8.5, 10.0, 10.5)),
             ((8.0, 0.0, 50.0), (7.0, 7.5, 50.0)),
             ((-8.0, 0.0, 50.0), (7.0, 7.5, 50.0))]
    for c, r in parts:
        e = R.ellipsoid(c, r)
        put(e, -100)
        mark_body(e)
    for c, r in parts:
        put(R.ellipsoid(c, tuple(x - 1.5 for x in r)), 40)
    # Skull: bone shell of the head, 0.7 cm.
    hc, hr = parts[2]
    put(R.shell(hc, hr, tuple(x - 0.7 for x in hr)), 1000)
    # Ribs: bands of a thin shell inside the torso wall.
    tc, tr = parts[0]
    sl, m = R.shell(tc, tuple(x - 1.5 for x in tr), tuple(x - 2.3 for x in tr))
    if sl is not None:
        zb = (origin[2] + (np.arange(sl[0].start, sl[0].stop) + 0.5) * dz) / s - z
        band = ((zb - 36.0) % 2.4 < 0.9) & (zb >= 36.0) & (zb <= 60.0)
        put((sl, m & band[:, None, None]), 800)
    # Spine and femurs.
    put(R.cylinder_z(0.0, 6.5, 1.8, 1.6, z + 8, z + 66), 700)
    put(R.cylinder_z(8.0, 0.5, 1.3, 1.3, 10.0, z + 4), 700)
    put(R.cylinder_z(-8.0, 0.5, 1.3, 1.3, 10.0, z + 4), 700)
    # Pelvic bone: shell around the bladder/rectum region.
    put(R.shell((0.0, 1.5, z + 13), (14.0, 8.0, 6.5), (12.5, 6.5, 5.5)), 700, LABEL["Pelvis"], where=body)
    # Organs.
    for name, h, kind, prm in _organ_table():
        e = R.ellipsoid(*prm) if kind == "ell" else R.cylinder_z(*prm)
        put(e, h, LABEL[name], where=body)
    # Lesions: spheres of 1-3 cm diameter with uptake 10-15, inside the torso.
    lesion_mask = np.zeros(shape, bool)
    lesion_uptake = []
    for _ in range(lesions):
        c = (rng.uniform(-10, 10), rng.uniform(-6, 6), z + rng.uniform(15, 58))
        rad = rng.uniform(0.5, 1.5)
        sl, m = R.ellipsoid(c, (rad, rad, rad))
        if sl is not None:
            lm = np.zeros(shape, bool)
            lm[sl] = m
            lesion_uptake.append((lm & body, rng.uniform(10.0, 15.0)))
            lesion_mask |= lm & body
    # CT noise inside the body.
    noise = rng.normal(0.0, 15.0, size=shape).astype(np.float32)
    hu_f = hu.astype(np.float32) + np.where(body, noise, 0.0)
    hu = np.clip(np.rint(hu_f), -1024, 3071).astype(np.int16)
    # PET: uptake ratio times lognormal(0, 0.3) voxel noise; air 0.
    up = np.where(body, 1.0, 0.0).astype(np.float32)
    for name, ratio in UPTAKE.items():
        jit = 1.0 + uptake_jitter * rng.uniform(-1.0, 1.0) if uptake_jitter else 1.0
        up[lab == LABEL[name]] = ratio * jit
    for m, ratio in lesion_uptake:
        up[m] = ratio
    act = up * rng.lognormal(0.0, 0.3, size=shape).astype(np.float32) * 5000.0
    act[~body] = 0.0
    return Phantom(hu, act.astype(np.float32), lab, tuple(spacing))


def adult_phantom(shape=(300, 256, 256), spacing=(0.2, 0.2, 0.3), seed: int = 1) -> Phantom:
    """Pelvis-to-head adult PET/CT phantom (default 256x256x300 voxels of
    2x2x3 mm).  Coarser grids of the same field of view give the same body."""
    rng = np.random.default_rng(seed)
    fov_z = shape[0] * spacing[2]
    scale = min(shape[2] * spacing[0] / 51.2, shape[1] * spacing[1] / 51.2, fov_z / 90.0)
    return _draw(shape, spacing, _ZH, rng, body_scale=scale)


def batch_phantoms(count: int = 16, seed0: int = 1):
    """Uneven-grid patients: grids between 128x128x160 and 256x256x320, voxel
    sizes 2-4 mm, organ uptake ratios jittered by +-30%, bodies scaled to fit."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(1000 + seed0 + i)
        nxy = int(rng.integers(128, 257))
        nz = int(rng.integers(160, 321))
        d = float(rng.uniform(0.2, 0.4))
        dz = float(rng.uniform(0.2, 0.4))
        shape = (nz, nxy, nxy)
        spacing = (d, d, dz)
        scale = min(nxy * d / 51.2, nz * dz / 90.0)
        out.append(_draw(shape, spacing, _ZH, rng, uptake_jitter=0.3, body_scale=scale))
    return out


def whole_body_phantom(shape=(600, 512, 512), spacing=(0.1, 0.1, 0.3), seed: int = 1,
                       lesions: int = 6) -> Phantom:
    """Feet-to-head phantom (default 512x512x600 voxels of 1x1x3 mm) with
    1-3 cm high-uptake lesions."""
    rng = np.random.default_rng(seed)
    scale = min(shape[2] * spacing[0] / 51.2, shape[0] * spacing[2] / 180.0)
    return _draw(shape, spacing, 0.0, rng, lesions=lesions, body_scale=scale)
