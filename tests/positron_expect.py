"""Brute-force expectation of positron tracks in a homogeneous cube (shared by
the oracle pins and the GPU tests; plain numpy, no code of either side)."""
import numpy as np


def cube_positron_expectation(rho, n_side, vox, t, rng):
    """Per decay, brute force: straight tracks from a uniform point of the
    central voxel in isotropic directions; the energy left when a track
    reaches the cube's surface escapes, the energy lost before it leaves the
    central voxel stays there."""
    L = n_side * vox
    c0 = (n_side // 2) * vox
    n = t.size
    x = c0 + vox * rng.random((n, 3))
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)

    def exit_dist(lo, hi):
        with np.errstate(divide="ignore"):
            d = np.where(u > 0, (hi - x) / u, np.where(u < 0, (lo - x) / u, np.inf))
        return d.min(axis=1)

    def kp(tt):
        lt = np.log(tt)
        return 0.412 * np.exp((1.265 - 0.0954 * lt) * lt)

    def kp_inv(r):
        c = np.log(r / 0.412)
        return np.exp((1.265 - np.sqrt(1.265 ** 2 - 4 * 0.0954 * c)) / (2 * 0.0954))

    r = kp(t)

    def residual(d):
        left = r - rho * d
        out = np.zeros_like(t)
        m = left > 0
        out[m] = kp_inv(left[m])
        return out

    esc = residual(exit_dist(0.0, L))
    centre = t - residual(exit_dist(c0, c0 + vox))
    return esc, centre
