"""Seeded synthetic inputs: cardiac-shaped phantom pairs.

The paper evaluates on 220 private 3D cardiac MRI ED/ES pairs resampled to
128x128x96 with RV, LV and LVM labels (Sec. 4, "Dataset").  That data is not
available, so this module stands in for it with seeded phantoms of the same
shape, label structure and intensity range:

* left-ventricle blood pool: an ellipsoid, intensity 0.9, label 1;
* myocardium: an ellipsoidal shell around the pool, intensity 0.5, label 2;
* right ventricle: an offset ellipsoid outside the shell, intensity 0.9,
  label 3;
* background 0.1, a one-voxel linear partial-volume ramp on every edge;
* the fixed image adds N(0, 0.02^2) noise;
* the moving image is the fixed image warped by a seeded smooth
  diffeomorphism: eight Gaussian velocity bumps (max amplitude 3 voxels)
  integrated by scaling and squaring (six squarings).

This module is shared by the CUDA path's tests/bench and by the oracle's tests.
It holds none of the registration method's arithmetic: its resampler is a
private helper used only to build the moving image, and nothing here is
imported by the oracle or by the CUDA binding.

Arrays are C-contiguous ``[nz][ny][nx]`` (x fastest); vector fields are
``[3][nz][ny][nx]`` with component 0 along x.  Displacements are in voxels.
"""
from __future__ import annotations

import numpy as np

__all__ = ["phantom", "random_velocity", "scaling_and_squaring", "make_pair",
           "translated_blob_pair"]


def _grid(dims):
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64),
                          np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y, z


def _radial_signed_distance(x, y, z, centre, radii):
    """Signed distance (voxels) to an ellipsoid, measured along the ray from
    its centre: negative inside, positive outside."""
    dx, dy, dz = x - centre[0], y - centre[1], z - centre[2]
    q = np.sqrt((dx / radii[0]) ** 2 + (dy / radii[1]) ** 2 + (dz / radii[2]) ** 2)
    r = np.sqrt(dx * dx + dy * dy + dz * dz)
    q_safe = np.maximum(q, 1e-12)
    return (q - 1.0) * r / q_safe


def _ramp(d):
    """Occupancy with a one-voxel linear partial-volume ramp."""
    return np.clip(0.5 - d, 0.0, 1.0)


def phantom(dims, rng):
    """Noise-free cardiac-shaped phantom and its label map.

    Returns ``(image float64 [nz][ny][nx], labels uint8 [nz][ny][nx])``.
    """
    nx, ny, nz = dims
    x, y, z = _grid(dims)
    centre = np.array([nx / 2.0, ny / 2.0, nz / 2.0]) + rng.uniform(-2.0, 2.0, 3)
    r_lv = np.array([0.14 * nx, 0.14 * ny, 0.30 * nz]) * rng.uniform(0.85, 1.15, 3)
    thick = rng.uniform(5.0, 9.0) * nx / 128.0
    r_outer = r_lv + thick
    side = 1.0 if rng.uniform() < 0.5 else -1.0
    centre_rv = centre + np.array([side * 0.2 * nx, rng.uniform(-0.03, 0.03) * ny, 0.0])
    r_rv = 0.8 * r_lv * rng.uniform(0.9, 1.1, 3)

    occ_lv = _ramp(_radial_signed_distance(x, y, z, centre, r_lv))
    occ_outer = _ramp(_radial_signed_distance(x, y, z, centre, r_outer))
    occ_myo = np.clip(occ_outer - occ_lv, 0.0, 1.0)
    occ_rv = _ramp(_radial_signed_distance(x, y, z, centre_rv, r_rv)) * (1.0 - occ_outer)
    occ_bg = np.clip(1.0 - occ_outer - occ_rv, 0.0, 1.0)
    image = 0.1 * occ_bg + 0.9 * occ_lv + 0.5 * occ_myo + 0.9 * occ_rv

    stack = np.stack([occ_bg, occ_lv, occ_myo, occ_rv])
    labels = np.argmax(stack, axis=0).astype(np.uint8)
    return image, labels


def random_velocity(dims, rng, nbumps=8, max_amp=3.0):
    """Sum of Gaussian velocity bumps, rescaled so that max |v| <= max_amp.

    Centres are uniform in the central 60 % of the volume, widths
    sigma ~ U(0.08, 0.16) * min(dims), amplitudes a random direction times
    U(0.5, 1) * max_amp.
    """
    nx, ny, nz = dims
    x, y, z = _grid(dims)
    lo = np.array([0.2 * nx, 0.2 * ny, 0.2 * nz])
    hi = np.array([0.8 * nx, 0.8 * ny, 0.8 * nz])
    v = np.zeros((3, nz, ny, nx))
    for _ in range(nbumps):
        c = rng.uniform(lo, hi)
        sigma = rng.uniform(0.08, 0.16) * min(dims)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        a = d * rng.uniform(0.5, 1.0) * max_amp
        g = np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) / (2.0 * sigma ** 2))
        for i in range(3):
            v[i] += a[i] * g
    peak = np.sqrt((v ** 2).sum(axis=0)).max()
    if peak > max_amp:
        v *= max_amp / peak
    return v


def _resample(f, px, py, pz):
    """Private trilinear resampler (border clamp) used only to build inputs."""
    nz, ny, nx = f.shape
    px = np.clip(px, 0.0, nx - 1.0)
    py = np.clip(py, 0.0, ny - 1.0)
    pz = np.clip(pz, 0.0, nz - 1.0)
    x0 = np.minimum(np.floor(px).astype(np.int64), nx - 2)
    y0 = np.minimum(np.floor(py).astype(np.int64), ny - 2)
    z0 = np.minimum(np.floor(pz).astype(np.int64), nz - 2)
    tx, ty, tz = px - x0, py - y0, pz - z0
    out = np.zeros(px.shape)
    for dz in (0, 1):
        wz = tz if dz else 1.0 - tz
        for dy in (0, 1):
            wy = ty if dy else 1.0 - ty
            for dx in (0, 1):
                wx = tx if dx else 1.0 - tx
                out += wz * wy * wx * f[z0 + dz, y0 + dy, x0 + dx]
    return out


def scaling_and_squaring(v, squarings=6):
    """Displacement of exp(v): start from v / 2^squarings, then compose the
    map with itself ``squarings`` times."""
    nz, ny, nx = v.shape[1:]
    x, y, z = _grid((nx, ny, nz))
    d = v / float(2 ** squarings)
    for _ in range(squarings):
        px, py, pz = x + d[0], y + d[1], z + d[2]
        d = d + np.stack([_resample(d[i], px, py, pz) for i in range(3)])
    return d


def make_pair(dims, seed, noise=0.02):
    """One seeded phantom pair.

    Returns a dict with float32 ``fixed`` (I0, target) and ``moving`` (I1,
    source), uint8 ``labels_fixed``/``labels_moving`` and the float64 true
    displacement ``d_true`` with moving(x) = fixed(x + d_true(x)).
    """
    dims = tuple(int(d) for d in dims)
    rng = np.random.default_rng(seed)
    img, lab = phantom(dims, rng)
    fixed = img + rng.normal(0.0, noise, img.shape)
    v = random_velocity(dims, rng)
    d = scaling_and_squaring(v)
    x, y, z = _grid(dims)
    px, py, pz = x + d[0], y + d[1], z + d[2]
    moving = _resample(fixed, px, py, pz)
    nz, ny, nx = img.shape
    ix = np.clip(np.rint(px), 0, nx - 1).astype(np.int64)
    iy = np.clip(np.rint(py), 0, ny - 1).astype(np.int64)
    iz = np.clip(np.rint(pz), 0, nz - 1).astype(np.int64)
    lab_moving = lab[iz, iy, ix]
    return {
        "fixed": np.ascontiguousarray(fixed, dtype=np.float32),
        "moving": np.ascontiguousarray(moving, dtype=np.float32),
        "labels_fixed": lab,
        "labels_moving": np.ascontiguousarray(lab_moving, dtype=np.uint8),
        "d_true": d,
    }


def translated_blob_pair(dims, shift, sigma_frac=0.18):
    """A smooth Gaussian blob and its copy translated by ``shift`` voxels
    (x, y, z), both sampled analytically: moving(x) = fixed(x + shift)."""
    nx, ny, nz = dims
    x, y, z = _grid(dims)
    c = np.array([nx / 2.0, ny / 2.0, nz / 2.0])
    s = sigma_frac * min(dims)

    def blob(px, py, pz):
        return 0.1 + 0.8 * np.exp(-((px - c[0]) ** 2 + (py - c[1]) ** 2 + (pz - c[2]) ** 2)
                                  / (2.0 * s * s))

    fixed = blob(x, y, z)
    moving = blob(x + shift[0], y + shift[1], z + shift[2])
    return (np.ascontiguousarray(fixed, dtype=np.float32),
            np.ascontiguousarray(moving, dtype=np.float32))


def random_linearisation(dims, seed, grad_scale=0.3, resid_scale=0.2):
    """Seeded random data-term inputs (J, c) for solver-level tests:
    J float32 [3][nz][ny][nx], c float32 [nz][ny][nx]."""
    nx, ny, nz = dims
    rng = np.random.default_rng(seed)
    J = rng.normal(0.0, grad_scale, (3, nz, ny, nx)).astype(np.float32)
    c = rng.normal(0.0, resid_scale, (nz, ny, nx)).astype(np.float32)
    return J, c


def random_field(shape, seed, scale=1.0):
    """Seeded float32 normal field of the given shape."""
    rng = np.random.default_rng(seed)
    return (scale * rng.normal(size=shape)).astype(np.float32)


BATCH_XY = (96, 112, 128, 144, 160)
BATCH_Z = (64, 80, 96, 112)


def draw_batch_dims(npairs, seed):
    """Grid sizes of a batch of uneven pairs: nx, ny uniform from
    {96, 112, 128, 144, 160}, nz uniform from {64, 80, 96, 112} (multiples of
    16, so every prime factor is 2, 3, 5 or 7).  Returns a list of (nx, ny, nz)."""
    rng = np.random.default_rng(seed)
    return [(int(rng.choice(BATCH_XY)), int(rng.choice(BATCH_XY)), int(rng.choice(BATCH_Z)))
            for _ in range(npairs)]


def phase_pair(dims, seed, noise=0.02):
    """A cheap pair for large batches: two independent phantoms (different
    centre offsets, radii and myocardial thickness, as between two cardiac
    phases) with noise on the fixed one.  Returns float32 (fixed, moving)."""
    dims = tuple(int(d) for d in dims)
    rng = np.random.default_rng(seed)
    fixed, _ = phantom(dims, rng)
    fixed = fixed + rng.normal(0.0, noise, fixed.shape)
    moving, _ = phantom(dims, np.random.default_rng(seed + 1_000_003))
    return (np.ascontiguousarray(fixed, dtype=np.float32),
            np.ascontiguousarray(moving, dtype=np.float32))
