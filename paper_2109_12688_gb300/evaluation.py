"""Registration quality measures of Sec. 4 ("Quantitative results").

Host-side scoring of a computed displacement u (device tensor or array
[3][nz][ny][nx], voxels): the source labels carried to the target grid by
nearest-neighbour sampling at x + u(x), their Dice overlap with the target
labels per class, the Hausdorff distance averaged over the 2D z-slices (mm,
1.2 mm isotropic voxels as in the paper's data) and the share of voxels
whose Jacobian determinant det(I + Du) is <= 0 (counted on the GPU by
nadmm_jacobian_det).

Readings: sample positions are rounded half up and clamped to the grid; a
slice contributes to the Hausdorff mean only where both label maps contain
the class in that slice.
"""
from __future__ import annotations

import numpy as np

CLASSES = {1: "LV", 2: "LVM", 3: "RV"}


def carry_labels(labels, u):
    """labels sampled at the nearest voxel of x + u(x) (clamped)."""
    labels = np.asarray(labels)
    u = np.asarray(u)
    nz, ny, nx = labels.shape
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    sx = np.clip(np.floor(ix + u[0].astype(np.float64) + 0.5), 0, nx - 1).astype(np.intp)
    sy = np.clip(np.floor(iy + u[1].astype(np.float64) + 0.5), 0, ny - 1).astype(np.intp)
    sz = np.clip(np.floor(iz + u[2].astype(np.float64) + 0.5), 0, nz - 1).astype(np.intp)
    return labels[sz, sy, sx]


def dice_overlap(a, b, cls):
    ma, mb = (np.asarray(a) == cls), (np.asarray(b) == cls)
    na, nb = int(np.count_nonzero(ma)), int(np.count_nonzero(mb))
    if na + nb == 0:
        return 1.0
    return 2.0 * int(np.count_nonzero(ma & mb)) / (na + nb)


def slice_hausdorff_mm(a, b, cls, spacing_mm=1.2):
    from scipy.ndimage import distance_transform_edt
    a, b = np.asarray(a), np.asarray(b)
    per_slice = []
    for za, zb in zip(a, b):
        ma, mb = za == cls, zb == cls
        if not (ma.any() and mb.any()):
            continue
        d_to_b = distance_transform_edt(np.logical_not(mb))
        d_to_a = distance_transform_edt(np.logical_not(ma))
        per_slice.append(max(d_to_b[ma].max(), d_to_a[mb].max()) * spacing_mm)
    return float(np.mean(per_slice)) if per_slice else float("nan")


def score(labels_fixed, labels_moving, u):
    """Dice and per-slice Hausdorff per class after and before registration."""
    warped = carry_labels(labels_moving, u)
    out = {}
    for cls, name in CLASSES.items():
        out[name] = {"dice": dice_overlap(warped, labels_fixed, cls),
                     "dice_unregistered": dice_overlap(labels_moving, labels_fixed, cls),
                     "hausdorff_mm": slice_hausdorff_mm(warped, labels_fixed, cls),
                     "hausdorff_mm_unregistered": slice_hausdorff_mm(labels_moving, labels_fixed,
                                                                     cls)}
    return out
