"""Evaluation measures of Sec. 4 ("Quantitative results") on label maps.

TEST INFRASTRUCTURE ONLY, like ``nadmm_oracle``.  The paper scores a
registration by the Dice overlap of the RV, LV and LVM labels, the Hausdorff
distance averaged over 2D slices (in mm, 1.2 mm isotropic voxels) and the
share of voxels with a non-positive Jacobian determinant.

Readings: labels are carried by nearest-neighbour sampling at x + u(x)
(coordinates rounded half away from zero and clamped); the per-slice
Hausdorff distance is the symmetric maximum over the label's pixels of each
z-slice in which both maps contain the label, averaged over those slices;
slices where either map lacks the label are skipped.
"""
from __future__ import annotations

import numpy as np
from scipy.ndimage import distance_transform_edt

from .nadmm_oracle import _grid, jacobian_determinant

__all__ = ["warp_labels", "dice", "hausdorff_per_slice", "nonpositive_jacobian_percent"]


def warp_labels(labels, u):
    """labels(x + u(x)) by nearest neighbour, coordinates clamped to the grid."""
    labels = np.asarray(labels)
    u = np.asarray(u, np.float64)
    nz, ny, nx = labels.shape
    x, y, z = _grid(labels.shape)

    def near(p, n):
        return np.clip(np.floor(p + 0.5), 0, n - 1).astype(np.int64)
    return labels[near(z + u[2], nz), near(y + u[1], ny), near(x + u[0], nx)]


def dice(a, b, label):
    """2 |A & B| / (|A| + |B|) for the voxels carrying `label`; 1 if both are empty."""
    A = np.asarray(a) == label
    B = np.asarray(b) == label
    s = int(A.sum()) + int(B.sum())
    return 1.0 if s == 0 else 2.0 * int((A & B).sum()) / s


def _directed(A, B):
    # largest distance from a pixel of A to the nearest pixel of B
    d = distance_transform_edt(~B)
    return float(d[A].max())


def hausdorff_per_slice(a, b, label, spacing=1.2):
    """Mean over z-slices of the symmetric Hausdorff distance (mm) of `label`."""
    a = np.asarray(a)
    b = np.asarray(b)
    vals = []
    for z in range(a.shape[0]):
        A = a[z] == label
        B = b[z] == label
        if A.any() and B.any():
            vals.append(max(_directed(A, B), _directed(B, A)) * spacing)
    return float(np.mean(vals)) if vals else float("nan")


def nonpositive_jacobian_percent(u):
    """100 x the share of voxels with det(I + Du) <= 0."""
    det = jacobian_determinant(u)
    return 100.0 * float((det <= 0).sum()) / det.size
