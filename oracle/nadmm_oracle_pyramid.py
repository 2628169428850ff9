"""The three-level pyramid around the registration (Sec. 4, "Hyperparameter
tuning").

TEST INFRASTRUCTURE ONLY, like ``nadmm_oracle``.

The paper embeds the method in a three-level pyramid and, for its first
hyper-parameter version, caps the ADMM iterations at ten on the first level
and five on the next two, and the warpings at ten on the first two levels
and five on the last.  Readings (the paper gives no further detail):

* the first level is the coarsest; each level halves every dimension;
* a coarser image is the 2 x 2 x 2 block average of the finer one;
* the displacement found on a coarser level starts the next finer level,
  resampled at cell centres and doubled:
  u_fine(x) = 2 u_coarse((x - 1/2) / 2), trilinear with clamped coordinates;
* lambda, theta, n, the data term and the velocity bound (in voxels of the
  level) are the same on every level.
"""
from __future__ import annotations

import numpy as np

from .nadmm_oracle import _grid, register, trilinear

__all__ = ["downsample2", "upsample_displacement", "register_pyramid",
           "PAPER_V1_OUTER", "PAPER_V1_INNER"]

# coarsest level first
PAPER_V1_OUTER = (10, 10, 5)
PAPER_V1_INNER = (10, 5, 5)


def downsample2(f):
    """2 x 2 x 2 block average of f [nz][ny][nx] (even dimensions)."""
    f = np.asarray(f, np.float64)
    nz, ny, nx = f.shape
    return f.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2).mean(axis=(1, 3, 5))


def upsample_displacement(uc, fine_shape):
    """u_fine(x) = 2 u_coarse((x - 1/2) / 2) per component, for the fine grid
    fine_shape = (nz, ny, nx); displacements in voxels of each grid."""
    uc = np.asarray(uc, np.float64)
    x, y, z = _grid(fine_shape)
    px, py, pz = (x - 0.5) / 2.0, (y - 0.5) / 2.0, (z - 0.5) / 2.0
    return np.stack([2.0 * trilinear(uc[i], px, py, pz) for i in range(3)])


def register_pyramid(I0, I1, outer=PAPER_V1_OUTER, inner=PAPER_V1_INNER, **kw):
    """Registration on len(outer) levels, coarsest first; outer[i], inner[i]
    are the warpings and ADMM iterations of level i.  Returns u on the finest
    grid."""
    levels = len(outer)
    assert len(inner) == levels
    I0s = [np.asarray(I0, np.float64)]
    I1s = [np.asarray(I1, np.float64)]
    for _ in range(levels - 1):
        I0s.append(downsample2(I0s[-1]))
        I1s.append(downsample2(I1s[-1]))
    u = None
    for i in range(levels):
        lvl = levels - 1 - i  # index into the finest-first image lists
        if u is not None:
            u = upsample_displacement(u, I0s[lvl].shape)
        u = register(I0s[lvl], I1s[lvl], outer=outer[i], inner=inner[i], u0=u, **kw)
    return u
