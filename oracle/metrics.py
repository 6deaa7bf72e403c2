"""FP64 CPU oracle for the registration-quality measures of §2.7 (surface and landmark error).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
may import it.  It shares no code with the CUDA path.

Definitions (Kutten et al., SPIE 2016, §2.7):
* Hausdorff distance between the deformed-template surface S(1) = boundary(M0 o phi^-1) and the
  target surface S1 = boundary(M1):
      d_H = max{ sup_{x in S(1)} inf_{y in S1} d(x, y),  sup_{y in S1} inf_{x in S(1)} d(x, y) }.
* Median surface distance: the median of the union of the two sets of directed distances
      { inf_{y in S1} d(x, y) : x in S(1) }  and  { inf_{x in S(1)} d(x, y) : y in S1 }.
* Landmark error: e_k = || phi(x_k) - y_k || for template landmark x_k and target landmark y_k.

Readings where the paper leaves the discrete form open:
* The surface of a binary mask is the set of its voxels with at least one of the six face
  neighbours outside the mask; a neighbour beyond the grid counts as outside.
* d is the Euclidean distance between voxel centres in physical units (spacing hx, hy, hz).
* The median of an even number of values is the mean of the two middle ones (numpy's median).
* phi(x_k) = x_k + u01(x_k), u01 = phi_{0,1} - id interpolated trilinearly (clamp to edge):
  phi_{0,1} carries a template point to the target point it lands on.

Arrays are C-ordered [z][y][x].
"""
from __future__ import annotations

import numpy as np
from scipy import ndimage

from . import lddmm as _L

__all__ = ["surface", "directed_distances", "surface_distances", "brute_surface_distances",
           "landmark_errors"]


def surface(mask):
    """Voxels of a binary mask with a face neighbour outside it (outside the grid counts)."""
    m = np.asarray(mask).astype(bool)
    p = np.pad(m, 1, mode="constant", constant_values=False)
    inner = np.ones_like(m)
    for ax in range(3):
        for s in (-1, 1):
            inner &= np.roll(p, s, axis=ax)[1:-1, 1:-1, 1:-1]
    return m & ~inner


def directed_distances(SA, SB, h=(1.0, 1.0, 1.0)):
    """For every voxel of the surface SA (in C order), the distance to the nearest voxel of SB,
    through the exact Euclidean distance transform of the complement of SB."""
    hx, hy, hz = h
    dt = ndimage.distance_transform_edt(~SB, sampling=(hz, hy, hx))
    return dt[SA]


def surface_distances(A, B, h=(1.0, 1.0, 1.0)):
    """(d_H, d_M) between the surfaces of masks A and B (§2.7)."""
    SA, SB = surface(A), surface(B)
    if not SA.any() or not SB.any():
        raise ValueError("a mask has no surface voxel")
    da = directed_distances(SA, SB, h)
    db = directed_distances(SB, SA, h)
    return float(max(da.max(), db.max())), float(np.median(np.concatenate([da, db])))


def brute_surface_distances(A, B, h=(1.0, 1.0, 1.0)):
    """The same by comparing every pair of surface voxels (small volumes only)."""
    SA, SB = surface(A), surface(B)
    pa = np.argwhere(SA)[:, ::-1] * np.asarray(h, dtype=np.float64)   # (x, y, z) physical
    pb = np.argwhere(SB)[:, ::-1] * np.asarray(h, dtype=np.float64)
    d = np.sqrt(((pa[:, None, :] - pb[None, :, :]) ** 2).sum(-1))
    da, db = d.min(axis=1), d.min(axis=0)
    return float(max(da.max(), db.max())), float(np.median(np.concatenate([da, db])))


def landmark_errors(u01, xk, yk, h=(1.0, 1.0, 1.0)):
    """e_k = |phi(x_k) - y_k| in physical units; xk, yk as (n, 3) voxel coordinates (x, y, z)."""
    xk = np.asarray(xk, dtype=np.float64)
    yk = np.asarray(yk, dtype=np.float64)
    d = _L.interp_vec(u01, xk[:, 0], xk[:, 1], xk[:, 2])   # (3, n) displacement in voxels
    px = xk + d.T
    return np.sqrt((((px - yk) * np.asarray(h, dtype=np.float64)) ** 2).sum(-1))
