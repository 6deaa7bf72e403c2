"""Seeded synthetic inputs for masked LDDMM (template/target mask pairs, atlas labels).

The paper registers CLARITY mouse brains to the Allen Reference Atlas (§2.1, §2.2); neither
dataset is available, so every workload here is generated: ellipsoid-union "brains", a smooth
random displacement made of Gaussian radial basis functions, Voronoi atlas regions with uint16
labels, and a sparsely labelled CLARITY-like target.  The masks follow the paper's recipe in
§2.2: the template mask is the union of the foreground labels, the target mask is a threshold
followed by a morphological opening and closing with ball kernels.

This module is shared by the CUDA path's tests/benchmark and by the CPU oracle's tests.  It
holds no arithmetic of the registration method itself (no flows, interpolation, smoothing or
energies): only data generation.  All arrays are C-ordered ``[z][y][x]`` (x fastest).
"""
from __future__ import annotations

import dataclasses

import numpy as np

__all__ = [
    "Pair",
    "ellipsoid",
    "ball",
    "rbf_displacement",
    "nn_pull",
    "dilate",
    "open_close",
    "ellipsoid_pair",
    "brain_pair",
    "union_pair",
    "smooth_velocity",
]


@dataclasses.dataclass
class Pair:
    """One registration problem: template I0, target I1, weight M (all float32 [Z,Y,X])."""

    I0: np.ndarray
    I1: np.ndarray
    M: np.ndarray
    L0: np.ndarray | None = None        # uint16 atlas labels in template space
    L1_true: np.ndarray | None = None   # uint16 labels pulled to target space by the true warp
    u_true: np.ndarray | None = None    # (3,Z,Y,X) float32 true displacement (voxels, x,y,z)
    image1: np.ndarray | None = None    # raw target intensities (before masking)


def _grid(shape):
    Z, Y, X = shape
    z, y, x = np.meshgrid(np.arange(Z, dtype=np.float64), np.arange(Y, dtype=np.float64),
                          np.arange(X, dtype=np.float64), indexing="ij")
    return x, y, z


def ellipsoid(shape, centre_xyz, semi_axes_xyz):
    """Boolean mask of the solid ellipsoid sum(((p - c)/a)^2) <= 1 over voxel centres."""
    x, y, z = _grid(shape)
    cx, cy, cz = centre_xyz
    ax, ay, az = semi_axes_xyz
    return ((x - cx) / ax) ** 2 + ((y - cy) / ay) ** 2 + ((z - cz) / az) ** 2 <= 1.0


def ball(r):
    """Boolean ball structuring element of radius r voxels (Euclidean, r >= 0)."""
    ri = int(np.floor(r))
    g = np.arange(-ri, ri + 1)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    return (x * x + y * y + z * z) <= r * r + 1e-9


def _jacobian_det_min(u):
    """Minimum over voxels of det(I + Du) for a displacement u (3,Z,Y,X) in voxels.

    Only used to reject folding synthetic warps; it is part of data generation, not of the
    registration method.
    """
    D = np.empty((3, 3) + u.shape[1:])
    for d in range(3):
        gz, gy, gx = np.gradient(u[d], axis=(0, 1, 2))
        D[d, 0], D[d, 1], D[d, 2] = gx, gy, gz
    for d in range(3):
        D[d, d] += 1.0
    det = (D[0, 0] * (D[1, 1] * D[2, 2] - D[1, 2] * D[2, 1])
           - D[0, 1] * (D[1, 0] * D[2, 2] - D[1, 2] * D[2, 0])
           + D[0, 2] * (D[1, 0] * D[2, 1] - D[1, 1] * D[2, 0]))
    return float(det.min())


def rbf_displacement(shape, n_rbf, width, amplitude, rng, min_det=0.1, tries=50):
    """Smooth random displacement u(p) = sum_k a_k exp(-|p - c_k|^2 / (2 width^2)).

    Centres c_k are uniform in the middle 60% of the box, a_k ~ N(0, I); the field is rescaled
    so that max |u| = amplitude voxels.  Draws whose map p -> p + u(p) has det(I + Du) <= min_det
    anywhere are rejected and redrawn.  Returns float64 (3,Z,Y,X), components (x, y, z).
    """
    Z, Y, X = shape
    x, y, z = _grid(shape)
    lo = np.array([0.2 * X, 0.2 * Y, 0.2 * Z])
    hi = np.array([0.8 * X, 0.8 * Y, 0.8 * Z])
    for _ in range(tries):
        c = lo + (hi - lo) * rng.random((n_rbf, 3))
        a = rng.standard_normal((n_rbf, 3))
        u = np.zeros((3,) + tuple(shape))
        for k in range(n_rbf):
            g = np.exp(-((x - c[k, 0]) ** 2 + (y - c[k, 1]) ** 2 + (z - c[k, 2]) ** 2)
                       / (2.0 * width * width))
            for d in range(3):
                u[d] += a[k, d] * g
        mag = np.sqrt((u * u).sum(axis=0)).max()
        if mag <= 0:
            continue
        u *= amplitude / mag
        if _jacobian_det_min(u) > min_det:
            return u
    raise RuntimeError("could not draw a non-folding RBF displacement")


def nn_pull(img, u):
    """img(round(p + u(p))) with clamp-to-edge: nearest-neighbour pull-back of any array."""
    Z, Y, X = img.shape
    x, y, z = _grid(img.shape)
    ix = np.clip(np.floor(x + u[0] + 0.5), 0, X - 1).astype(np.int64)
    iy = np.clip(np.floor(y + u[1] + 0.5), 0, Y - 1).astype(np.int64)
    iz = np.clip(np.floor(z + u[2] + 0.5), 0, Z - 1).astype(np.int64)
    return img[iz, iy, ix]


def dilate(mask, r):
    from scipy import ndimage
    if r <= 0:
        return mask.copy()
    return ndimage.binary_dilation(mask, structure=ball(r))


def open_close(mask, r_open, r_close):
    """Opening (removes grains) then closing (fills holes) with ball kernels (§2.2)."""
    from scipy import ndimage
    m = mask
    if r_open > 0:
        m = ndimage.binary_opening(m, structure=ball(r_open))
    if r_close > 0:
        m = ndimage.binary_closing(m, structure=ball(r_close))
    return m


def ellipsoid_pair(shape=(32, 32, 32), centre=(15.5, 15.5, 15.5), semi_axes=(10, 8, 7),
                   n_rbf=8, width=6.0, amplitude=3.0, seed=0, dilate_r=2):
    """Single-ellipsoid mask pair: template mask, same mask pulled through a random RBF warp.

    Mask-LDDMM (§2.3) registers the masks themselves: I0 = M0, I1 = M1.  The weight M is the
    union of both masks dilated by ``dilate_r`` voxels.
    """
    rng = np.random.default_rng(seed)
    m0 = ellipsoid(shape, centre, semi_axes)
    u = rbf_displacement(shape, n_rbf, width, amplitude, rng)
    m1 = nn_pull(m0, u)
    M = dilate(m0 | m1, dilate_r)
    return Pair(I0=m0.astype(np.float32), I1=m1.astype(np.float32), M=M.astype(np.float32),
                u_true=u.astype(np.float32))


def union_pair(shape, n_ell=3, n_rbf=16, width=None, amplitude=5.0, seed=100, dilate_r=2):
    """Ellipsoid-union mask pair (2 to n_ell overlapping ellipsoids) warped by RBFs."""
    rng = np.random.default_rng(seed)
    Z, Y, X = shape
    n = int(rng.integers(2, n_ell + 1))
    m0 = np.zeros(shape, bool)
    for _ in range(n):
        c = (X * rng.uniform(0.4, 0.6), Y * rng.uniform(0.4, 0.6), Z * rng.uniform(0.4, 0.6))
        a = (X * rng.uniform(0.15, 0.3), Y * rng.uniform(0.15, 0.3), Z * rng.uniform(0.15, 0.3))
        m0 |= ellipsoid(shape, c, a)
    if width is None:
        width = 0.08 * min(shape)
    u = rbf_displacement(shape, n_rbf, width, amplitude, rng)
    m1 = nn_pull(m0, u)
    M = dilate(m0 | m1, dilate_r)
    return Pair(I0=m0.astype(np.float32), I1=m1.astype(np.float32), M=M.astype(np.float32),
                u_true=u.astype(np.float32))


def brain_pair(shape=(114, 80, 132), base_shape=(114, 80, 132), n_regions=50, n_rbf=16,
               amplitude=6.0, seed=1, dilate_r=2):
    """Brain-shaped atlas and sparsely labelled target (stand-ins for the ARA and a CLARITY brain).

    Atlas: union of three overlapping ellipsoids; ``n_regions`` Voronoi regions with labels
    1..n (ties go to the lower index) and grey levels N(0.5, 0.15).  Target: the atlas shape
    pulled through a 16-RBF warp (max |u| = ``amplitude`` voxels of ``base_shape``); inside it a
    0.05 background plus Bernoulli(1%) voxels carrying LogNormal(0, 1) intensities; zero outside;
    N(0, 0.02^2) noise everywhere.  Masks per §2.2: M0 = union of foreground labels; M1 =
    threshold of the Gaussian-smoothed target, opened then closed with ball kernels (radii 50 and
    125 um at a 100 um grid = 1 voxel each, scaled with the grid).  Geometry is defined relative
    to the box, so the same brain appears at any grid size; ``base_shape`` fixes the physical
    scale of the warp amplitude, RBF width and morphology radii.
    """
    from scipy import ndimage
    rng = np.random.default_rng(seed)
    Z, Y, X = shape
    s = X / float(base_shape[2])            # grid refinement relative to the base grid
    cen = [(0.5, 0.5, 0.5), (0.38, 0.5, 0.55), (0.62, 0.5, 0.55)]
    axes = [(0.36, 0.30, 0.30), (0.2, 0.22, 0.22), (0.2, 0.22, 0.22)]
    m0 = np.zeros(shape, bool)
    for c, a in zip(cen, axes):
        m0 |= ellipsoid(shape, (c[0] * X - 0.5, c[1] * Y - 0.5, c[2] * Z - 0.5),
                        (a[0] * X, a[1] * Y, a[2] * Z))
    # Voronoi regions: seeds uniform among atlas voxels, nearest seed wins, ties -> lower index
    inside = np.flatnonzero(m0.ravel())
    seeds = inside[rng.choice(inside.size, size=n_regions, replace=False)]
    sz, sy, sx = np.unravel_index(seeds, shape)
    sxyz = np.stack([sx, sy, sz], 1).astype(np.float64)
    pz, py, px = np.unravel_index(inside, shape)
    lab = np.empty(inside.size, np.int64)
    chunk = 1 << 18
    for i in range(0, inside.size, chunk):
        p = np.stack([px[i:i + chunk], py[i:i + chunk], pz[i:i + chunk]], 1).astype(np.float64)
        d2 = ((p[:, None, :] - sxyz[None, :, :]) ** 2).sum(-1)
        lab[i:i + chunk] = np.argmin(d2, axis=1)
    L0 = np.zeros(Z * Y * X, np.uint16)
    L0[inside] = (lab + 1).astype(np.uint16)
    L0 = L0.reshape(shape)
    grey = rng.normal(0.5, 0.15, n_regions + 1)
    grey[0] = 0.0
    atlas_img = grey[L0.astype(np.int64)].astype(np.float32)
    # target geometry: RBF warp, amplitude and width in base-grid voxels scaled to this grid
    u = rbf_displacement(shape, n_rbf, 10.0 * s, amplitude * s, rng)
    m_t = nn_pull(m0, u)
    L1_true = nn_pull(L0, u)
    bright = rng.random(shape) < 0.01
    inten = np.where(bright, rng.lognormal(0.0, 1.0, shape), 0.0) + 0.05
    image1 = np.where(m_t, inten, 0.0) + rng.normal(0.0, 0.02, shape)
    # target mask per §2.2: threshold -> open -> close
    sm = ndimage.gaussian_filter(image1, 1.0 * s)
    r1 = max(1, int(round(1.0 * s)))
    r2 = max(1, int(round(1.25 * s)))
    m1 = open_close(sm > 0.025, r1, r2)
    M = dilate(m0 | m1, max(1, int(round(dilate_r * s))))
    return Pair(I0=m0.astype(np.float32), I1=m1.astype(np.float32), M=M.astype(np.float32),
                L0=L0, L1_true=L1_true, u_true=u.astype(np.float32),
                image1=image1.astype(np.float32)), atlas_img


def smooth_velocity(T, shape, amplitude, seed, n_rbf=4, width=None):
    """A smooth random time-varying velocity field (T,3,Z,Y,X) float32 for parity tests."""
    rng = np.random.default_rng(seed)
    Z, Y, X = shape
    if width is None:
        width = 0.25 * min(shape)
    x, y, z = _grid(shape)
    v = np.zeros((T, 3) + tuple(shape))
    for t in range(T):
        for _ in range(n_rbf):
            c = rng.random(3) * np.array([X, Y, Z])
            a = rng.standard_normal(3)
            g = np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) / (2 * width ** 2))
            for d in range(3):
                v[t, d] += a[d] * g
    m = np.abs(v).max()
    if m > 0:
        v *= amplitude / m
    return v.astype(np.float32)
