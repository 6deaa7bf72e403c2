"""FP64 CPU oracle for the Image-LDDMM preprocessing and the mask generation of §2.2.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU-baseline leg
may import it.  It shares no code with the CUDA path.

Passages followed (Kutten et al., SPIE 2016, §2.2):
* Image-LDDMM preprocessing: the masks M0, M1 are applied to I0, I1; the masked I0 is then
  histogram-matched to the masked I1 with 32-bin histograms of both, matched exactly at 8
  quantile points and by interpolation at all other intensities.
* Target mask: I1 is thresholded to remove the background, the rough mask is opened with a
  ball (radius 50 um) to remove foreground grains, then closed with a ball (radius 125 um) to
  remove large foreground holes.

Readings where the paper leaves the discrete form open:
* The histograms count the voxels inside each mask, in `bins` equal bins over [min, max] of the
  in-mask intensities (a value equal to max falls in the last bin).
* The quantile at fraction f is read off the cumulative histogram: the first bin b whose
  cumulative count reaches f n, plus the fraction of that bin's count still needed:
      q(f) = min + w (b + (f n - C_{b-1}) / c_b),   w = (max - min) / bins.
* The match points are f = k / (points + 1), k = 1..points, and the two ends map min to min and
  max to max.  Between consecutive points the map is linear; beyond the ends it continues the end
  segments.  Voxels outside M0 stay 0.
* Ball of radius r: the offsets with dx^2 + dy^2 + dz^2 <= r^2 (voxels).  Voxels beyond the grid
  count as background for erosion and dilation (opening = erosion then dilation, closing =
  dilation then erosion).
"""
from __future__ import annotations

import numpy as np
from scipy import ndimage

__all__ = ["match_nodes", "histogram_match", "ball", "mask_morphology", "erode_brute",
           "dilate_brute"]


def _quantile(vals, lo, hi, bins, f):
    n = vals.size
    w = (hi - lo) / bins
    if w <= 0.0:
        return lo
    b = np.minimum(np.floor((vals - lo) / w).astype(np.int64), bins - 1)
    c = np.bincount(b, minlength=bins).astype(np.float64)
    C = np.cumsum(c)
    t = f * n
    k = int(np.searchsorted(C, t, side="left"))
    k = min(k, bins - 1)
    prev = C[k - 1] if k > 0 else 0.0
    return lo + w * (k + (t - prev) / c[k]) if c[k] > 0 else lo + w * k


def match_nodes(I0, M0, I1, M1, bins=32, points=8):
    """The piecewise-linear map's nodes (x: source intensities, y: reference intensities)."""
    s = np.asarray(I0, np.float64)[np.asarray(M0) > 0.5]
    r = np.asarray(I1, np.float64)[np.asarray(M1) > 0.5]
    xs = [s.min()] + [_quantile(s, s.min(), s.max(), bins, k / (points + 1))
                      for k in range(1, points + 1)] + [s.max()]
    ys = [r.min()] + [_quantile(r, r.min(), r.max(), bins, k / (points + 1))
                      for k in range(1, points + 1)] + [r.max()]
    return np.array(xs), np.array(ys)


def _map(v, xs, ys):
    n = len(xs)
    # segment index: the last k with xs[k] <= v, clipped to the end segments
    k = np.clip(np.searchsorted(xs, v, side="right") - 1, 0, n - 2)
    x0, x1, y0, y1 = xs[k], xs[k + 1], ys[k], ys[k + 1]
    dx = x1 - x0
    slope = np.where(dx > 0, (y1 - y0) / np.where(dx > 0, dx, 1.0), 0.0)
    return y0 + (v - x0) * slope


def histogram_match(I0, M0, I1, M1, bins=32, points=8):
    """Masked I0 matched to masked I1 (float64; 0 outside M0)."""
    xs, ys = match_nodes(I0, M0, I1, M1, bins, points)
    v = np.asarray(I0, np.float64)
    out = _map(v, xs, ys)
    return np.where(np.asarray(M0) > 0.5, out, 0.0)


def ball(r):
    d = np.arange(-r, r + 1)
    z, y, x = np.meshgrid(d, d, d, indexing="ij")
    return (x * x + y * y + z * z) <= r * r


def mask_morphology(I, threshold, r_open, r_close):
    """[I > threshold], opened with ball(r_open), then closed with ball(r_close)."""
    m = np.asarray(I) > threshold
    if r_open > 0:
        m = ndimage.binary_opening(m, structure=ball(r_open), border_value=0)
    if r_close > 0:
        m = ndimage.binary_closing(m, structure=ball(r_close), border_value=0)
    return m


def _shifted(m, dz, dy, dx):
    """m shifted so that out[z, y, x] = m[z + dz, y + dy, x + dx], background beyond the grid."""
    Z, Y, X = m.shape
    out = np.zeros_like(m)
    zs, ys, xs = slice(max(0, -dz), min(Z, Z - dz)), slice(max(0, -dy), min(Y, Y - dy)), slice(max(0, -dx), min(X, X - dx))
    zd, yd, xd = slice(max(0, dz), min(Z, Z + dz)), slice(max(0, dy), min(Y, Y + dy)), slice(max(0, dx), min(X, X + dx))
    out[zs, ys, xs] = m[zd, yd, xd]
    return out


def erode_brute(m, r):
    """Erosion by ball(r), one offset at a time (small volumes)."""
    m = np.asarray(m, bool)
    out = np.ones_like(m)
    for dz, dy, dx in np.argwhere(ball(r)) - r:
        out &= _shifted(m, dz, dy, dx)
    return out


def dilate_brute(m, r):
    """Dilation by ball(r), one offset at a time (small volumes)."""
    m = np.asarray(m, bool)
    out = np.zeros_like(m)
    for dz, dy, dx in np.argwhere(ball(r)) - r:
        out |= _shifted(m, dz, dy, dx)
    return out
