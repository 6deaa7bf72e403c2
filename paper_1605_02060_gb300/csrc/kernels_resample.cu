// Warm-start support: resampling fields between grids of the same box, and scaling a field.
//
// The learned warm start runs its network on a coarse n^3 grid that covers the whole box
// (an anisotropic resample of the registration grid), so the masks go down to n^3 and the
// predicted velocity comes back up to the registration grid.  Both use trilinear interpolation
// at cell-centred coordinates (voxel i of a grid of size d covers [i, i + 1) in units of the box
// divided by d): q = (i + 0.5) s / d - 0.5 in source voxels, clamped to the source grid.
// A velocity in voxels of the coarse grid becomes one in voxels of the fine grid by the ratio of
// the sizes along its own axis, so component c of a vector field is multiplied by scale[c].
#include "../../include/lddmm.h"
#include "kernels.h"

namespace lddmm {

namespace {

// The sample coordinate is formed in double precision (the ratio s/d is not a float), so the
// interpolation weight carries no error beyond its final rounding to float.
__device__ __forceinline__ void axis_weight(double q, int n, int& i0, int& i1, float& t) {
  q = fmin(fmax(q, 0.0), (double)(n - 1));
  int i = (int)floor(q);
  if (i > n - 2) i = n - 2;
  if (i < 0) i = 0;
  i0 = i;
  i1 = n > 1 ? i + 1 : i;
  t = n > 1 ? (float)(q - (double)i) : 0.f;
}

// One thread per destination voxel and field; fields are [nfields][dz][dy][dx].
__global__ void k_resample(const float* __restrict__ src, int sx, int sy, int sz,
                           float* __restrict__ dst, int dx, int dy, int dz, int nfields,
                           int ncomp, float s0, float s1, float s2) {
  const long long nd = (long long)dx * dy * dz;
  const long long total = nd * nfields;
  const double rx = (double)sx / dx, ry = (double)sy / dy, rz = (double)sz / dz;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(i / nd);
    const long long v = i - (long long)f * nd;
    const int x = (int)(v % dx), y = (int)((v / dx) % dy), z = (int)(v / ((long long)dx * dy));
    int x0, x1, y0, y1, z0, z1;
    float tx, ty, tz;
    axis_weight((x + 0.5) * rx - 0.5, sx, x0, x1, tx);
    axis_weight((y + 0.5) * ry - 0.5, sy, y0, y1, ty);
    axis_weight((z + 0.5) * rz - 0.5, sz, z0, z1, tz);
    const float* s = src + (long long)f * sx * sy * sz;
    auto at = [&](int zz, int yy, int xx) { return __ldg(s + ((long long)zz * sy + yy) * sx + xx); };
    const float c00 = at(z0, y0, x0) + tx * (at(z0, y0, x1) - at(z0, y0, x0));
    const float c01 = at(z0, y1, x0) + tx * (at(z0, y1, x1) - at(z0, y1, x0));
    const float c10 = at(z1, y0, x0) + tx * (at(z1, y0, x1) - at(z1, y0, x0));
    const float c11 = at(z1, y1, x0) + tx * (at(z1, y1, x1) - at(z1, y1, x0));
    const float c0 = c00 + ty * (c01 - c00), c1 = c10 + ty * (c11 - c10);
    const int comp = f % ncomp;
    const float sc = comp == 0 ? s0 : comp == 1 ? s1 : s2;
    dst[i] = sc * (c0 + tz * (c1 - c0));
  }
}

__global__ void k_scale(float* __restrict__ x, long long n, float c) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    x[i] *= c;
}

int grid_for(long long n) {
  const long long b = (n + 255) / 256;
  return (int)(b < 152 * 32 ? (b > 0 ? b : 1) : 152 * 32);
}

}  // namespace

}  // namespace lddmm

using namespace lddmm;

extern "C" {

int lddmm_resample(const float* src, int sx, int sy, int sz, float* dst, int dx, int dy, int dz,
                   int nfields, int ncomp, float s0, float s1, float s2, void* stream) {
  if (!src || !dst || sx < 1 || sy < 1 || sz < 1 || dx < 1 || dy < 1 || dz < 1 || nfields < 1 ||
      (ncomp != 1 && ncomp != 3) || nfields % ncomp)
    return LDDMM_ERR_INVALID_ARG;
  if ((long long)dx * dy * dz * nfields > (1LL << 40)) return LDDMM_ERR_INVALID_ARG;
  const long long total = (long long)dx * dy * dz * nfields;
  k_resample<<<grid_for(total), 256, 0, (cudaStream_t)stream>>>(src, sx, sy, sz, dst, dx, dy, dz,
                                                                 nfields, ncomp, s0, s1, s2);
  return cudaGetLastError() == cudaSuccess ? LDDMM_OK : LDDMM_ERR_CUDA;
}

int lddmm_scale(float* x, int64_t count, float c, void* stream) {
  if (!x || count < 0) return LDDMM_ERR_INVALID_ARG;
  if (count == 0) return LDDMM_OK;
  k_scale<<<grid_for(count), 256, 0, (cudaStream_t)stream>>>(x, count, c);
  return cudaGetLastError() == cudaSuccess ? LDDMM_OK : LDDMM_ERR_CUDA;
}

}  // extern "C"
