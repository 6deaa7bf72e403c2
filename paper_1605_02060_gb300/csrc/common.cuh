// Device helpers shared by the liblddmm kernels: grid geometry, clamped trilinear sampling,
// finite-difference stencils and block reductions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <cuda_bf16.h>

namespace lddmm {

struct Grid {
  int nx, ny, nz;
  int N;          // nx*ny*nz (checked < 2^31 / 3 on the host)
};

// Corner index and weights of a clamped trilinear lookup at voxel coordinate q.
// Coordinates are clamped to [0, n-1]; the lower corner to [0, n-2] (n >= 2 everywhere),
// so the fraction lies in [0, 1].
struct Tri {
  int base;       // linear index of the lower corner
  int sx, sy, sz; // strides to the upper corner along each axis
  float tx, ty, tz;
};

__device__ __forceinline__ void axis_corner(float q, int n, int& i0, float& t) {
  q = fminf(fmaxf(q, 0.0f), (float)(n - 1));
  int i = (int)floorf(q);
  i = min(i, n - 2);
  i0 = i;
  t = q - (float)i;
}

__device__ __forceinline__ Tri tri_setup(const Grid& g, float qx, float qy, float qz) {
  Tri w;
  int ix, iy, iz;
  axis_corner(qx, g.nx, ix, w.tx);
  axis_corner(qy, g.ny, iy, w.ty);
  axis_corner(qz, g.nz, iz, w.tz);
  w.base = (iz * g.ny + iy) * g.nx + ix;
  w.sx = 1;
  w.sy = g.nx;
  w.sz = g.nx * g.ny;
  return w;
}

// Interpolate x first, then y, then z (the order of the lerps is part of the FP32 result).
__device__ __forceinline__ float tri_apply(const float* __restrict__ f, const Tri& w) {
  const float* p = f + w.base;
  float c000 = __ldg(p), c001 = __ldg(p + w.sx);
  float c010 = __ldg(p + w.sy), c011 = __ldg(p + w.sy + w.sx);
  float c100 = __ldg(p + w.sz), c101 = __ldg(p + w.sz + w.sx);
  float c110 = __ldg(p + w.sz + w.sy), c111 = __ldg(p + w.sz + w.sy + w.sx);
  float a00 = c000 + w.tx * (c001 - c000);
  float a01 = c010 + w.tx * (c011 - c010);
  float a10 = c100 + w.tx * (c101 - c100);
  float a11 = c110 + w.tx * (c111 - c110);
  float b0 = a00 + w.ty * (a01 - a00);
  float b1 = a10 + w.ty * (a11 - a10);
  return b0 + w.tz * (b1 - b0);
}

__device__ __forceinline__ float tri_sample(const float* __restrict__ f, const Grid& g,
                                            float qx, float qy, float qz) {
  return tri_apply(f, tri_setup(g, qx, qy, qz));
}

// Storage-type-generic loads: fields may be stored as float or bf16; arithmetic is FP32.
__device__ __forceinline__ float ldf(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ldf(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }
__device__ __forceinline__ void stf(float* p, float v) { *p = v; }
// Loads issued where they are written (volatile asm is not moved by the compiler): used for
// prefetches whose value is consumed several iterations later, which the compiler would
// otherwise sink next to the use and so expose the full memory latency.
__device__ __forceinline__ float ldf_now(const float* p) {
  float v;
  asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ float ldf_now(const __nv_bfloat16* p) {
  unsigned short h;
  asm volatile("ld.global.nc.u16 %0, [%1];" : "=h"(h) : "l"(p));
  return __bfloat162float(__ushort_as_bfloat16(h));
}
__device__ __forceinline__ void stf(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

template <typename T>
__device__ __forceinline__ float tri_apply_t(const T* __restrict__ f, const Tri& w) {
  const T* p = f + w.base;
  const float c000 = ldf(p), c001 = ldf(p + w.sx);
  const float c010 = ldf(p + w.sy), c011 = ldf(p + w.sy + w.sx);
  const float c100 = ldf(p + w.sz), c101 = ldf(p + w.sz + w.sx);
  const float c110 = ldf(p + w.sz + w.sy), c111 = ldf(p + w.sz + w.sy + w.sx);
  const float a00 = c000 + w.tx * (c001 - c000);
  const float a01 = c010 + w.tx * (c011 - c010);
  const float a10 = c100 + w.tx * (c101 - c100);
  const float a11 = c110 + w.tx * (c111 - c110);
  const float b0 = a00 + w.ty * (a01 - a00);
  const float b1 = a10 + w.ty * (a11 - a10);
  return b0 + w.tz * (b1 - b0);
}

// Neighbour offsets and divisor of the first-derivative stencil along one axis at index i:
// central (i-1, i+1)/2 inside, one-sided (i, i+1) or (i-1, i) at the faces.
__device__ __forceinline__ void fd_stencil(int i, int n, int stride, int& lo, int& hi,
                                           float& inv) {
  if (i == 0) { lo = 0; hi = stride; inv = 1.0f; }
  else if (i == n - 1) { lo = -stride; hi = 0; inv = 1.0f; }
  else { lo = -stride; hi = stride; inv = 0.5f; }
}

// Linear thread index within the block (warps are 32 consecutive linear indices).
__device__ __forceinline__ int linear_tid() {
  return (threadIdx.z * blockDim.y + threadIdx.y) * blockDim.x + threadIdx.x;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum of a double, one atomicAdd per block into *dst.  blockDim.x % 32 == 0.
__device__ __forceinline__ void block_sum_atomic(double v, double* dst) {
  __shared__ double red[32];
  v = warp_sum(v);
  const int lt = linear_tid(), lane = lt & 31, wid = lt >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x * blockDim.y * blockDim.z) >> 5;
    double s = lane < nw ? red[lane] : 0.0;
    s = warp_sum(s);
    if (lane == 0 && s != 0.0) atomicAdd(dst, s);
  }
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of per-thread float partials: FP32 within a warp (32 terms), FP64 across warps
// and for the global accumulator (one atomicAdd per block).
__device__ __forceinline__ void block_sum_f_atomic(float v, double* dst) {
  __shared__ double redf[32];
  v = warp_sum_f(v);
  const int lt = linear_tid(), lane = lt & 31, wid = lt >> 5;
  if (lane == 0) redf[wid] = (double)v;
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x * blockDim.y * blockDim.z) >> 5;
    double s = lane < nw ? redf[lane] : 0.0;
    s = warp_sum(s);
    if (lane == 0 && s != 0.0) atomicAdd(dst, s);
  }
}

// Float min through an order-preserving int encoding (atomicMin on int).
__device__ __forceinline__ int float_to_ordered(float f) {
  int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}

__device__ __forceinline__ void block_min_atomic(float v, int* dst) {
  __shared__ float redm[32];
  v = warp_min(v);
  const int lt = linear_tid(), lane = lt & 31, wid = lt >> 5;
  if (lane == 0) redm[wid] = v;
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x * blockDim.y * blockDim.z) >> 5;
    float s = lane < nw ? redm[lane] : 3.0e38f;
    s = warp_min(s);
    if (lane == 0) atomicMin(dst, float_to_ordered(s));
  }
}

}  // namespace lddmm
