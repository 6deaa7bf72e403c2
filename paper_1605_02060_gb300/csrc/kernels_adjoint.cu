// Exact gradient of the discrete masked-LDDMM energy with respect to v (reverse mode of the
// forward sweep and of the regulariser), for the autograd path.
//
// Energy (§2.4, discretised): E = dt h^3 sum_j |(gamma - alpha Lap_h) v_j|^2
//                                  + sigma^-2 h^3 sum_x M (I0(x + u_T) - I1)^2,
// forward sweep u_0 = 0, u_{j+1}(x) = -d_j(x) + U_j(q_j(x)),  d_j = dt v_j / h,  q_j = x - d_j,
// with U_j the clamped trilinear interpolant of u_j.  Reverse sweep (g_j = dE/du_j):
//   g_T(x)   = (2 h^3 / sigma^2) M (I0(x + u_T) - I1) grad~I0(x + u_T)
//   dE/dv_j,e(x) = -(dt/h_e) [g_{j+1,e}(x) + sum_c g_{j+1,c}(x) dU_{j,c}/dq_e(q_j(x))]
//                 + 2 dt h^3 (L^2 v_j)_e(x)
//   g_j      = (interpolation at q_j)^T g_{j+1}   (scatter-add with the trilinear weights)
// grad~ is the gradient of the trilinear interpolant; along an axis whose coordinate was clamped
// it is zero.  The scatter uses float atomics, so sums are order-dependent at FP32 rounding.
#include "kernels.h"

namespace lddmm {

namespace {

__device__ __forceinline__ bool vox(const Grid& g, int& x, int& y, int& z, int& idx) {
  x = blockIdx.x * 32 + threadIdx.x;
  y = blockIdx.y * 8 + threadIdx.y;
  z = blockIdx.z;
  idx = (z * g.ny + y) * g.nx + x;
  return x < g.nx && y < g.ny;
}
inline dim3 grid_of(const Grid& g) { return dim3((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz); }
const dim3 kBlk(32, 8, 1);

// Value and coordinate gradient of the trilinear interpolant of f at w (clamped setup); the
// per-axis `in` flags zero the gradient where the coordinate lay outside [0, n-1].
__device__ __forceinline__ float tri_val_grad(const float* __restrict__ f, const Tri& w, float inx,
                                              float iny, float inz, float& gx, float& gy,
                                              float& gz) {
  const float* p = f + w.base;
  const float c000 = __ldg(p), c001 = __ldg(p + w.sx);
  const float c010 = __ldg(p + w.sy), c011 = __ldg(p + w.sy + w.sx);
  const float c100 = __ldg(p + w.sz), c101 = __ldg(p + w.sz + w.sx);
  const float c110 = __ldg(p + w.sz + w.sy), c111 = __ldg(p + w.sz + w.sy + w.sx);
  const float ux = 1.f - w.tx, uy = 1.f - w.ty, uz = 1.f - w.tz;
  const float a00 = c000 + w.tx * (c001 - c000), a01 = c010 + w.tx * (c011 - c010);
  const float a10 = c100 + w.tx * (c101 - c100), a11 = c110 + w.tx * (c111 - c110);
  const float b0 = a00 + w.ty * (a01 - a00), b1 = a10 + w.ty * (a11 - a10);
  gx = inx * (uy * uz * (c001 - c000) + w.ty * uz * (c011 - c010) + uy * w.tz * (c101 - c100) +
              w.ty * w.tz * (c111 - c110));
  gy = iny * (uz * (a01 - a00) + w.tz * (a11 - a10));
  gz = inz * (b1 - b0);
  return b0 + w.tz * (b1 - b0);
}

__device__ __forceinline__ float inside(float q, int n) {
  return (q >= 0.f && q <= (float)(n - 1)) ? 1.f : 0.f;
}

}  // namespace

// g_T = scale M (I0(x + u_T) - I1) grad~I0(x + u_T), scale = 2 h^3 / sigma^2
__global__ void k_adj_init(Grid g, const float* __restrict__ uT, const float* __restrict__ I0,
                           const float* __restrict__ I1, const float* __restrict__ M,
                           float* __restrict__ gT, float scale) {
  int x, y, z, idx;
  if (!vox(g, x, y, z, idx)) return;
  const int N = g.N;
  const float px = (float)x + uT[idx], py = (float)y + uT[N + idx], pz = (float)z + uT[2 * N + idx];
  const Tri w = tri_setup(g, px, py, pz);
  float gx, gy, gz;
  const float j0 = tri_val_grad(I0, w, inside(px, g.nx), inside(py, g.ny), inside(pz, g.nz), gx,
                                gy, gz);
  const float c = scale * M[idx] * (j0 - I1[idx]);
  gT[idx] = c * gx;
  gT[N + idx] = c * gy;
  gT[2 * N + idx] = c * gz;
}

// One reverse step: data part of dE/dv_j into grad_j, and g_j += interp^T g_{j+1} (if gcur).
__global__ void k_adj_step(Grid g, const float* __restrict__ vj, const float* __restrict__ uj,
                           const float* __restrict__ gnext, float* __restrict__ gcur,
                           float* __restrict__ gradj, float dtx, float dty, float dtz) {
  int x, y, z, idx;
  if (!vox(g, x, y, z, idx)) return;
  const int N = g.N;
  const float dx = dtx * vj[idx], dy = dty * vj[N + idx], dz = dtz * vj[2 * N + idx];
  const float qx = (float)x - dx, qy = (float)y - dy, qz = (float)z - dz;
  const float gv[3] = {gnext[idx], gnext[N + idx], gnext[2 * N + idx]};
  const Tri w = tri_setup(g, qx, qy, qz);
  float s[3] = {gv[0], gv[1], gv[2]};
  if (uj) {
    const float ix = inside(qx, g.nx), iy = inside(qy, g.ny), iz = inside(qz, g.nz);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float jx, jy, jz;
      tri_val_grad(uj + c * N, w, ix, iy, iz, jx, jy, jz);
      s[0] = fmaf(gv[c], jx, s[0]);
      s[1] = fmaf(gv[c], jy, s[1]);
      s[2] = fmaf(gv[c], jz, s[2]);
    }
  }
  gradj[idx] = -dtx * s[0];
  gradj[N + idx] = -dty * s[1];
  gradj[2 * N + idx] = -dtz * s[2];
  if (gcur) {
    const float wx[2] = {1.f - w.tx, w.tx}, wy[2] = {1.f - w.ty, w.ty}, wz[2] = {1.f - w.tz, w.tz};
#pragma unroll
    for (int cz = 0; cz < 2; ++cz)
#pragma unroll
      for (int cy = 0; cy < 2; ++cy)
#pragma unroll
        for (int cx = 0; cx < 2; ++cx) {
          const float wt = wz[cz] * wy[cy] * wx[cx];
          if (wt == 0.f) continue;
          const int o = w.base + cz * w.sz + cy * w.sy + cx * w.sx;
          atomicAdd(gcur + o, wt * gv[0]);
          atomicAdd(gcur + N + o, wt * gv[1]);
          atomicAdd(gcur + 2 * N + o, wt * gv[2]);
        }
  }
}

// dst (+)= scale (gamma - alpha Lap_h) src for 3 components, periodic 7-point stencil.
__global__ void k_apply_L3(Grid g, const float* __restrict__ src, float* __restrict__ dst,
                           float alpha, float gamma, float ihx2, float ihy2, float ihz2,
                           float scale, int accumulate) {
  int x, y, z, idx;
  if (!vox(g, x, y, z, idx)) return;
  const int xm = (x == 0 ? g.nx - 1 : -1), xp = (x == g.nx - 1 ? -(g.nx - 1) : 1);
  const int sy = g.nx, sz = g.nx * g.ny;
  const int ym = (y == 0 ? (g.ny - 1) * sy : -sy), yp = (y == g.ny - 1 ? -(g.ny - 1) * sy : sy);
  const int zm = (z == 0 ? (g.nz - 1) * sz : -sz), zp = (z == g.nz - 1 ? -(g.nz - 1) * sz : sz);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float* p = src + c * g.N + idx;
    const float v = p[0];
    const float lap = (__ldg(p + xm) - 2.f * v + __ldg(p + xp)) * ihx2 +
                      (__ldg(p + ym) - 2.f * v + __ldg(p + yp)) * ihy2 +
                      (__ldg(p + zm) - 2.f * v + __ldg(p + zp)) * ihz2;
    const float r = scale * (gamma * v - alpha * lap);
    if (accumulate) dst[c * g.N + idx] += r;
    else dst[c * g.N + idx] = r;
  }
}

void launch_adj_init(const Grid& g, const float* uT, const float* I0, const float* I1,
                     const float* M, float* gT, float scale, cudaStream_t s) {
  k_adj_init<<<grid_of(g), kBlk, 0, s>>>(g, uT, I0, I1, M, gT, scale);
}

void launch_adj_step(const Grid& g, const float* vj, const float* uj, const float* gnext,
                     float* gcur, float* gradj, float dtx, float dty, float dtz, cudaStream_t s) {
  k_adj_step<<<grid_of(g), kBlk, 0, s>>>(g, vj, uj, gnext, gcur, gradj, dtx, dty, dtz);
}

void launch_apply_L3(const Grid& g, const float* src, float* dst, float alpha, float gamma,
                     float ihx2, float ihy2, float ihz2, float scale, bool accumulate,
                     cudaStream_t s) {
  k_apply_L3<<<grid_of(g), kBlk, 0, s>>>(g, src, dst, alpha, gamma, ihx2, ihy2, ihz2, scale,
                                         accumulate ? 1 : 0);
}

}  // namespace lddmm
