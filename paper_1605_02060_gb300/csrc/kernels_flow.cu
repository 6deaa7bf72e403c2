// Flow, residual, update, warp, label and resampling kernels of one masked-LDDMM iteration.
//
// Method: §2.4 of Kutten et al. (SPIE 2016) — the energy E(v), the operator L and the flow of a
// time-varying velocity field — with the gradient and update of Beg et al. 2005 (cited there):
//   backward sweep  phi_{j,1}(x) = phi_{j+1,1}(x + dt v_j(x)),  J1_j = I1 o phi_{j,1},
//                   W_j = (M o phi_{j,1}) det D phi_{j,1};
//   forward sweep   J0_j = I0 o phi_{j,0},  b_j = (2/sigma^2) W_j (J0_j - J1_j) grad J0_j,
//                   phi_{j+1,0}(x) = phi_{j,0}(x - dt v_j(x));
//   update          v_j <- v_j - eps (2 v_j - K b_j).
// Maps are displacements u = phi - id in voxels; dt v / h converts a velocity to voxels.
// The velocity field and the images are stored as ST = float or bf16 (the precision form);
// every computation is FP32 and reductions are FP64.  Kernels run on (32, 8) blocks over a
// (ceil(nx/32), ceil(ny/8), nz) grid: rows of x are coalesced and no voxel index is divided.
#include "kernels.h"

namespace lddmm {

static inline int nblocks(int64_t n, int t) { return (int)((n + t - 1) / t); }

__device__ __forceinline__ bool voxel3d(const Grid& g, int& x, int& y, int& z, int& idx) {
  x = blockIdx.x * 32 + threadIdx.x;
  y = blockIdx.y * 8 + threadIdx.y;
  z = blockIdx.z;
  idx = (z * g.ny + y) * g.nx + x;
  return x < g.nx && y < g.ny;
}

static inline dim3 grid3d(const Grid& g) { return dim3((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz); }
static const dim3 kBlock3d(32, 8, 1);

// --------------------------------------------------------------------------------------------
// One semi-Lagrangian step of a map, marching ZC planes in z per thread:
//   u_out(x) = s dt v_j(x)/h + u_in(x + s dt v_j(x)/h)   (u_in == nullptr: the identity),
// s = +1 for phi_{j,1} (backward sweep) and s = -1 for phi_{j+1,0} (forward sweep).  A voxel
// costs two dependent memory latencies (v_j, then the eight corners at the displaced point); the
// velocity of plane z+1 is loaded before the corners of plane z are requested, so the two
// overlap.  Consecutive planes also gather from overlapping cells, which L1 keeps.
// Maps (displacements u = phi - id, voxel units) in one of two layouts: planar, [3][N] (the
// layout of the public entry points, the exact gradient and shooting), or quad, [N] x (u_x, u_y,
// u_z, 0) in 16 bytes (the iteration's own sweeps: a stencil neighbour or a trilinear corner is
// one 16-byte load instead of three).  Lookups interpolate each component in the same order
// (x, then y, then z), so both layouts give the same values.
template <bool Q> struct MapL;
template <> struct MapL<false> {
  static __device__ __forceinline__ float3 at(const float* __restrict__ u, int N, int i) {
    return make_float3(__ldg(u + i), __ldg(u + N + i), __ldg(u + 2 * N + i));
  }
  static __device__ __forceinline__ void put(float* __restrict__ u, int N, int i, float a, float b,
                                             float c) {
    u[i] = a;
    u[N + i] = b;
    u[2 * N + i] = c;
  }
  static __device__ __forceinline__ float3 lerp(const float* __restrict__ u, int N, const Tri& w) {
    return make_float3(tri_apply(u, w), tri_apply(u + N, w), tri_apply(u + 2 * N, w));
  }
};
template <> struct MapL<true> {
  static __device__ __forceinline__ float3 at(const float* __restrict__ u, int, int i) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(u) + i);
    return make_float3(q.x, q.y, q.z);
  }
  static __device__ __forceinline__ void put(float* __restrict__ u, int, int i, float a, float b,
                                             float c) {
    reinterpret_cast<float4*>(u)[i] = make_float4(a, b, c, 0.f);
  }
  static __device__ __forceinline__ float lerp1(float c000, float c001, float c010, float c011,
                                                float c100, float c101, float c110, float c111,
                                                const Tri& w) {
    const float a00 = c000 + w.tx * (c001 - c000);
    const float a01 = c010 + w.tx * (c011 - c010);
    const float a10 = c100 + w.tx * (c101 - c100);
    const float a11 = c110 + w.tx * (c111 - c110);
    const float b0 = a00 + w.ty * (a01 - a00);
    const float b1 = a10 + w.ty * (a11 - a10);
    return b0 + w.tz * (b1 - b0);
  }
  static __device__ __forceinline__ float3 lerp(const float* __restrict__ u, int, const Tri& w) {
    const float4* p = reinterpret_cast<const float4*>(u) + w.base;
    const float4 c000 = __ldg(p), c001 = __ldg(p + w.sx);
    const float4 c010 = __ldg(p + w.sy), c011 = __ldg(p + w.sy + w.sx);
    const float4 c100 = __ldg(p + w.sz), c101 = __ldg(p + w.sz + w.sx);
    const float4 c110 = __ldg(p + w.sz + w.sy), c111 = __ldg(p + w.sz + w.sy + w.sx);
    return make_float3(lerp1(c000.x, c001.x, c010.x, c011.x, c100.x, c101.x, c110.x, c111.x, w),
                       lerp1(c000.y, c001.y, c010.y, c011.y, c100.y, c101.y, c110.y, c111.y, w),
                       lerp1(c000.z, c001.z, c010.z, c011.z, c100.z, c101.z, c110.z, c111.z, w));
  }
};

// RK4 displacement (voxels) of one time step of dy/dt = s v_j(y) / h from the grid point
// (x, y, z), v_j held over the step (the paper's 4th-order Runge-Kutta, §2.4): k1 from the grid
// value (a0, a1, a2), k2, k3, k4 from trilinear lookups of v_j at the stage points;
// c = s dt / h per axis.
template <typename ST>
__device__ __forceinline__ void rk4_disp(const Grid& g, const ST* __restrict__ vj, float x,
                                         float y, float z, float a0, float a1, float a2,
                                         float cx, float cy, float cz, float& d0, float& d1,
                                         float& d2) {
  const float k1x = cx * a0, k1y = cy * a1, k1z = cz * a2;
  Tri w = tri_setup(g, x + 0.5f * k1x, y + 0.5f * k1y, z + 0.5f * k1z);
  const float k2x = cx * tri_apply_t(vj, w), k2y = cy * tri_apply_t(vj + g.N, w),
              k2z = cz * tri_apply_t(vj + 2 * g.N, w);
  w = tri_setup(g, x + 0.5f * k2x, y + 0.5f * k2y, z + 0.5f * k2z);
  const float k3x = cx * tri_apply_t(vj, w), k3y = cy * tri_apply_t(vj + g.N, w),
              k3z = cz * tri_apply_t(vj + 2 * g.N, w);
  w = tri_setup(g, x + k3x, y + k3y, z + k3z);
  const float k4x = cx * tri_apply_t(vj, w), k4y = cy * tri_apply_t(vj + g.N, w),
              k4z = cz * tri_apply_t(vj + 2 * g.N, w);
  d0 = (k1x + 2.f * k2x + 2.f * k3x + k4x) / 6.f;
  d1 = (k1y + 2.f * k2y + 2.f * k3y + k4y) / 6.f;
  d2 = (k1z + 2.f * k2z + 2.f * k3z + k4z) / 6.f;
}

template <typename ST, int SGN, int ZC, bool RK, bool Q>
__global__ void __launch_bounds__(256) k_disp_march(Grid g, const ST* __restrict__ vj,
                                                    const float* __restrict__ uin,
                                                    float* __restrict__ uout, float dtx,
                                                    float dty, float dtz) {
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  const int z0 = blockIdx.z * ZC, z1 = min(z0 + ZC, g.nz);
  const int plane = g.nx * g.ny;
  int idx = (z0 * g.ny + y) * g.nx + x;
  float a0 = ldf(vj + idx), a1 = ldf(vj + g.N + idx), a2 = ldf(vj + 2 * g.N + idx);
  for (int z = z0; z < z1; ++z, idx += plane) {
    float n0 = 0.f, n1 = 0.f, n2 = 0.f;
    if (z + 1 < z1) {
      n0 = ldf_now(vj + idx + plane);
      n1 = ldf_now(vj + g.N + idx + plane);
      n2 = ldf_now(vj + 2 * g.N + idx + plane);
    }
    float dx, dy, dz;
    if (RK) {
      rk4_disp(g, vj, (float)x, (float)y, (float)z, a0, a1, a2, (float)SGN * dtx,
               (float)SGN * dty, (float)SGN * dtz, dx, dy, dz);
    } else {
      dx = (float)SGN * (dtx * a0);
      dy = (float)SGN * (dty * a1);
      dz = (float)SGN * (dtz * a2);
    }
    float ox = dx, oy = dy, oz = dz;
    if (uin) {
      const float3 r = MapL<Q>::lerp(uin, g.N, tri_setup(g, (float)x + dx, (float)y + dy, (float)z + dz));
      ox += r.x;
      oy += r.y;
      oz += r.z;
    }
    MapL<Q>::put(uout, g.N, idx, ox, oy, oz);
    a0 = n0;
    a1 = n1;
    a2 = n2;
  }
}

// Four planes per thread: deep enough to overlap the two latencies, short enough that the grid
// (ceil(nz/4) blocks along z) fills the GPU several times over.
constexpr int kFlowZ = 4;

template <typename ST, int SGN, bool Q>
static void launch_disp_march(const Grid& g, const void* vj, const float* uin, float* uout,
                              float dtx, float dty, float dtz, cudaStream_t s, int rk) {
  const dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, (g.nz + kFlowZ - 1) / kFlowZ);
  if (rk)
    k_disp_march<ST, SGN, kFlowZ, true, Q><<<grid, kBlock3d, 0, s>>>(g, (const ST*)vj, uin, uout,
                                                                     dtx, dty, dtz);
  else
    k_disp_march<ST, SGN, kFlowZ, false, Q><<<grid, kBlock3d, 0, s>>>(g, (const ST*)vj, uin,
                                                                      uout, dtx, dty, dtz);
}

template <bool Q>
static void disp_step_l(int sgn, const Grid& g, const void* vj, const float* uin, float* uout,
                        float dtx, float dty, float dtz, cudaStream_t s, int st, int rk) {
  if (sgn > 0) {
    if (st) launch_disp_march<__nv_bfloat16, 1, Q>(g, vj, uin, uout, dtx, dty, dtz, s, rk);
    else launch_disp_march<float, 1, Q>(g, vj, uin, uout, dtx, dty, dtz, s, rk);
  } else {
    if (st) launch_disp_march<__nv_bfloat16, -1, Q>(g, vj, uin, uout, dtx, dty, dtz, s, rk);
    else launch_disp_march<float, -1, Q>(g, vj, uin, uout, dtx, dty, dtz, s, rk);
  }
}

static void disp_step(int sgn, const Grid& g, const void* vj, const float* uin, float* uout,
                      float dtx, float dty, float dtz, cudaStream_t s, int st, int rk, int quad) {
  if (quad) disp_step_l<true>(sgn, g, vj, uin, uout, dtx, dty, dtz, s, st, rk);
  else disp_step_l<false>(sgn, g, vj, uin, uout, dtx, dty, dtz, s, st, rk);
}

// Backward sweep, part 2: J1_j = I1 o phi_{j,1}, W_j = (M o phi_{j,1}) det D phi_{j,1}.
// I1 and M are read as interleaved pairs (one 8-byte load per trilinear corner for fp32
// storage).  A thread marches ZC planes in z, keeping u at z-1, z, z+1 (and the next plane, in
// flight) in registers: the z-derivative of the map needs no loads, and the lookup position of
// plane z+1 is known before plane z is finished.  The stencil is central inside and one-sided
// at the faces, the trilinear lerps run x, then y, then z: the values equal those of a
// one-voxel-per-thread evaluation.
template <typename ST> struct Pair;
template <> struct Pair<float> { typedef float2 T; };
template <> struct Pair<__nv_bfloat16> { typedef __nv_bfloat162 T; };
__device__ __forceinline__ float2 ldpair(const float2* p) { return __ldg(p); }
__device__ __forceinline__ float2 ldpair(const __nv_bfloat162* p) {
  return __bfloat1622float2(__ldg(p));
}

template <typename PT>
__device__ __forceinline__ float2 tri_apply_pair(const PT* __restrict__ f, const Tri& w) {
  const PT* p = f + w.base;
  const float2 c000 = ldpair(p), c001 = ldpair(p + w.sx);
  const float2 c010 = ldpair(p + w.sy), c011 = ldpair(p + w.sy + w.sx);
  const float2 c100 = ldpair(p + w.sz), c101 = ldpair(p + w.sz + w.sx);
  const float2 c110 = ldpair(p + w.sz + w.sy), c111 = ldpair(p + w.sz + w.sy + w.sx);
  float2 r;
  {
    const float a00 = c000.x + w.tx * (c001.x - c000.x), a01 = c010.x + w.tx * (c011.x - c010.x);
    const float a10 = c100.x + w.tx * (c101.x - c100.x), a11 = c110.x + w.tx * (c111.x - c110.x);
    const float b0 = a00 + w.ty * (a01 - a00), b1 = a10 + w.ty * (a11 - a10);
    r.x = b0 + w.tz * (b1 - b0);
  }
  {
    const float a00 = c000.y + w.tx * (c001.y - c000.y), a01 = c010.y + w.tx * (c011.y - c010.y);
    const float a10 = c100.y + w.tx * (c101.y - c100.y), a11 = c110.y + w.tx * (c111.y - c110.y);
    const float b0 = a00 + w.ty * (a01 - a00), b1 = a10 + w.ty * (a11 - a10);
    r.y = b0 + w.tz * (b1 - b0);
  }
  return r;
}

// At most 40 registers (6 blocks of 256 threads per SM): the march waits on its lookups, and the
// extra warps in flight outweigh the few spilled values (48 registers, 5 blocks: 93 against
// 87 us at 264x160x228; 32 registers spill inside the loop and take 130 us).
template <typename ST, int ZC, bool Q>
__global__ void __launch_bounds__(256, 6) k_back_terms_march(Grid g, const float* __restrict__ uc,
                                                          const typename Pair<ST>::T* __restrict__ IM,
                                                          float* __restrict__ J1j,
                                                          float* __restrict__ Wj, Acc* acc) {
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
  const bool in = x < g.nx && y < g.ny;
  float dmin = 3.0e38f;
  if (in) {
    const int z0 = blockIdx.z * ZC, z1 = min(z0 + ZC, g.nz);
    const int plane = g.nx * g.ny, rowoff = y * g.nx;
    // x and y stencils (central inside, one-sided at the faces)
    const int xlo = x > 0 ? x - 1 : x, xhi = x < g.nx - 1 ? x + 1 : x;
    const int ylo = y > 0 ? y - 1 : y, yhi = y < g.ny - 1 ? y + 1 : y;
    const float ix = (x > 0 && x < g.nx - 1) ? 0.5f : 1.0f;
    const float iy = (y > 0 && y < g.ny - 1) ? 0.5f : 1.0f;
    auto ld3 = [&](int z, float* u) {
      const float3 r = MapL<Q>::at(uc, g.N, z * plane + rowoff + x);
      u[0] = r.x; u[1] = r.y; u[2] = r.z;
    };
    float uP[3], uC[3], uN[3], uNN[3];
    ld3(z0 > 0 ? z0 - 1 : z0, uP);
    ld3(z0, uC);
    ld3(z0 + 1 < g.nz ? z0 + 1 : z0, uN);
    for (int z = z0; z < z1; ++z) {
      // the plane after next, for the z-derivative of plane z + 1
      const int zn = z + 2 < g.nz ? z + 2 : g.nz - 1;
      if (z + 1 < z1) ld3(zn, uNN);
      const int i = z * plane + rowoff + x;
      float D[3][3];
      const float iz = (z > 0 && z < g.nz - 1) ? 0.5f : 1.0f;
      {
        const int zp = z * plane;
        const float3 xh = MapL<Q>::at(uc, g.N, zp + rowoff + xhi);
        const float3 xl = MapL<Q>::at(uc, g.N, zp + rowoff + xlo);
        const float3 yh = MapL<Q>::at(uc, g.N, zp + yhi * g.nx + x);
        const float3 yl = MapL<Q>::at(uc, g.N, zp + ylo * g.nx + x);
        const float xhv[3] = {xh.x, xh.y, xh.z}, xlv[3] = {xl.x, xl.y, xl.z};
        const float yhv[3] = {yh.x, yh.y, yh.z}, ylv[3] = {yl.x, yl.y, yl.z};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          D[d][0] = (xhv[d] - xlv[d]) * ix;
          D[d][1] = (yhv[d] - ylv[d]) * iy;
          const float zh = z < g.nz - 1 ? uN[d] : uC[d], zl = z > 0 ? uP[d] : uC[d];
          D[d][2] = (zh - zl) * iz;
          D[d][d] += 1.0f;
        }
      }
      const float det = D[0][0] * (D[1][1] * D[2][2] - D[1][2] * D[2][1]) -
                        D[0][1] * (D[1][0] * D[2][2] - D[1][2] * D[2][0]) +
                        D[0][2] * (D[1][0] * D[2][1] - D[1][1] * D[2][0]);
      const Tri w = tri_setup(g, (float)x + uC[0], (float)y + uC[1], (float)z + uC[2]);
      const float2 jm = tri_apply_pair(IM, w);
      J1j[i] = jm.x;
      Wj[i] = jm.y * det;
      dmin = fminf(dmin, det);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        uP[d] = uC[d];
        uC[d] = uN[d];
        uN[d] = uNN[d];
      }
    }
  }
  block_min_atomic(dmin, &acc->min_det_ord);
}

template <typename ST>
__global__ void k_interleave(const ST* __restrict__ a, const ST* __restrict__ b,
                             typename Pair<ST>::T* __restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    typename Pair<ST>::T v;
    v.x = a[i];
    v.y = b[i];
    out[i] = v;
  }
}

void launch_interleave(const void* a, const void* b, void* out, int64_t n, cudaStream_t s,
                       int st) {
  const int t = 256;
  const int nb = (int)((n + t - 1) / t);
  if (st)
    k_interleave<<<nb, t, 0, s>>>((const __nv_bfloat16*)a, (const __nv_bfloat16*)b,
                                  (__nv_bfloat162*)out, n);
  else
    k_interleave<<<nb, t, 0, s>>>((const float*)a, (const float*)b, (float2*)out, n);
}

void launch_flow_back(const Grid& g, const void* vj, const float* u_next, float* u_cur,
                      const void* IM, float* J1j, float* Wj, float dtx, float dty, float dtz,
                      Acc* acc, cudaStream_t s, const Hook& hook, int st, int rk) {
  hook(KID_BACK_DISP, 0);
  disp_step(+1, g, vj, u_next, u_cur, dtx, dty, dtz, s, st, rk, 1);
  hook(KID_BACK_DISP, 1);
  hook(KID_BACK_TERMS, 0);
  const dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, (g.nz + kFlowZ - 1) / kFlowZ);
  if (st)
    k_back_terms_march<__nv_bfloat16, kFlowZ, true><<<grid, kBlock3d, 0, s>>>(
        g, u_cur, (const __nv_bfloat162*)IM, J1j, Wj, acc);
  else
    k_back_terms_march<float, kFlowZ, true><<<grid, kBlock3d, 0, s>>>(g, u_cur, (const float2*)IM,
                                                                      J1j, Wj, acc);
  hook(KID_BACK_TERMS, 1);
}

void launch_flow_only_back(const Grid& g, const void* vj, const float* u_next, float* u_cur,
                           float dtx, float dty, float dtz, cudaStream_t s, int st, int rk,
                           int quad) {
  disp_step(+1, g, vj, u_next, u_cur, dtx, dty, dtz, s, st, rk, quad);
}

// --------------------------------------------------------------------------------------------
// Forward sweep, residual: b_j = c W_j (J0_j - J1_j) grad J0_j / h.
// grad J0_j needs J0_j at the stencil neighbours; each is one trilinear lookup of I0 at the
// neighbour's own mapped position (phi_{j,0} is known at every grid point).
template <bool Q, typename ST>
__device__ __forceinline__ float J0_at(const Grid& g, const float* __restrict__ u,
                                       const ST* __restrict__ I0, int idx, int x, int y, int z) {
  const float3 d = MapL<Q>::at(u, g.N, idx);
  return tri_apply_t(I0, tri_setup(g, (float)x + d.x, (float)y + d.y, (float)z + d.z));
}

// b_j at voxel (x, y, z) = idx, as fp32 components (bsplit == 0), or split into bf16 hi/lo
// planes for the pre-split K (bsplit 1: hi plane only, 2: hi and lo): element
// ((comp Z + z) Y + y) px + x of each plane, planes 3 Z Y px elements apart.
template <bool Q, typename ST>
__device__ __forceinline__ void fwd_terms_at(const Grid& g, const float* __restrict__ uc,
                                             const ST* __restrict__ I0,
                                             const float* __restrict__ J1j,
                                             const float* __restrict__ Wj, float* __restrict__ b,
                                             float c, float ihx, float ihy, float ihz, int bsplit,
                                             int px, int x, int y, int z, int idx) {
  const float w = Wj[idx];
  float bx = 0.f, by = 0.f, bz = 0.f;
  if (w != 0.0f) {
    float j0;
    if (uc) j0 = J0_at<Q>(g, uc, I0, idx, x, y, z);
    else j0 = ldf(I0 + idx);
    const float r = c * w * (j0 - J1j[idx]);
    if (r != 0.0f) {
      float gr[3];
      const int n[3] = {g.nx, g.ny, g.nz};
      const int st[3] = {1, g.nx, g.nx * g.ny};
      const int co[3] = {x, y, z};
#pragma unroll
      for (int e = 0; e < 3; ++e) {
        int lo, hi;
        float inv;
        fd_stencil(co[e], n[e], st[e], lo, hi, inv);
        float fh, fl;
        const int dh = hi / st[e], dl = lo / st[e];
        int ph[3] = {x, y, z}, pl[3] = {x, y, z};
        ph[e] += dh;
        pl[e] += dl;
        if (uc) {
          fh = (dh == 0) ? j0 : J0_at<Q>(g, uc, I0, idx + hi, ph[0], ph[1], ph[2]);
          fl = (dl == 0) ? j0 : J0_at<Q>(g, uc, I0, idx + lo, pl[0], pl[1], pl[2]);
        } else {
          fh = ldf(I0 + idx + hi);
          fl = ldf(I0 + idx + lo);
        }
        gr[e] = (fh - fl) * inv;
      }
      bx = r * gr[0] * ihx;
      by = r * gr[1] * ihy;
      bz = r * gr[2] * ihz;
    }
  }
  if (bsplit) {
    __nv_bfloat16* h = reinterpret_cast<__nv_bfloat16*>(b);
    const int64_t cs = (int64_t)g.nz * g.ny * px;
    const int64_t o = ((int64_t)z * g.ny + y) * px + x;
    const float bc[3] = {bx, by, bz};
#pragma unroll
    for (int e = 0; e < 3; ++e) {
      const __nv_bfloat16 hb = __float2bfloat16_rn(bc[e]);
      h[e * cs + o] = hb;
      if (bsplit == 2) h[3 * cs + e * cs + o] = __float2bfloat16_rn(bc[e] - __bfloat162float(hb));
    }
  } else {
    b[idx] = bx;
    b[g.N + idx] = by;
    b[2 * g.N + idx] = bz;
  }
}

// Forward sweep, step j in one pass over u_j = phi_{j,0} - id: the residual b_j (fwd_terms_at)
// and the next map u_{j+1}(x) = -dt v_j(x)/h + u_j(x - dt v_j(x)/h) (as k_disp_march, s = -1;
// uc == nullptr: u_j = 0).  A thread marches ZC planes in z; the velocity of plane z+1 is
// requested before plane z's lookups, and the residual's lookups are independent of the map's.
// J0_T and E_data of the last step come from u_T in a pass of their own (k_j0_edata_march):
// folded in here they doubled this kernel's time for that step.
template <typename ST, int ZC, bool RK, bool Q>
__global__ void __launch_bounds__(256) k_fwd_fused_march(
    Grid g, const ST* __restrict__ vj, const float* __restrict__ uc, float* __restrict__ un,
    float dtx, float dty, float dtz, const ST* __restrict__ I0, const float* __restrict__ J1j,
    const float* __restrict__ Wj, float* __restrict__ b, float c, float ihx, float ihy, float ihz,
    int bsplit, int px) {
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
  if (x < g.nx && y < g.ny) {
    const int z0 = blockIdx.z * ZC, z1 = min(z0 + ZC, g.nz);
    const int plane = g.nx * g.ny;
    int idx = (z0 * g.ny + y) * g.nx + x;
    float a0 = ldf(vj + idx), a1 = ldf(vj + g.N + idx), a2 = ldf(vj + 2 * g.N + idx);
    for (int z = z0; z < z1; ++z, idx += plane) {
      float n0 = 0.f, n1 = 0.f, n2 = 0.f;
      if (z + 1 < z1) {
        n0 = ldf_now(vj + idx + plane);
        n1 = ldf_now(vj + g.N + idx + plane);
        n2 = ldf_now(vj + 2 * g.N + idx + plane);
      }
      float dx, dy, dz;       // the step's displacement (voxels), backward in time
      if (RK) {
        rk4_disp(g, vj, (float)x, (float)y, (float)z, a0, a1, a2, -dtx, -dty, -dtz, dx, dy, dz);
      } else {
        dx = -(dtx * a0);
        dy = -(dty * a1);
        dz = -(dtz * a2);
      }
      float ox = dx, oy = dy, oz = dz;
      if (uc) {
        const float3 r =
            MapL<Q>::lerp(uc, g.N, tri_setup(g, (float)x + dx, (float)y + dy, (float)z + dz));
        ox += r.x;
        oy += r.y;
        oz += r.z;
      }
      fwd_terms_at<Q>(g, uc, I0, J1j, Wj, b, c, ihx, ihy, ihz, bsplit, px, x, y, z, idx);
      MapL<Q>::put(un, g.N, idx, ox, oy, oz);
      a0 = n0;
      a1 = n1;
      a2 = n2;
    }
  }
}

// J0_T = I0 o (id + u_T) and E_data = sum M (J0_T - I1)^2 from the final forward map u_T.
// A thread marches ZC planes in z and requests plane z+1's map before plane z's lookup.
template <typename ST, int ZC, bool Q>
__global__ void __launch_bounds__(256) k_j0_edata_march(Grid g, const float* __restrict__ u,
                                                        const ST* __restrict__ I0,
                                                        const ST* __restrict__ I1,
                                                        const ST* __restrict__ M,
                                                        float* __restrict__ J0T, Acc* acc) {
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
  float edata = 0.f;
  if (x < g.nx && y < g.ny) {
    const int z0 = blockIdx.z * ZC, z1 = min(z0 + ZC, g.nz);
    const int plane = g.nx * g.ny;
    int idx = (z0 * g.ny + y) * g.nx + x;
    float3 d = MapL<Q>::at(u, g.N, idx);
    for (int z = z0; z < z1; ++z, idx += plane) {
      float3 dn = make_float3(0.f, 0.f, 0.f);
      if (z + 1 < z1) dn = MapL<Q>::at(u, g.N, idx + plane);
      const float j0 = tri_apply_t(I0, tri_setup(g, (float)x + d.x, (float)y + d.y, (float)z + d.z));
      J0T[idx] = j0;
      const float r = j0 - ldf(I1 + idx);
      edata = fmaf(ldf(M + idx) * r, r, edata);
      d = dn;
    }
  }
  block_sum_f_atomic(edata, &acc->e_data);
}

// Forward sweep, last step: u_T = -dt v_{T-1}/h + u_cur(x - dt v_{T-1}/h), then J0_T = I0 o
// (id + u_T) and E_data = sum M (J0_T - I1)^2.  Marches ZC planes per thread like k_disp_march
// (the velocity of plane z+1 is loaded before plane z's lookups), so the three dependent
// latencies of a voxel (v, the map at the displaced point, I0 at the mapped point) overlap with
// the next plane's.
template <typename ST, int ZC, bool RK, bool Q>
__global__ void __launch_bounds__(256) k_fwd_last_march(Grid g, const ST* __restrict__ vj,
                                                        const float* __restrict__ uc,
                                                        float* __restrict__ un, float dtx,
                                                        float dty, float dtz,
                                                        const ST* __restrict__ I0,
                                                        const ST* __restrict__ I1,
                                                        const ST* __restrict__ M,
                                                        float* __restrict__ J0T, Acc* acc) {
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
  float edata = 0.f;
  if (x < g.nx && y < g.ny) {
    const int z0 = blockIdx.z * ZC, z1 = min(z0 + ZC, g.nz);
    const int plane = g.nx * g.ny;
    int idx = (z0 * g.ny + y) * g.nx + x;
    float a0 = ldf(vj + idx), a1 = ldf(vj + g.N + idx), a2 = ldf(vj + 2 * g.N + idx);
    for (int z = z0; z < z1; ++z, idx += plane) {
      float n0 = 0.f, n1 = 0.f, n2 = 0.f;
      if (z + 1 < z1) {
        n0 = ldf_now(vj + idx + plane);
        n1 = ldf_now(vj + g.N + idx + plane);
        n2 = ldf_now(vj + 2 * g.N + idx + plane);
      }
      float dx, dy, dz;       // the step's displacement (voxels), backward in time
      if (RK) {
        rk4_disp(g, vj, (float)x, (float)y, (float)z, a0, a1, a2, -dtx, -dty, -dtz, dx, dy, dz);
      } else {
        dx = -(dtx * a0);
        dy = -(dty * a1);
        dz = -(dtz * a2);
      }
      float ox = dx, oy = dy, oz = dz;
      if (uc) {
        const float3 r =
            MapL<Q>::lerp(uc, g.N, tri_setup(g, (float)x + dx, (float)y + dy, (float)z + dz));
        ox += r.x;
        oy += r.y;
        oz += r.z;
      }
      MapL<Q>::put(un, g.N, idx, ox, oy, oz);
      const float j0 = tri_apply_t(I0, tri_setup(g, (float)x + ox, (float)y + oy, (float)z + oz));
      J0T[idx] = j0;
      const float r = j0 - ldf(I1 + idx);
      edata = fmaf(ldf(M + idx) * r, r, edata);
      a0 = n0;
      a1 = n1;
      a2 = n2;
    }
  }
  block_sum_f_atomic(edata, &acc->e_data);
}

void launch_fwd_fused(const Grid& g, const void* vj, const float* u_cur, float* u_next,
                      float dtx, float dty, float dtz, const void* I0, const float* J1j,
                      const float* Wj, float* b, float c, float ihx, float ihy, float ihz,
                      int bsplit, int px, cudaStream_t s, int st, int rk) {
  const dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, (g.nz + kFlowZ - 1) / kFlowZ);
#define FWD_FUSED(ST_, RK_)                                                                    \
  k_fwd_fused_march<ST_, kFlowZ, RK_, false><<<grid, kBlock3d, 0, s>>>(                       \
      g, (const ST_*)vj, u_cur, u_next, dtx, dty, dtz, (const ST_*)I0, J1j, Wj, b, c, ihx, ihy, \
      ihz, bsplit, px)
  if (st) {
    if (rk) FWD_FUSED(__nv_bfloat16, true); else FWD_FUSED(__nv_bfloat16, false);
  } else {
    if (rk) FWD_FUSED(float, true); else FWD_FUSED(float, false);
  }
#undef FWD_FUSED
}

void launch_j0_edata(const Grid& g, const float* u, const void* I0, const void* I1,
                     const void* M, float* J0T, Acc* acc, cudaStream_t s, int st) {
  const dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, (g.nz + kFlowZ - 1) / kFlowZ);
  if (st)
    k_j0_edata_march<__nv_bfloat16, kFlowZ, false><<<grid, kBlock3d, 0, s>>>(
        g, u, (const __nv_bfloat16*)I0, (const __nv_bfloat16*)I1, (const __nv_bfloat16*)M, J0T,
        acc);
  else
    k_j0_edata_march<float, kFlowZ, false><<<grid, kBlock3d, 0, s>>>(
        g, u, (const float*)I0, (const float*)I1, (const float*)M, J0T, acc);
}

void launch_fwd_flow(const Grid& g, const void* vj, const float* u_cur, float* u_next,
                     float dtx, float dty, float dtz, bool last, const void* I0, const void* I1,
                     const void* M, float* J0T, Acc* acc, cudaStream_t s, int st, int rk,
                     int quad) {
  if (!last) {
    disp_step(-1, g, vj, u_cur, u_next, dtx, dty, dtz, s, st, rk, quad);
    return;
  }
  const dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, (g.nz + kFlowZ - 1) / kFlowZ);
#define FWD_LAST(ST_, RK_, Q_)                                                                \
  k_fwd_last_march<ST_, kFlowZ, RK_, Q_><<<grid, kBlock3d, 0, s>>>(                           \
      g, (const ST_*)vj, u_cur, u_next, dtx, dty, dtz, (const ST_*)I0, (const ST_*)I1,       \
      (const ST_*)M, J0T, acc)
  if (quad) {
    if (st) { if (rk) FWD_LAST(__nv_bfloat16, true, true); else FWD_LAST(__nv_bfloat16, false, true); }
    else { if (rk) FWD_LAST(float, true, true); else FWD_LAST(float, false, true); }
  } else {
    if (st) { if (rk) FWD_LAST(__nv_bfloat16, true, false); else FWD_LAST(__nv_bfloat16, false, false); }
    else { if (rk) FWD_LAST(float, true, false); else FWD_LAST(float, false, false); }
  }
#undef FWD_LAST
}

// --------------------------------------------------------------------------------------------
// Regulariser energy of all T velocity fields (the first term of the energy, §2.4):
//   sum_j sum_c sum_x ((gamma - alpha Lap_h) v_{j,c})(x)^2,  Lap_h the periodic 7-point stencil.
// The 3T components are independent scalar fields.  A thread owns VEC consecutive x of one row
// and marches kEregZ planes in z, keeping the planes z-1, z, z+1 of its VEC voxels in registers;
// threads run over the (x/VEC, y) slots of a plane in order, so a warp holds adjacent vectors of
// a row and takes the x-neighbours across vectors from the neighbouring lanes by shuffle (the
// lanes at a warp or row edge load them).  Rows y+-1 are loaded (L1 hits: they are other
// threads' centres).  The loads for plane z+1 are issued before plane z is evaluated.  The
// stencil is ALU work (eight FP32 operations a voxel in the form c0 u + cx (u_x- + u_x+) + ...),
// and the kernel is bound by instruction issue more than by DRAM: the vector width and the
// two-way unrolled march cut the per-voxel instruction count; a field is read once from DRAM.
// Per-plane partial sums are FP32, accumulated with compensated (Kahan) addition per thread; the
// block total goes to FP64.  64 planes per thread (268 -> 262 us against 32 at 264x160x228).
constexpr int kEregZ = 64;

template <int VEC>
__device__ __forceinline__ void ldvec(const float* p, float (&o)[VEC]) {
  if constexpr (VEC == 4) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
  } else {
#pragma unroll
    for (int k = 0; k < VEC; ++k) o[k] = __ldg(p + k);
  }
}
template <int VEC>
__device__ __forceinline__ void ldvec(const __nv_bfloat16* p, float (&o)[VEC]) {
  if constexpr (VEC == 4) {
    const uint2 q = __ldg(reinterpret_cast<const uint2*>(p));
    const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162*>(&q.x);
    const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162*>(&q.y);
    o[0] = __low2float(lo); o[1] = __high2float(lo);
    o[2] = __low2float(hi); o[3] = __high2float(hi);
  } else {
#pragma unroll
    for (int k = 0; k < VEC; ++k) o[k] = ldf(p + k);
  }
}

template <typename ST, int VEC>
__global__ void __launch_bounds__(256) k_ereg(Grid g, const ST* __restrict__ v, int nfield,
                                              float alpha, float gamma, float ihx2, float ihy2,
                                              float ihz2, Acc* acc) {
  const int nxv = g.nx / VEC, slots = nxv * g.ny;
  const int sl = blockIdx.x * 256 + threadIdx.x, lane = threadIdx.x & 31;
  const bool in = sl < slots;
  const int y = in ? sl / nxv : 0, xv = in ? sl - y * nxv : 0, x0 = xv * VEC;
  const int ym = y == 0 ? g.ny - 1 : y - 1, yp = y + 1 == g.ny ? 0 : y + 1;
  const bool lw = lane > 0 && xv > 0;            // lane - 1 holds the vector on the left
  const bool rw = lane < 31 && xv + 1 < nxv;     // lane + 1 holds the vector on the right
  const int xl = x0 == 0 ? g.nx - 1 : x0 - 1, xr = x0 + VEC == g.nx ? 0 : x0 + VEC;
  const int oc = y * g.nx + x0, oym = ym * g.nx + x0, oyp = yp * g.nx + x0;
  const int ol = y * g.nx + xl, orr = y * g.nx + xr;
  const int nzc = (g.nz + kEregZ - 1) / kEregZ;
  const int64_t plane = (int64_t)g.nx * g.ny;
  // (gamma - alpha Lap_h) u = c0 u + cx (u_x- + u_x+) + cy (u_y- + u_y+) + cz (u_z- + u_z+)
  const float c0 = gamma + 2.f * alpha * (ihx2 + ihy2 + ihz2);
  const float cx = -alpha * ihx2, cy = -alpha * ihy2, cz = -alpha * ihz2;
  float sum = 0.f, comp = 0.f;
  for (int q = blockIdx.y; q < nzc * nfield; q += gridDim.y) {
    const int f = q / nzc, z0 = (q - f * nzc) * kEregZ;
    const int z1 = min(z0 + kEregZ, g.nz);
    const ST* fb = v + (int64_t)f * g.N;
    const ST* fe = fb + g.N;
    auto P = [&](int z) -> const ST* {
      z = z < 0 ? z + g.nz : (z >= g.nz ? z - g.nz : z);
      return fb + (int64_t)z * plane;
    };
    float prv[VEC], cur[VEC], nxt[VEC], am[VEC], bp[VEC];
    float hl = 0.f, hr = 0.f;
#pragma unroll
    for (int k = 0; k < VEC; ++k) prv[k] = cur[k] = nxt[k] = am[k] = bp[k] = 0.f;
    const ST* p1 = P(z0 + 1);     // plane z + 1 and plane z + 2, advanced with periodic wrap
    const ST* p2 = P(z0 + 2);
    if (in) {
      ldvec<VEC>(P(z0 - 1) + oc, prv);
      const ST* p0 = P(z0);
      ldvec<VEC>(p0 + oc, cur);
      ldvec<VEC>(p1 + oc, nxt);
      ldvec<VEC>(p0 + oym, am);
      ldvec<VEC>(p0 + oyp, bp);
      if (!lw) hl = ldf(p0 + ol);
      if (!rw) hr = ldf(p0 + orr);
    }
    // unrolled by two, so the shift of the plane window costs no moves
#pragma unroll 2
    for (int z = z0; z < z1; ++z) {
      // loads for the next plane: centre of z + 2, neighbours of z + 1
      float nn[VEC], am2[VEC], bp2[VEC];
      float hl2 = 0.f, hr2 = 0.f;
      if (in && z + 1 < z1) {
        ldvec<VEC>(p2 + oc, nn);
        ldvec<VEC>(p1 + oym, am2);
        ldvec<VEC>(p1 + oyp, bp2);
        if (!lw) hl2 = ldf(p1 + ol);
        if (!rw) hr2 = ldf(p1 + orr);
      } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) nn[k] = am2[k] = bp2[k] = 0.f;
      }
      p1 = p2;
      p2 += plane;
      if (p2 >= fe) p2 -= g.N;
      const float fromL = __shfl_up_sync(0xffffffffu, cur[VEC - 1], 1);
      const float fromR = __shfl_down_sync(0xffffffffu, cur[0], 1);
      if (in) {
        float e = 0.f;
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
          const float l = k > 0 ? cur[k - 1] : (lw ? fromL : hl);
          const float r = k + 1 < VEC ? cur[k + 1] : (rw ? fromR : hr);
          const float Lv =
              fmaf(cz, prv[k] + nxt[k], fmaf(cy, am[k] + bp[k], fmaf(cx, l + r, c0 * cur[k])));
          e = fmaf(Lv, Lv, e);
        }
        const float yk = e - comp;
        const float tt = sum + yk;
        comp = (tt - sum) - yk;
        sum = tt;
      }
#pragma unroll
      for (int k = 0; k < VEC; ++k) {
        prv[k] = cur[k];
        cur[k] = nxt[k];
        nxt[k] = nn[k];
        am[k] = am2[k];
        bp[k] = bp2[k];
      }
      hl = hl2;
      hr = hr2;
    }
  }
  block_sum_f_atomic(sum, &acc->e_reg);
}

void launch_ereg(const Grid& g, const void* v, int T, float alpha, float gamma, float ihx2,
                 float ihy2, float ihz2, Acc* acc, cudaStream_t s, int st) {
  // 4-wide vectors when every row starts on a vector boundary (the field bases are then aligned
  // too: N is a multiple of nx and the buffer comes from cudaMalloc)
  const bool v4 = g.nx % 4 == 0 && ((uintptr_t)v % 16) == 0;
  const int vec = v4 ? 4 : 1;
  const int64_t slots = (int64_t)(g.nx / vec) * g.ny;
  const int nzc = (g.nz + kEregZ - 1) / kEregZ;
  const int64_t nq = (int64_t)nzc * 3 * T;
  const dim3 grid((unsigned)((slots + 255) / 256), (unsigned)(nq < 65535 ? nq : 65535));
  if (st) {
    const __nv_bfloat16* p = (const __nv_bfloat16*)v;
    if (v4) k_ereg<__nv_bfloat16, 4><<<grid, 256, 0, s>>>(g, p, 3 * T, alpha, gamma, ihx2, ihy2, ihz2, acc);
    else k_ereg<__nv_bfloat16, 1><<<grid, 256, 0, s>>>(g, p, 3 * T, alpha, gamma, ihx2, ihy2, ihz2, acc);
  } else {
    const float* p = (const float*)v;
    if (v4) k_ereg<float, 4><<<grid, 256, 0, s>>>(g, p, 3 * T, alpha, gamma, ihx2, ihy2, ihz2, acc);
    else k_ereg<float, 1><<<grid, 256, 0, s>>>(g, p, 3 * T, alpha, gamma, ihx2, ihy2, ihz2, acc);
  }
}

void launch_flow_only_fwd(const Grid& g, const void* vj, const float* u_cur, float* u_next,
                          float dtx, float dty, float dtz, cudaStream_t s, int st, int rk,
                          int quad) {
  disp_step(-1, g, vj, u_cur, u_next, dtx, dty, dtz, s, st, rk, quad);
}

// quad map [N] x (x, y, z, 0) -> planar [3][N]
__global__ void k_quad_to_planar(const float4* __restrict__ q, float* __restrict__ p, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const float4 v = __ldg(q + i);
    p[i] = v.x;
    p[n + i] = v.y;
    p[2 * n + i] = v.z;
  }
}

void launch_quad_to_planar(const float* quad, float* planar, int64_t n, cudaStream_t s) {
  if (n > 0)
    k_quad_to_planar<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
        reinterpret_cast<const float4*>(quad), planar, n);
}

// --------------------------------------------------------------------------------------------
// Update: v_j <- v_j - eps (2 v_j - K b_j) over the 3 components (float4 streaming).
__global__ void k_update(int n4, int n, float4* __restrict__ v, const float4* __restrict__ kb,
                         float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n4) {
    float4 a = v[i];
    const float4 k = kb[i];
    a.x -= eps * (2.f * a.x - k.x);
    a.y -= eps * (2.f * a.y - k.y);
    a.z -= eps * (2.f * a.z - k.z);
    a.w -= eps * (2.f * a.w - k.w);
    v[i] = a;
  }
  // scalar tail (n not a multiple of 4)
  if (i == 0) {
    float* vs = reinterpret_cast<float*>(v);
    const float* ks = reinterpret_cast<const float*>(kb);
    for (int t = n4 * 4; t < n; ++t) vs[t] -= eps * (2.f * vs[t] - ks[t]);
  }
}

template <typename ST>
__global__ void k_update_scalar(int n, ST* __restrict__ v, const float* __restrict__ kb,
                                float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const float a = ldf(v + i);
    stf(v + i, a - eps * (2.f * a - kb[i]));
  }
}

void launch_update(const Grid& g, void* vj, const float* Kb, float eps, cudaStream_t s, int st) {
  const int n = 3 * g.N;
  const int t = 256;
  if (st) {
    k_update_scalar<<<nblocks(n, t), t, 0, s>>>(n, (__nv_bfloat16*)vj, Kb, eps);
    return;
  }
  // float4 streaming when both fields start on a 16-byte boundary (v_j does not when 3N is odd
  // and j is odd), scalar otherwise.
  if (((uintptr_t)vj & 15) == 0 && ((uintptr_t)Kb & 15) == 0) {
    const int n4 = n / 4;
    k_update<<<nblocks(n4 > 0 ? n4 : 1, t), t, 0, s>>>(n4, n, reinterpret_cast<float4*>(vj),
                                                       reinterpret_cast<const float4*>(Kb), eps);
  } else {
    k_update_scalar<<<nblocks(n, t), t, 0, s>>>(n, (float*)vj, Kb, eps);
  }
}

// --------------------------------------------------------------------------------------------
// Warp (trilinear pull-back) and label transfer (nearest neighbour, float32 rounding rule).
__global__ void k_warp(Grid g, const float* __restrict__ src, const float* __restrict__ u,
                       float* __restrict__ dst) {
  int x, y, z, idx;
  if (!voxel3d(g, x, y, z, idx)) return;
  dst[idx] = tri_sample(src, g, (float)x + u[idx], (float)y + u[g.N + idx], (float)z + u[2 * g.N + idx]);
}

void launch_warp(const Grid& g, const float* src, const float* u, float* dst, cudaStream_t s) {
  k_warp<<<grid3d(g), kBlock3d, 0, s>>>(g, src, u, dst);
}

__device__ __forceinline__ int nn_index(float i, float u, int n) {
  // (i + u) is rounded to float32, then + 0.5 rounded to float32, then floor: no contraction.
  const float p = __fadd_rn(__fadd_rn(i, u), 0.5f);
  int k = (int)floorf(p);
  return min(max(k, 0), n - 1);
}

__global__ void k_labels(Grid g, const uint16_t* __restrict__ L0, const float* __restrict__ u,
                         uint16_t* __restrict__ dst) {
  int x, y, z, idx;
  if (!voxel3d(g, x, y, z, idx)) return;
  const int ix = nn_index((float)x, u[idx], g.nx);
  const int iy = nn_index((float)y, u[g.N + idx], g.ny);
  const int iz = nn_index((float)z, u[2 * g.N + idx], g.nz);
  dst[idx] = L0[(iz * g.ny + iy) * g.nx + ix];
}

void launch_labels(const Grid& g, const uint16_t* L0, const float* u, uint16_t* dst,
                   cudaStream_t s) {
  k_labels<<<grid3d(g), kBlock3d, 0, s>>>(g, L0, u, dst);
}

// --------------------------------------------------------------------------------------------
// Multiscale: block mean with edge replication; trilinear cell-centred upsampling.
template <typename DT>
__global__ void k_downsample(Grid f, Grid c, int factor, const float* __restrict__ src,
                             DT* __restrict__ dst) {
  int x, y, z, idx;
  if (!voxel3d(c, x, y, z, idx)) return;
  double s = 0.0;
  for (int dz = 0; dz < factor; ++dz) {
    const int zz = min(z * factor + dz, f.nz - 1);
    for (int dy = 0; dy < factor; ++dy) {
      const int yy = min(y * factor + dy, f.ny - 1);
      for (int dx = 0; dx < factor; ++dx) {
        const int xx = min(x * factor + dx, f.nx - 1);
        s += (double)src[(zz * f.ny + yy) * f.nx + xx];
      }
    }
  }
  stf(dst + idx, (float)(s / (double)(factor * factor * factor)));
}

void launch_downsample(const Grid& fine, const Grid& coarse, int factor, const float* src,
                       void* dst, cudaStream_t s, int st) {
  if (st) k_downsample<<<grid3d(coarse), kBlock3d, 0, s>>>(fine, coarse, factor, src, (__nv_bfloat16*)dst);
  else k_downsample<<<grid3d(coarse), kBlock3d, 0, s>>>(fine, coarse, factor, src, (float*)dst);
}

template <typename ST>
__global__ void k_upsample(Grid c, Grid f, float ratio, const ST* __restrict__ src,
                           ST* __restrict__ dst, int nfields) {
  int x, y, z, idx;
  if (!voxel3d(f, x, y, z, idx)) return;
  Tri w = tri_setup(c, ((float)x + 0.5f) * ratio - 0.5f, ((float)y + 0.5f) * ratio - 0.5f,
                    ((float)z + 0.5f) * ratio - 0.5f);
  for (int k = 0; k < nfields; ++k)
    stf(dst + (int64_t)k * f.N + idx, tri_apply_t(src + (int64_t)k * c.N, w));
}

void launch_upsample(const Grid& coarse, const Grid& fine, float ratio, const void* src,
                     void* dst, int nfields, cudaStream_t s, int st) {
  if (st)
    k_upsample<<<grid3d(fine), kBlock3d, 0, s>>>(coarse, fine, ratio, (const __nv_bfloat16*)src,
                                                 (__nv_bfloat16*)dst, nfields);
  else
    k_upsample<<<grid3d(fine), kBlock3d, 0, s>>>(coarse, fine, ratio, (const float*)src,
                                                 (float*)dst, nfields);
}

// --------------------------------------------------------------------------------------------
// Storage conversion (fp32 <-> bf16, round to nearest) for the precision form.
__global__ void k_to_bf16(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) b[i] = __float2bfloat16_rn(a[i]);
}
__global__ void k_to_f32(const __nv_bfloat16* __restrict__ a, float* __restrict__ b, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) b[i] = __bfloat162float(a[i]);
}

void launch_to_storage(const float* src, void* dst, int64_t n, cudaStream_t s, int st) {
  if (n <= 0) return;
  if (st) k_to_bf16<<<152 * 8, 256, 0, s>>>(src, (__nv_bfloat16*)dst, n);
  else cudaMemcpyAsync(dst, src, n * sizeof(float), cudaMemcpyDeviceToDevice, s);
}

void launch_from_storage(const void* src, float* dst, int64_t n, cudaStream_t s, int st) {
  if (n <= 0) return;
  if (st) k_to_f32<<<152 * 8, 256, 0, s>>>((const __nv_bfloat16*)src, dst, n);
  else cudaMemcpyAsync(dst, src, n * sizeof(float), cudaMemcpyDeviceToDevice, s);
}

// --------------------------------------------------------------------------------------------
__global__ void k_check_finite(const float* __restrict__ a, int64_t n, int* flag, int bit) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int bad = 0;
  for (; i < n; i += stride) bad |= !isfinite(a[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, bit);
}

void launch_check_finite(const float* a, int64_t n, int* flag, cudaStream_t s, int bit) {
  if (n <= 0) return;
  k_check_finite<<<152 * 8, 256, 0, s>>>(a, n, flag, bit);
}

__global__ void k_fill(float* a, int64_t n, float value) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) a[i] = value;
}

void launch_fill(float* a, int64_t n, float value, cudaStream_t s) {
  if (n <= 0) return;
  k_fill<<<152 * 8, 256, 0, s>>>(a, n, value);
}

__global__ void k_dice_hist(const uint16_t* __restrict__ A, const uint16_t* __restrict__ B,
                            int64_t n, unsigned long long* hist) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) {
    const unsigned a = A[i], b = B[i];
    if (a) atomicAdd(&hist[a], 1ull);
    if (b) atomicAdd(&hist[65536 + b], 1ull);
    if (a && a == b) atomicAdd(&hist[2 * 65536 + a], 1ull);
  }
}

void launch_dice_hist(const uint16_t* A, const uint16_t* B, int64_t n, unsigned long long* hist,
                      cudaStream_t s) {
  if (n <= 0) return;
  k_dice_hist<<<152 * 8, 256, 0, s>>>(A, B, n, hist);
}

}  // namespace lddmm
