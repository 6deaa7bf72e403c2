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
// Backward sweep, part 1: displacement of phi_{j,1}.
template <typename ST>
__global__ void k_back_disp(Grid g, const ST* __restrict__ vj, const float* __restrict__ un,
                            float* __restrict__ uc, float dtx, float dty, float dtz) {
  int x, y, z, idx;
  if (!voxel3d(g, x, y, z, idx)) return;
  const float dx = dtx * ldf(vj + idx), dy = dty * ldf(vj + g.N + idx),
              dz = dtz * ldf(vj + 2 * g.N + idx);
  float ox = dx, oy = dy, oz = dz;
  if (un) {
    Tri w = tri_setup(g, (float)x + dx, (float)y + dy, (float)z + dz);
    ox += tri_apply(un, w);
    oy += tri_apply(un + g.N, w);
    oz += tri_apply(un + 2 * g.N, w);
  }
  uc[idx] = ox;
  uc[g.N + idx] = oy;
  uc[2 * g.N + idx] = oz;
}

// det(I + Du) at voxel (x,y,z) with the one-sided/central stencil.
__device__ __forceinline__ float jac_det(const Grid& g, const float* __restrict__ u, int idx,
                                         int x, int y, int z) {
  int lo[3], hi[3];
  float inv[3];
  fd_stencil(x, g.nx, 1, lo[0], hi[0], inv[0]);
  fd_stencil(y, g.ny, g.nx, lo[1], hi[1], inv[1]);
  fd_stencil(z, g.nz, g.nx * g.ny, lo[2], hi[2], inv[2]);
  float D[3][3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float* ud = u + d * g.N + idx;
#pragma unroll
    for (int e = 0; e < 3; ++e) D[d][e] = (__ldg(ud + hi[e]) - __ldg(ud + lo[e])) * inv[e];
    D[d][d] += 1.0f;
  }
  return D[0][0] * (D[1][1] * D[2][2] - D[1][2] * D[2][1]) -
         D[0][1] * (D[1][0] * D[2][2] - D[1][2] * D[2][0]) +
         D[0][2] * (D[1][0] * D[2][1] - D[1][1] * D[2][0]);
}

// Backward sweep, part 2: J1_j = I1 o phi_{j,1}, W_j = (M o phi_{j,1}) det D phi_{j,1}.
template <typename ST>
__global__ void k_back_terms(Grid g, const float* __restrict__ uc, const ST* __restrict__ I1,
                             const ST* __restrict__ M, float* __restrict__ J1j,
                             float* __restrict__ Wj, Acc* acc) {
  int x, y, z, idx;
  const bool in = voxel3d(g, x, y, z, idx);
  float dmin = 3.0e38f;
  if (in) {
    const float det = jac_det(g, uc, idx, x, y, z);
    Tri w = tri_setup(g, (float)x + uc[idx], (float)y + uc[g.N + idx], (float)z + uc[2 * g.N + idx]);
    J1j[idx] = tri_apply_t(I1, w);
    Wj[idx] = tri_apply_t(M, w) * det;
    dmin = det;
  }
  block_min_atomic(dmin, &acc->min_det_ord);
}

void launch_flow_back(const Grid& g, const void* vj, const float* u_next, float* u_cur,
                      const void* I1, const void* M, float* J1j, float* Wj, float dtx,
                      float dty, float dtz, Acc* acc, cudaStream_t s, const Hook& hook, int st) {
  hook(KID_BACK_DISP, 0);
  if (st) k_back_disp<<<grid3d(g), kBlock3d, 0, s>>>(g, (const __nv_bfloat16*)vj, u_next, u_cur, dtx, dty, dtz);
  else k_back_disp<<<grid3d(g), kBlock3d, 0, s>>>(g, (const float*)vj, u_next, u_cur, dtx, dty, dtz);
  hook(KID_BACK_DISP, 1);
  hook(KID_BACK_TERMS, 0);
  if (st)
    k_back_terms<<<grid3d(g), kBlock3d, 0, s>>>(g, u_cur, (const __nv_bfloat16*)I1,
                                                (const __nv_bfloat16*)M, J1j, Wj, acc);
  else
    k_back_terms<<<grid3d(g), kBlock3d, 0, s>>>(g, u_cur, (const float*)I1, (const float*)M, J1j,
                                                Wj, acc);
  hook(KID_BACK_TERMS, 1);
}

void launch_flow_only_back(const Grid& g, const void* vj, const float* u_next, float* u_cur,
                           float dtx, float dty, float dtz, cudaStream_t s, int st) {
  if (st) k_back_disp<<<grid3d(g), kBlock3d, 0, s>>>(g, (const __nv_bfloat16*)vj, u_next, u_cur, dtx, dty, dtz);
  else k_back_disp<<<grid3d(g), kBlock3d, 0, s>>>(g, (const float*)vj, u_next, u_cur, dtx, dty, dtz);
}

// --------------------------------------------------------------------------------------------
// Forward sweep, residual: b_j = c W_j (J0_j - J1_j) grad J0_j / h.
// grad J0_j needs J0_j at the stencil neighbours; each is one trilinear lookup of I0 at the
// neighbour's own mapped position (phi_{j,0} is known at every grid point).
template <typename ST>
__device__ __forceinline__ float J0_at(const Grid& g, const float* __restrict__ u,
                                       const ST* __restrict__ I0, int idx, int x, int y, int z) {
  return tri_apply_t(I0, tri_setup(g, (float)x + __ldg(u + idx), (float)y + __ldg(u + g.N + idx),
                                   (float)z + __ldg(u + 2 * g.N + idx)));
}

template <typename ST>
__global__ void k_fwd_terms(Grid g, const float* __restrict__ uc, const ST* __restrict__ I0,
                            const float* __restrict__ J1j, const float* __restrict__ Wj,
                            float* __restrict__ b, float c, float ihx, float ihy, float ihz) {
  int x, y, z, idx;
  if (!voxel3d(g, x, y, z, idx)) return;
  const float w = Wj[idx];
  float bx = 0.f, by = 0.f, bz = 0.f;
  if (w != 0.0f) {
    float j0;
    if (uc) j0 = J0_at(g, uc, I0, idx, x, y, z);
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
          fh = (dh == 0) ? j0 : J0_at(g, uc, I0, idx + hi, ph[0], ph[1], ph[2]);
          fl = (dl == 0) ? j0 : J0_at(g, uc, I0, idx + lo, pl[0], pl[1], pl[2]);
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
  b[idx] = bx;
  b[g.N + idx] = by;
  b[2 * g.N + idx] = bz;
}

void launch_fwd_terms(const Grid& g, const float* u_cur, const void* I0, const float* J1j,
                      const float* Wj, float* b, float c, float ihx, float ihy, float ihz,
                      cudaStream_t s, int st) {
  if (st)
    k_fwd_terms<<<grid3d(g), kBlock3d, 0, s>>>(g, u_cur, (const __nv_bfloat16*)I0, J1j, Wj, b, c,
                                               ihx, ihy, ihz);
  else
    k_fwd_terms<<<grid3d(g), kBlock3d, 0, s>>>(g, u_cur, (const float*)I0, J1j, Wj, b, c, ihx, ihy,
                                               ihz);
}

// Forward sweep, flow: u_next = -dt v_j/h + u_cur(x - dt v_j/h); E_reg of v_j (periodic
// 7-point (gamma - alpha Lap_h) v_j, summed over components); at the last step J0_T and E_data.
template <typename ST>
__global__ void k_fwd_flow(Grid g, const ST* __restrict__ vj, const float* __restrict__ uc,
                           float* __restrict__ un, float dtx, float dty, float dtz, float alpha,
                           float gamma, float ihx2, float ihy2, float ihz2, int last,
                           const ST* __restrict__ I0, const ST* __restrict__ I1,
                           const ST* __restrict__ M, float* __restrict__ J0T, Acc* acc) {
  int x, y, z, idx;
  const bool in = voxel3d(g, x, y, z, idx);
  float ereg = 0.f, edata = 0.f;
  if (in) {
    const float v0 = ldf(vj + idx), v1 = ldf(vj + g.N + idx), v2 = ldf(vj + 2 * g.N + idx);
    const float dx = dtx * v0, dy = dty * v1, dz = dtz * v2;
    float ox = -dx, oy = -dy, oz = -dz;
    if (uc) {
      Tri w = tri_setup(g, (float)x - dx, (float)y - dy, (float)z - dz);
      ox += tri_apply(uc, w);
      oy += tri_apply(uc + g.N, w);
      oz += tri_apply(uc + 2 * g.N, w);
    }
    un[idx] = ox;
    un[g.N + idx] = oy;
    un[2 * g.N + idx] = oz;
    // regulariser: periodic neighbours
    const int xm = (x == 0 ? g.nx - 1 : -1), xp = (x == g.nx - 1 ? -(g.nx - 1) : 1);
    const int sy = g.nx, sz = g.nx * g.ny;
    const int ym = (y == 0 ? (g.ny - 1) * sy : -sy), yp = (y == g.ny - 1 ? -(g.ny - 1) * sy : sy);
    const int zm = (z == 0 ? (g.nz - 1) * sz : -sz), zp = (z == g.nz - 1 ? -(g.nz - 1) * sz : sz);
    const float vc[3] = {v0, v1, v2};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const ST* p = vj + c * g.N + idx;
      const float lap = (ldf(p + xm) - 2.f * vc[c] + ldf(p + xp)) * ihx2 +
                        (ldf(p + ym) - 2.f * vc[c] + ldf(p + yp)) * ihy2 +
                        (ldf(p + zm) - 2.f * vc[c] + ldf(p + zp)) * ihz2;
      const float Lv = gamma * vc[c] - alpha * lap;
      ereg = fmaf(Lv, Lv, ereg);
    }
    if (last) {
      const float j0 = tri_apply_t(I0, tri_setup(g, (float)x + ox, (float)y + oy, (float)z + oz));
      J0T[idx] = j0;
      const float r = j0 - ldf(I1 + idx);
      edata = ldf(M + idx) * r * r;
    }
  }
  block_sum_f_atomic(ereg, &acc->e_reg);
  if (last) {
    __syncthreads();
    block_sum_f_atomic(edata, &acc->e_data);
  }
}

void launch_fwd_flow(const Grid& g, const void* vj, const float* u_cur, float* u_next,
                     float dtx, float dty, float dtz, float alpha, float gamma, float ihx2,
                     float ihy2, float ihz2, bool last, const void* I0, const void* I1,
                     const void* M, float* J0T, Acc* acc, cudaStream_t s, int st) {
  if (st)
    k_fwd_flow<<<grid3d(g), kBlock3d, 0, s>>>(
        g, (const __nv_bfloat16*)vj, u_cur, u_next, dtx, dty, dtz, alpha, gamma, ihx2, ihy2, ihz2,
        last ? 1 : 0, (const __nv_bfloat16*)I0, (const __nv_bfloat16*)I1, (const __nv_bfloat16*)M,
        J0T, acc);
  else
    k_fwd_flow<<<grid3d(g), kBlock3d, 0, s>>>(g, (const float*)vj, u_cur, u_next, dtx, dty, dtz,
                                              alpha, gamma, ihx2, ihy2, ihz2, last ? 1 : 0,
                                              (const float*)I0, (const float*)I1,
                                              (const float*)M, J0T, acc);
}

template <typename ST>
__global__ void k_fwd_disp(Grid g, const ST* __restrict__ vj, const float* __restrict__ uc,
                           float* __restrict__ un, float dtx, float dty, float dtz) {
  int x, y, z, idx;
  if (!voxel3d(g, x, y, z, idx)) return;
  const float dx = dtx * ldf(vj + idx), dy = dty * ldf(vj + g.N + idx),
              dz = dtz * ldf(vj + 2 * g.N + idx);
  float ox = -dx, oy = -dy, oz = -dz;
  if (uc) {
    Tri w = tri_setup(g, (float)x - dx, (float)y - dy, (float)z - dz);
    ox += tri_apply(uc, w);
    oy += tri_apply(uc + g.N, w);
    oz += tri_apply(uc + 2 * g.N, w);
  }
  un[idx] = ox;
  un[g.N + idx] = oy;
  un[2 * g.N + idx] = oz;
}

void launch_flow_only_fwd(const Grid& g, const void* vj, const float* u_cur, float* u_next,
                          float dtx, float dty, float dtz, cudaStream_t s, int st) {
  if (st) k_fwd_disp<<<grid3d(g), kBlock3d, 0, s>>>(g, (const __nv_bfloat16*)vj, u_cur, u_next, dtx, dty, dtz);
  else k_fwd_disp<<<grid3d(g), kBlock3d, 0, s>>>(g, (const float*)vj, u_cur, u_next, dtx, dty, dtz);
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
__global__ void k_check_finite(const float* __restrict__ a, int64_t n, int* flag) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int bad = 0;
  for (; i < n; i += stride) bad |= !isfinite(a[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

void launch_check_finite(const float* a, int64_t n, int* flag, cudaStream_t s) {
  if (n <= 0) return;
  k_check_finite<<<152 * 8, 256, 0, s>>>(a, n, flag);
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
