// Geodesic shooting (EPDiff): the momentum m_0 = L^T L v_0 transported by the flow,
//     m_t(x) = |D phi(x)| (D phi(x))^T m_0(phi(x)),   phi = phi_{t,0} = id + u,
// the solution of d m / dt = -ad*_v m for LDDMM's metric (Beg et al. 2005, cited in §2.4);
// v_t = K m_t follows with the registration's smoothing operator.  m_0 o phi is a trilinear
// lookup (clamp to edge); D phi is taken by central differences inside and one-sided at the
// faces, in physical units: (D phi)_ik = (h_i / h_k) d phi_i / d x_k in voxel coordinates.
#include "kernels.h"

namespace lddmm {

namespace {

__global__ void k_transport_momentum(Grid g, const float* __restrict__ m0,
                                     const float* __restrict__ u, float hx, float hy, float hz,
                                     float* __restrict__ m) {
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y, z = blockIdx.z;
  if (x >= g.nx || y >= g.ny) return;
  const int idx = (z * g.ny + y) * g.nx + x;
  const float ux = u[idx], uy = u[g.N + idx], uz = u[2 * g.N + idx];
  const Tri w = tri_setup(g, (float)x + ux, (float)y + uy, (float)z + uz);
  const float mm[3] = {tri_apply(m0, w), tri_apply(m0 + g.N, w), tri_apply(m0 + 2 * g.N, w)};
  // J[i][k] = d phi_i / d x_k (voxel coordinates), then scaled by h_i / h_k
  const int n[3] = {g.nx, g.ny, g.nz};
  const int st[3] = {1, g.nx, g.nx * g.ny};
  const int co[3] = {x, y, z};
  const float h[3] = {hx, hy, hz};
  float J[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    int lo, hi;
    float inv;
    fd_stencil(co[k], n[k], st[k], lo, hi, inv);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float* ui = u + i * g.N + idx;
      J[i][k] = ((__ldg(ui + hi) - __ldg(ui + lo)) * inv + (i == k ? 1.f : 0.f)) * (h[i] / h[k]);
    }
  }
  const float det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                    J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                    J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
#pragma unroll
  for (int k = 0; k < 3; ++k)
    m[k * g.N + idx] = det * (J[0][k] * mm[0] + J[1][k] * mm[1] + J[2][k] * mm[2]);
}

}  // namespace

cudaError_t transport_momentum(const Grid& g, const float* m0, const float* u, float hx,
                               float hy, float hz, float* m, cudaStream_t s) {
  const dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
  k_transport_momentum<<<grid, dim3(32, 8, 1), 0, s>>>(g, m0, u, hx, hy, hz, m);
  return cudaGetLastError();
}

}  // namespace lddmm
