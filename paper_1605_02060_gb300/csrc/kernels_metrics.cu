// Registration-quality measures of §2.7 on the GPU:
//   Hausdorff distance  d_H = max{ sup_{x in S(1)} inf_{y in S1} d(x, y), sup_{y in S1} inf_{x in S(1)} d(x, y) }
//   median distance     d_M = median of the union of both sets of directed distances
//   landmark error      e_k = | phi(x_k) - y_k |
// S(1) and S1 are the surfaces of two binary masks: mask voxels with a face neighbour outside
// the mask (a neighbour beyond the grid counts as outside).  d is the Euclidean distance between
// voxel centres in physical units.
//
// The directed distances are found by brute force over the surface lists: every surface voxel
// compares itself with every voxel of the other surface, the other list staged through shared
// memory in tiles.  A brain-sized mask at 264x160x228 has ~1e5 surface voxels, so the search is
// ~1e10 distance evaluations in FP32; the winner's distance is then recomputed in FP64.  The
// median and the maximum come from one block that bisects on the bit patterns of the (non-
// negative) FP64 distances, so no sort and no host round trip is needed.
#include "kernels.h"

namespace lddmm {

namespace {

__global__ void k_surface_list(Grid g, const uint8_t* __restrict__ m, int4* __restrict__ list,
                               unsigned* count, unsigned cap) {
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y, z = blockIdx.z;
  if (x >= g.nx || y >= g.ny) return;
  const int64_t idx = ((int64_t)z * g.ny + y) * g.nx + x;
  if (!m[idx]) return;
  const int64_t sy = g.nx, sz = (int64_t)g.nx * g.ny;
  const bool s = x == 0 || x == g.nx - 1 || y == 0 || y == g.ny - 1 || z == 0 || z == g.nz - 1 ||
                 !m[idx - 1] || !m[idx + 1] || !m[idx - sy] || !m[idx + sy] || !m[idx - sz] ||
                 !m[idx + sz];
  if (s) {
    const unsigned k = atomicAdd(count, 1u);
    if (k < cap) list[k] = make_int4(x, y, z, 0);
  }
}

constexpr int kTile = 1024;

// d[i] = distance from src[i] to the nearest point of dst (physical units, FP64).
__global__ void __launch_bounds__(256) k_nearest(const int4* __restrict__ src, unsigned ns,
                                                 const int4* __restrict__ dst, unsigned nd,
                                                 float hx, float hy, float hz,
                                                 double* __restrict__ d) {
  __shared__ int4 tile[kTile];
  const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  const int4 p = i < ns ? src[i] : make_int4(0, 0, 0, 0);
  float best = 3.0e38f;
  unsigned bj = 0;
  for (unsigned t0 = 0; t0 < nd; t0 += kTile) {
    const unsigned nt = min((unsigned)kTile, nd - t0);
    __syncthreads();
    for (unsigned k = threadIdx.x; k < nt; k += blockDim.x) tile[k] = dst[t0 + k];
    __syncthreads();
    for (unsigned k = 0; k < nt; ++k) {
      const int4 q = tile[k];
      const float dx = (float)(p.x - q.x) * hx, dy = (float)(p.y - q.y) * hy,
                  dz = (float)(p.z - q.z) * hz;
      const float d2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      if (d2 < best) {
        best = d2;
        bj = t0 + k;
      }
    }
  }
  if (i < ns) {
    const int4 q = dst[bj];
    const double dx = (double)(p.x - q.x) * hx, dy = (double)(p.y - q.y) * hy,
                 dz = (double)(p.z - q.z) * hz;
    d[i] = sqrt(dx * dx + dy * dy + dz * dz);
  }
}

// One block: out[0] = max, out[1] = k1-th and out[2] = k2-th smallest of d[0..n) (0-based).
// Non-negative doubles order like their bit patterns, so each order statistic is the smallest
// bit pattern b with #{d <= b} > k, found by 64 halvings of the bit range.
__global__ void __launch_bounds__(1024) k_order_stats(const double* __restrict__ d, unsigned n,
                                                      unsigned k1, unsigned k2, double* out) {
  __shared__ unsigned long long red[32];
  __shared__ unsigned long long bcast;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // maximum (as bits)
  unsigned long long mx = 0;
  for (unsigned i = tid; i < n; i += blockDim.x)
    mx = max(mx, (unsigned long long)__double_as_longlong(d[i]));
  for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) red[wid] = mx;
  __syncthreads();
  if (tid == 0) {
    unsigned long long m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, red[w]);
    bcast = m;
  }
  __syncthreads();
  const unsigned long long top = bcast;
  if (tid == 0) out[0] = __longlong_as_double((long long)top);
  const unsigned ks[2] = {k1, k2};
  for (int s = 0; s < 2; ++s) {
    unsigned long long lo = 0, hi = top;          // answer in [lo, hi]
    while (lo < hi) {
      const unsigned long long mid = lo + (hi - lo) / 2;
      unsigned long long c = 0;
      for (unsigned i = tid; i < n; i += blockDim.x)
        c += (unsigned long long)__double_as_longlong(d[i]) <= mid ? 1ull : 0ull;
      for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
      __syncthreads();
      if (lane == 0) red[wid] = c;
      __syncthreads();
      if (tid == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        bcast = t;
      }
      __syncthreads();
      if (bcast > ks[s]) hi = mid;
      else lo = mid + 1;
    }
    if (tid == 0) out[1 + s] = __longlong_as_double((long long)lo);
  }
}

// e_k = |(x_k + u01(x_k) - y_k) h| with u01 (3 components of N, voxel units) interpolated
// trilinearly with clamp-to-edge coordinates.
__global__ void k_landmarks(Grid g, const float* __restrict__ u01, const float* __restrict__ xk,
                            const float* __restrict__ yk, int n, float hx, float hy, float hz,
                            double* __restrict__ e) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float x = xk[3 * k], y = xk[3 * k + 1], z = xk[3 * k + 2];
  const Tri w = tri_setup(g, x, y, z);
  const double px = (double)x + tri_apply(u01, w), py = (double)y + tri_apply(u01 + g.N, w),
               pz = (double)z + tri_apply(u01 + 2 * g.N, w);
  const double dx = (px - yk[3 * k]) * hx, dy = (py - yk[3 * k + 1]) * hy,
               dz = (pz - yk[3 * k + 2]) * hz;
  e[k] = sqrt(dx * dx + dy * dy + dz * dz);
}

}  // namespace

cudaError_t surface_list(const Grid& g, const uint8_t* m, int4* list, unsigned* count,
                         unsigned cap, cudaStream_t s) {
  const dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
  k_surface_list<<<grid, dim3(32, 8, 1), 0, s>>>(g, m, list, count, cap);
  return cudaGetLastError();
}

cudaError_t nearest_distances(const int4* src, unsigned ns, const int4* dst, unsigned nd,
                              float hx, float hy, float hz, double* d, cudaStream_t s) {
  if (ns == 0) return cudaSuccess;
  k_nearest<<<(ns + 255) / 256, 256, 0, s>>>(src, ns, dst, nd, hx, hy, hz, d);
  return cudaGetLastError();
}

cudaError_t order_stats(const double* d, unsigned n, unsigned k1, unsigned k2, double* out,
                        cudaStream_t s) {
  k_order_stats<<<1, 1024, 0, s>>>(d, n, k1, k2, out);
  return cudaGetLastError();
}

cudaError_t landmark_errors(const Grid& g, const float* u01, const float* xk, const float* yk,
                            int n, float hx, float hy, float hz, double* e, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_landmarks<<<(n + 127) / 128, 128, 0, s>>>(g, u01, xk, yk, n, hx, hy, hz, e);
  return cudaGetLastError();
}

}  // namespace lddmm
