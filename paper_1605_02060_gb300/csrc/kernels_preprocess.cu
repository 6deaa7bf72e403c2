// Preprocessing of §2.2 on the GPU.
//
// Image-LDDMM: the masks are applied to I0 and I1, and the masked I0 is histogram-matched to the
// masked I1.  Both images get a `bins`-bin histogram of their in-mask voxels over [min, max];
// `points` quantiles at k / (points + 1) are read off the cumulative counts (interpolated inside
// the bin that reaches the fraction); min maps to min, max to max, each quantile of I0 to the
// same quantile of I1, linearly in between and along the end segments beyond.
//
// Mask generation: [I > threshold], opened with a ball of radius r_open (erosion, then
// dilation), then closed with a ball of radius r_close (dilation, then erosion); voxels beyond
// the grid count as background.
//
// The histogram counts are integers (exact), and every floating-point step of the quantiles and
// of the map is FP64 with explicitly rounded operations, in the order of the definition above.
#include "kernels.h"

namespace lddmm {

namespace {

__device__ __forceinline__ int ord_of(float f) {
  const int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7fffffff;
}
__device__ __forceinline__ float float_of(int i) {
  return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff);
}

// st[0] = min, st[1] = max (ordered ints), st[2] = count (as int) of voxels with M > 0.5.
__global__ void k_masked_range(const float* __restrict__ I, const float* __restrict__ M,
                               int64_t n, int* st) {
  int mn = 0x7fffffff, mx = (int)0x80000000, c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (M[i] > 0.5f) {
      const int o = ord_of(I[i]);
      mn = min(mn, o);
      mx = max(mx, o);
      ++c;
    }
  }
  for (int o = 16; o; o >>= 1) {
    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(st, mn);
    atomicMax(st + 1, mx);
    atomicAdd(st + 2, c);
  }
}

__device__ __forceinline__ int bin_of(double v, double lo, double w, int bins) {
  if (w <= 0.0) return 0;
  const int b = (int)floor(__ddiv_rn(__dsub_rn(v, lo), w));
  return min(max(b, 0), bins - 1);
}

__global__ void k_masked_hist(const float* __restrict__ I, const float* __restrict__ M, int64_t n,
                              const int* st, int bins, unsigned long long* counts) {
  extern __shared__ unsigned int sh[];
  for (int b = threadIdx.x; b < bins; b += blockDim.x) sh[b] = 0;
  __syncthreads();
  const double lo = float_of(st[0]), hi = float_of(st[1]);
  const double w = __ddiv_rn(__dsub_rn(hi, lo), (double)bins);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (M[i] > 0.5f) atomicAdd(&sh[bin_of((double)I[i], lo, w, bins)], 1u);
  __syncthreads();
  for (int b = threadIdx.x; b < bins; b += blockDim.x)
    if (sh[b]) atomicAdd(&counts[b], (unsigned long long)sh[b]);
}

__device__ double quantile(const unsigned long long* c, int bins, double lo, double hi, double n,
                           double f) {
  const double w = __ddiv_rn(__dsub_rn(hi, lo), (double)bins);
  if (w <= 0.0) return lo;
  const double t = __dmul_rn(f, n);
  double C = 0.0, prev = 0.0;
  int k = bins - 1;
  for (int b = 0; b < bins; ++b) {
    prev = C;
    C = __dadd_rn(C, (double)c[b]);
    if (C >= t) {
      k = b;
      break;
    }
  }
  if (k == bins - 1 && C < t) {            // not reached (rounding): the last bin
    prev = __dsub_rn(C, (double)c[bins - 1]);
  }
  if (c[k] == 0) return __dadd_rn(lo, __dmul_rn(w, (double)k));
  return __dadd_rn(lo, __dmul_rn(w, __dadd_rn((double)k, __ddiv_rn(__dsub_rn(t, prev), (double)c[k]))));
}

// nodes[0..P+1] = x (source), nodes[P+2..2P+3] = y (reference), P = points.
__global__ void k_match_nodes(const int* st0, const unsigned long long* c0, const int* st1,
                              const unsigned long long* c1, int bins, int points, double* nodes) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double lo0 = float_of(st0[0]), hi0 = float_of(st0[1]), n0 = (double)st0[2];
  const double lo1 = float_of(st1[0]), hi1 = float_of(st1[1]), n1 = (double)st1[2];
  const int m = points + 2;
  nodes[0] = lo0;
  nodes[m] = lo1;
  for (int k = 1; k <= points; ++k) {
    const double f = __ddiv_rn((double)k, (double)(points + 1));
    nodes[k] = quantile(c0, bins, lo0, hi0, n0, f);
    nodes[m + k] = quantile(c1, bins, lo1, hi1, n1, f);
  }
  nodes[m - 1] = hi0;
  nodes[2 * m - 1] = hi1;
}

__global__ void k_apply_match(const float* __restrict__ I0, const float* __restrict__ M0,
                              int64_t n, const double* __restrict__ nodes, int m,
                              float* __restrict__ out) {
  __shared__ double xs[66], ys[66];
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    xs[k] = nodes[k];
    ys[k] = nodes[m + k];
  }
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (!(M0[i] > 0.5f)) {
      out[i] = 0.f;
      continue;
    }
    const double v = (double)I0[i];
    int k = 0;                                // last node with x <= v, kept inside [0, m-2]
    for (int j = 1; j < m - 1; ++j)
      if (xs[j] <= v) k = j;
    const double dx = __dsub_rn(xs[k + 1], xs[k]);
    const double slope = dx > 0.0 ? __ddiv_rn(__dsub_rn(ys[k + 1], ys[k]), dx) : 0.0;
    out[i] = (float)__dadd_rn(ys[k], __dmul_rn(__dsub_rn(v, xs[k]), slope));
  }
}

__global__ void k_threshold(const float* __restrict__ I, int64_t n, float t, uint8_t* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = I[i] > t ? 1 : 0;
}

// ERODE: 1 where every ball offset lands on a 1 inside the grid; dilate: 1 where any does.
template <bool ERODE>
__global__ void k_ball_op(Grid g, const uint8_t* __restrict__ in, int r, uint8_t* __restrict__ out) {
  const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y, z = blockIdx.z;
  if (x >= g.nx || y >= g.ny) return;
  const int64_t idx = ((int64_t)z * g.ny + y) * g.nx + x;
  bool res = ERODE;
  for (int dz = -r; dz <= r && res == ERODE; ++dz)
    for (int dy = -r; dy <= r && res == ERODE; ++dy)
      for (int dx = -r; dx <= r; ++dx) {
        if (dx * dx + dy * dy + dz * dz > r * r) continue;
        const int xx = x + dx, yy = y + dy, zz = z + dz;
        const bool inside = xx >= 0 && xx < g.nx && yy >= 0 && yy < g.ny && zz >= 0 && zz < g.nz;
        const bool v = inside && in[((int64_t)zz * g.ny + yy) * g.nx + xx];
        if (ERODE && !v) { res = false; break; }
        if (!ERODE && v) { res = true; break; }
      }
  out[idx] = res ? 1 : 0;
}

int grid_1d(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

}  // namespace

cudaError_t masked_range(const float* I, const float* M, int64_t n, int* st, cudaStream_t s) {
  const int init[3] = {0x7fffffff, (int)0x80000000, 0};
  cudaError_t e = cudaMemcpyAsync(st, init, sizeof(init), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  k_masked_range<<<grid_1d(n), 256, 0, s>>>(I, M, n, st);
  return cudaGetLastError();
}

cudaError_t masked_hist(const float* I, const float* M, int64_t n, const int* st, int bins,
                        unsigned long long* counts, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(counts, 0, (size_t)bins * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  k_masked_hist<<<grid_1d(n), 256, (size_t)bins * sizeof(unsigned int), s>>>(I, M, n, st, bins, counts);
  return cudaGetLastError();
}

cudaError_t match_nodes(const int* st0, const unsigned long long* c0, const int* st1,
                        const unsigned long long* c1, int bins, int points, double* nodes,
                        cudaStream_t s) {
  k_match_nodes<<<1, 32, 0, s>>>(st0, c0, st1, c1, bins, points, nodes);
  return cudaGetLastError();
}

cudaError_t apply_match(const float* I0, const float* M0, int64_t n, const double* nodes,
                        int points, float* out, cudaStream_t s) {
  k_apply_match<<<grid_1d(n), 256, 0, s>>>(I0, M0, n, nodes, points + 2, out);
  return cudaGetLastError();
}

cudaError_t threshold_mask(const float* I, int64_t n, float t, uint8_t* out, cudaStream_t s) {
  k_threshold<<<grid_1d(n), 256, 0, s>>>(I, n, t, out);
  return cudaGetLastError();
}

cudaError_t ball_op(const Grid& g, const uint8_t* in, int r, bool erode, uint8_t* out,
                    cudaStream_t s) {
  const dim3 grid((g.nx + 31) / 32, (g.ny + 7) / 8, g.nz);
  if (erode) k_ball_op<true><<<grid, dim3(32, 8, 1), 0, s>>>(g, in, r, out);
  else k_ball_op<false><<<grid, dim3(32, 8, 1), 0, s>>>(g, in, r, out);
  return cudaGetLastError();
}

}  // namespace lddmm
