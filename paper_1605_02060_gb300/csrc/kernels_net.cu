// Kernels of the learned warm start: a small 3D convolutional encoder-decoder that maps a
// template/target mask pair to an initial velocity field, trained and evaluated entirely here.
//
// Layout: activations [B][C][n][n][n] float32 (x fastest); weights [Co][Ci][k^3] (k = 3 or 1)
// stored bf16 for the forward and data-gradient products (FP32 master copy for the optimiser),
// all products accumulated in FP32.  3x3x3 convolutions use zero padding 1.
//
//   conv_fwd   y[b,co,v] = bias[co] + sum_ci sum_t w[co,ci,t] x[b,ci,v+o(t)]   (+ ReLU)
//   conv_dgrad dx[b,ci,v] = sum_co sum_t w[co,ci,t] dy[b,co,v-o(t)]  (= conv_fwd with the
//              transposed, flipped kernel, since o(26-t) = -o(t))
//   conv_wgrad dw[co,ci,t] += sum_b sum_v dy[b,co,v] x[b,ci,v+o(t)],  db[co] += sum dy[b,co,v]
//              (fixed-order partial sums in caller scratch: the same bits on every run)
// plus 2x average pooling, 2x nearest upsampling, channel concatenation, ReLU backward, the MSE
// loss and Adam.  Convolutions whose input channels come in groups of 16 run on the tensor cores
// (kernels_conv_tc.cu); the others (the 2-channel network input, the 3-channel head gradient)
// here: 8x8x4 output voxels x 16 output channels per block, input channels staged 8 at a time
// with a one-voxel halo in shared memory.
#include <cuda_bf16.h>

#include "kernels.h"

namespace lddmm {

namespace {

constexpr int BX = 8, BY = 8, BZ = 4, NTV = BX * BY * BZ;   // 256 voxels per block
constexpr int CT = 16;                                      // output channels per block
constexpr int CC = 8;                                       // input channels per stage
constexpr int HXn = BX + 2, HYn = BY + 2, HZn = BZ + 2, HV = HXn * HYn * HZn;

__device__ __forceinline__ float xval(const float* __restrict__ x, int n, int gx, int gy, int gz) {
  return (gx >= 0 && gx < n && gy >= 0 && gy < n && gz >= 0 && gz < n)
             ? __ldg(x + ((size_t)gz * n + gy) * n + gx)
             : 0.f;
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// Forward convolution (also the data gradient with transposed weights).
// grid: (tiles of 8x8x4, ceil(Co/16), B); block: 256 threads, one output voxel each.
__global__ void __launch_bounds__(NTV) k_conv_fwd(const float* __restrict__ x,
                                                  const __nv_bfloat16* __restrict__ w,
                                                  const float* __restrict__ bias,
                                                  float* __restrict__ y, int Ci, int Co, int n,
                                                  int ks, int relu, int accumulate) {
  __shared__ float xs[CC][HV];
  __shared__ __align__(16) float ws[CC][27][CT];
  const int tid = threadIdx.x;
  const int ntx = (n + BX - 1) / BX, nty = (n + BY - 1) / BY;
  const int tile = blockIdx.x;
  const int tx0 = (tile % ntx) * BX, ty0 = ((tile / ntx) % nty) * BY, tz0 = (tile / (ntx * nty)) * BZ;
  const int co0 = blockIdx.y * CT, b = blockIdx.z;
  const int lx = tid % BX, ly = (tid / BX) % BY, lz = tid / (BX * BY);
  const int gx = tx0 + lx, gy = ty0 + ly, gz = tz0 + lz;
  const size_t nv = (size_t)n * n * n;
  const int taps = ks * ks * ks, pad = ks / 2;
  float acc[CT];
#pragma unroll
  for (int c = 0; c < CT; ++c) acc[c] = 0.f;
  for (int ci0 = 0; ci0 < Ci; ci0 += CC) {
    const int cc = min(CC, Ci - ci0);
    // input tile (with halo) for cc channels
    for (int i = tid; i < cc * HV; i += NTV) {
      const int c = i / HV, h = i % HV;
      const int hx = h % HXn, hy = (h / HXn) % HYn, hz = h / (HXn * HYn);
      xs[c][h] = xval(x + ((size_t)b * Ci + ci0 + c) * nv, n, tx0 + hx - 1, ty0 + hy - 1, tz0 + hz - 1);
    }
    // weights [c][t][co] as float
    for (int i = tid; i < cc * taps * CT; i += NTV) {
      const int co = i % CT, t = (i / CT) % taps, c = i / (CT * taps);
      const int gco = co0 + co;
      ws[c][t][co] = gco < Co ? __bfloat162float(w[((size_t)gco * Ci + ci0 + c) * taps + t]) : 0.f;
    }
    __syncthreads();
    for (int c = 0; c < cc; ++c) {
      for (int t = 0; t < taps; ++t) {
        int ox, oy, oz;
        if (ks == 3) { ox = t % 3 - 1; oy = (t / 3) % 3 - 1; oz = t / 9 - 1; }
        else { ox = oy = oz = 0; }
        const float xv = xs[c][((lz + 1 + oz) * HYn + (ly + 1 + oy)) * HXn + (lx + 1 + ox)];
        const float4* w4 = reinterpret_cast<const float4*>(&ws[c][t][0]);
#pragma unroll
        for (int q = 0; q < CT / 4; ++q) {
          const float4 wv = w4[q];
          acc[4 * q] = fmaf(wv.x, xv, acc[4 * q]);
          acc[4 * q + 1] = fmaf(wv.y, xv, acc[4 * q + 1]);
          acc[4 * q + 2] = fmaf(wv.z, xv, acc[4 * q + 2]);
          acc[4 * q + 3] = fmaf(wv.w, xv, acc[4 * q + 3]);
        }
      }
    }
    __syncthreads();
  }
  (void)pad;
  if (gx < n && gy < n && gz < n) {
    const size_t v = ((size_t)gz * n + gy) * n + gx;
#pragma unroll
    for (int c = 0; c < CT; ++c) {
      const int co = co0 + c;
      if (co >= Co) break;
      float r = acc[c] + (bias ? bias[co] : 0.f);
      float* o = y + ((size_t)b * Co + co) * nv + v;
      if (accumulate) r += *o;
      if (relu) r = fmaxf(r, 0.f);
      *o = r;
    }
  }
}

// wT[ci][co][t'] = w[co][ci][taps-1-t'] (bf16): the data-gradient kernel in forward form.
__global__ void k_transpose_flip(const __nv_bfloat16* __restrict__ w, __nv_bfloat16* __restrict__ wT,
                                 int Ci, int Co, int taps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Ci * Co * taps) return;
  const int t = i % taps, co = (i / taps) % Co, ci = i / (taps * Co);
  wT[i] = w[((size_t)co * Ci + ci) * taps + (taps - 1 - t)];
}

// Weight gradient, deterministic: block (g, ci * co-tile) sums, in a fixed order, the
// (batch, tile) units g, g + G, g + 2G, ... into one partial per (output channel, tap), written
// to part[g][co][ci][t]; k_wgrad_reduce then adds the G partials of every weight in order g = 0..G-1.
// No floating-point atomics, so the result is the same on every run.
__global__ void __launch_bounds__(512) k_conv_wgrad(const float* __restrict__ x,
                                                    const float* __restrict__ dy,
                                                    float* __restrict__ part, int B, int Ci, int Co,
                                                    int n, int ks, int G) {
  __shared__ float xs[HV];
  __shared__ float dys[CT][NTV];
  const int tid = threadIdx.x;
  const int ntx = (n + BX - 1) / BX, nty = (n + BY - 1) / BY, ntz = (n + BZ - 1) / BZ;
  const int tiles = ntx * nty * ntz;
  const int g = blockIdx.x;
  const int ci = blockIdx.y % Ci, cot = blockIdx.y / Ci;
  const int co0 = cot * CT;
  const size_t nv = (size_t)n * n * n;
  const int taps = ks * ks * ks;
  const int c = tid / taps, t = tid % taps;
  int ox = 0, oy = 0, oz = 0;
  if (ks == 3) { ox = t % 3 - 1; oy = (t / 3) % 3 - 1; oz = t / 9 - 1; }
  float s = 0.f;
  for (int u = g; u < tiles * B; u += G) {
    const int b = u / tiles, tile = u % tiles;
    const int tx0 = (tile % ntx) * BX, ty0 = ((tile / ntx) % nty) * BY, tz0 = (tile / (ntx * nty)) * BZ;
    for (int i = tid; i < HV; i += blockDim.x) {
      const int hx = i % HXn, hy = (i / HXn) % HYn, hz = i / (HXn * HYn);
      xs[i] = xval(x + ((size_t)b * Ci + ci) * nv, n, tx0 + hx - 1, ty0 + hy - 1, tz0 + hz - 1);
    }
    for (int i = tid; i < CT * NTV; i += blockDim.x) {
      const int cc = i / NTV, vv = i % NTV;
      const int lx = vv % BX, ly = (vv / BX) % BY, lz = vv / (BX * BY);
      const int gx = tx0 + lx, gy = ty0 + ly, gz = tz0 + lz;
      const int co = co0 + cc;
      dys[cc][vv] = (co < Co && gx < n && gy < n && gz < n)
                        ? dy[((size_t)b * Co + co) * nv + ((size_t)gz * n + gy) * n + gx]
                        : 0.f;
    }
    __syncthreads();
    if (tid < CT * taps) {
      for (int vv = 0; vv < NTV; ++vv) {
        const int lx = vv % BX, ly = (vv / BX) % BY, lz = vv / (BX * BY);
        s = fmaf(dys[c][vv], xs[((lz + 1 + oz) * HYn + (ly + 1 + oy)) * HXn + (lx + 1 + ox)], s);
      }
    }
    __syncthreads();
  }
  if (tid < CT * taps && co0 + c < Co)
    part[(size_t)g * Co * Ci * taps + ((size_t)(co0 + c) * Ci + ci) * taps + t] = s;
}

// dw[i] += sum_{g = 0..G-1} part[g][i], in that order.
__global__ void k_wgrad_reduce(const float* __restrict__ part, float* __restrict__ dw, int64_t count,
                               int G) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (; i < count; i += st) {
    float s = 0.f;
    for (int g = 0; g < G; ++g) s += part[(size_t)g * count + i];
    dw[i] += s;
  }
}

// Bias gradient, deterministic: block (co, g) sums the fixed chunk g of the B * n^3 values of
// channel co (tree reduction of fixed shape) into partb[co][g]; k_bias_reduce adds them in order.
__global__ void k_bias_partial(const float* __restrict__ dy, float* __restrict__ partb, int B, int Co,
                               int n, int GB) {
  const int co = blockIdx.x, g = blockIdx.y;
  const size_t nv = (size_t)n * n * n;
  const size_t total = (size_t)B * nv, chunk = (total + GB - 1) / GB;
  const size_t lo = (size_t)g * chunk, hi = lo + chunk < total ? lo + chunk : total;
  float s = 0.f;
  for (size_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    const size_t b = i / nv, v = i % nv;
    s += dy[(b * Co + co) * nv + v];
  }
  __shared__ float red[32];
  s = warp_sum_f(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    float t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    t = warp_sum_f(t);
    if (threadIdx.x == 0) partb[(size_t)co * GB + g] = t;
  }
}

__global__ void k_bias_reduce(const float* __restrict__ partb, float* __restrict__ db, int Co, int GB) {
  const int co = blockIdx.x * blockDim.x + threadIdx.x;
  if (co >= Co) return;
  float s = 0.f;
  for (int g = 0; g < GB; ++g) s += partb[(size_t)co * GB + g];
  db[co] += s;
}

// ---------------------------------------------------------------------------------------------
// elementwise and resampling kernels (n = size of the finer grid where it matters)
__global__ void k_relu_bwd(float* __restrict__ dy, const float* __restrict__ y, int64_t count) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (; i < count; i += st)
    if (y[i] <= 0.f) dy[i] = 0.f;
}

// avg pool 2x: x [BC][n^3] -> y [BC][(n/2)^3]
__global__ void k_pool_fwd(const float* __restrict__ x, float* __restrict__ y, int64_t BC, int n) {
  const int m = n / 2;
  const int64_t total = BC * m * m * m;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (; i < total; i += st) {
    const int X = i % m, Y = (i / m) % m, Z = (i / ((int64_t)m * m)) % m;
    const int64_t c = i / ((int64_t)m * m * m);
    const float* p = x + c * n * n * n;
    float s = 0.f;
    for (int dz = 0; dz < 2; ++dz)
      for (int dyy = 0; dyy < 2; ++dyy)
        for (int dx = 0; dx < 2; ++dx) s += p[((int64_t)(2 * Z + dz) * n + 2 * Y + dyy) * n + 2 * X + dx];
    y[i] = 0.125f * s;
  }
}

// dx[fine] = dy[coarse] / 8
__global__ void k_pool_bwd(const float* __restrict__ dy, float* __restrict__ dx, int64_t BC, int n) {
  const int m = n / 2;
  const int64_t total = BC * n * n * n;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (; i < total; i += st) {
    const int X = i % n, Y = (i / n) % n, Z = (i / ((int64_t)n * n)) % n;
    const int64_t c = i / ((int64_t)n * n * n);
    dx[i] = 0.125f * dy[c * m * m * m + ((int64_t)(Z / 2) * m + Y / 2) * m + X / 2];
  }
}

// nearest upsample 2x: x [B][C][m^3] -> y[b][coff + c][n^3] inside a buffer of Cy channels
__global__ void k_up_fwd(const float* __restrict__ x, float* __restrict__ y, int B, int C, int m,
                         int Cy, int coff) {
  const int n = 2 * m;
  const int64_t total = (int64_t)B * C * n * n * n;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (; i < total; i += st) {
    const int X = i % n, Y = (i / n) % n, Z = (i / ((int64_t)n * n)) % n;
    const int64_t bc = i / ((int64_t)n * n * n);
    const int c = (int)(bc % C), b = (int)(bc / C);
    y[((int64_t)b * Cy + coff + c) * n * n * n + ((int64_t)Z * n + Y) * n + X] =
        x[bc * m * m * m + ((int64_t)(Z / 2) * m + Y / 2) * m + X / 2];
  }
}

// dx[b][c][m^3] = sum of the 8 children of dy[b][coff + c][n^3] (Cy channels in dy)
__global__ void k_up_bwd(const float* __restrict__ dy, float* __restrict__ dx, int B, int C, int m,
                         int Cy, int coff) {
  const int n = 2 * m;
  const int64_t total = (int64_t)B * C * m * m * m;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (; i < total; i += st) {
    const int X = i % m, Y = (i / m) % m, Z = (i / ((int64_t)m * m)) % m;
    const int64_t bc = i / ((int64_t)m * m * m);
    const int c = (int)(bc % C), b = (int)(bc / C);
    const float* p = dy + ((int64_t)b * Cy + coff + c) * n * n * n;
    float s = 0.f;
    for (int dz = 0; dz < 2; ++dz)
      for (int dyy = 0; dyy < 2; ++dyy)
        for (int dx2 = 0; dx2 < 2; ++dx2) s += p[((int64_t)(2 * Z + dz) * n + 2 * Y + dyy) * n + 2 * X + dx2];
    dx[i] = s;
  }
}

// copy channels: dst[b][doff + c][v] = src[b][soff + c][v] for c < C (accumulate optional)
__global__ void k_copy_ch(const float* __restrict__ src, float* __restrict__ dst, int B, int C,
                          int64_t nv, int Cs, int soff, int Cd, int doff, int accumulate) {
  const int64_t total = (int64_t)B * C * nv;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (; i < total; i += st) {
    const int64_t v = i % nv;
    const int64_t bc = i / nv;
    const int c = (int)(bc % C), b = (int)(bc / C);
    const float s = src[((int64_t)b * Cs + soff + c) * nv + v];
    float* d = dst + ((int64_t)b * Cd + doff + c) * nv + v;
    *d = accumulate ? *d + s : s;
  }
}

// MSE: loss = mean (p - t)^2 (FP64 sum); grad = 2 (p - t) / count
__global__ void k_mse(const float* __restrict__ p, const float* __restrict__ t, float* __restrict__ g,
                      int64_t count, double* loss) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  float s = 0.f;
  const float sc = 2.f / (float)count;
  for (; i < count; i += st) {
    const float d = p[i] - t[i];
    s = fmaf(d, d, s);
    if (g) g[i] = sc * d;
  }
  block_sum_f_atomic(s, loss);
}

// Adam on FP32 master weights, with the bf16 copy used by the products refreshed in place.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, __nv_bfloat16* __restrict__ wb, int64_t count,
                       float lr, float b1, float b2, float eps, float c1, float c2) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (; i < count; i += st) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16_rn(wi);
  }
}

__global__ void k_cast_bf16(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, int64_t count) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t st = (int64_t)gridDim.x * blockDim.x;
  for (; i < count; i += st) b[i] = __float2bfloat16_rn(a[i]);
}

// ---------------------------------------------------------------------------------------------
static inline int gs(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

static int tiles_of(int n) { return ((n + BX - 1) / BX) * ((n + BY - 1) / BY) * ((n + BZ - 1) / BZ); }

bool conv_tc_supported(int Ci, int Co);
cudaError_t conv_tc_fwd(const float* x, const void* w, const float* bias, float* y, int B, int Ci,
                        int Co, int n, int ks, int relu, int accumulate, cudaStream_t s);

cudaError_t net_conv_fwd(const float* x, const void* w, const float* bias, float* y, int B, int Ci,
                         int Co, int n, int ks, int relu, int accumulate, cudaStream_t s) {
  // input channels in groups of 16: the tensor-core implicit GEMM (kernels_conv_tc.cu)
  if (conv_tc_supported(Ci, Co))
    return conv_tc_fwd(x, w, bias, y, B, Ci, Co, n, ks, relu, accumulate, s);
  dim3 grid(tiles_of(n), (Co + CT - 1) / CT, B);
  k_conv_fwd<<<grid, NTV, 0, s>>>(x, (const __nv_bfloat16*)w, bias, y, Ci, Co, n, ks, relu,
                                  accumulate);
  return cudaGetLastError();
}

cudaError_t net_conv_dgrad(const float* dy, const void* w, void* wT_scratch, float* dx, int B,
                           int Ci, int Co, int n, int ks, cudaStream_t s) {
  const int taps = ks * ks * ks;
  const int cnt = Ci * Co * taps;
  k_transpose_flip<<<(cnt + 255) / 256, 256, 0, s>>>((const __nv_bfloat16*)w,
                                                     (__nv_bfloat16*)wT_scratch, Ci, Co, taps);
  return net_conv_fwd(dy, wT_scratch, nullptr, dx, B, Co, Ci, n, ks, 0, 0, s);
}

// Partition of the weight-gradient sums: G voxel groups (about 2048 blocks in all, at most one
// group per (batch, tile) unit), GB chunks per bias channel.
static void wgrad_groups(int B, int Ci, int Co, int n, int* G, int* GB) {
  const int units = tiles_of(n) * B;
  const int cb = Ci * ((Co + CT - 1) / CT);
  int g = (2048 + cb - 1) / cb;
  *G = g < 1 ? 1 : (g > units ? units : g);
  const int64_t total = (int64_t)B * n * n * n;
  int64_t gb = (total + 8191) / 8192;
  *GB = (int)(gb < 1 ? 1 : (gb > 64 ? 64 : gb));
}

int64_t net_conv_wgrad_scratch(int B, int Ci, int Co, int n, int ks) {
  int G, GB;
  wgrad_groups(B, Ci, Co, n, &G, &GB);
  return (int64_t)G * Co * Ci * ks * ks * ks + (int64_t)Co * GB;
}

cudaError_t net_conv_wgrad(const float* x, const float* dy, float* dw, float* db, float* scratch,
                           int B, int Ci, int Co, int n, int ks, cudaStream_t s) {
  int G, GB;
  wgrad_groups(B, Ci, Co, n, &G, &GB);
  const int64_t count = (int64_t)Co * Ci * ks * ks * ks;
  dim3 grid(G, Ci * ((Co + CT - 1) / CT));
  k_conv_wgrad<<<grid, 512, 0, s>>>(x, dy, scratch, B, Ci, Co, n, ks, G);
  k_wgrad_reduce<<<gs(count), 256, 0, s>>>(scratch, dw, count, G);
  if (db) {
    float* partb = scratch + (size_t)G * count;
    k_bias_partial<<<dim3(Co, GB), 256, 0, s>>>(dy, partb, B, Co, n, GB);
    k_bias_reduce<<<(Co + 127) / 128, 128, 0, s>>>(partb, db, Co, GB);
  }
  return cudaGetLastError();
}

cudaError_t net_relu_bwd(float* dy, const float* y, int64_t count, cudaStream_t s) {
  k_relu_bwd<<<gs(count), 256, 0, s>>>(dy, y, count);
  return cudaGetLastError();
}
cudaError_t net_pool_fwd(const float* x, float* y, int64_t BC, int n, cudaStream_t s) {
  k_pool_fwd<<<gs(BC * n * n * n / 8), 256, 0, s>>>(x, y, BC, n);
  return cudaGetLastError();
}
cudaError_t net_pool_bwd(const float* dy, float* dx, int64_t BC, int n, cudaStream_t s) {
  k_pool_bwd<<<gs(BC * n * n * n), 256, 0, s>>>(dy, dx, BC, n);
  return cudaGetLastError();
}
cudaError_t net_up_fwd(const float* x, float* y, int B, int C, int m, int Cy, int coff,
                       cudaStream_t s) {
  k_up_fwd<<<gs((int64_t)B * C * 8 * m * m * m), 256, 0, s>>>(x, y, B, C, m, Cy, coff);
  return cudaGetLastError();
}
cudaError_t net_up_bwd(const float* dy, float* dx, int B, int C, int m, int Cy, int coff,
                       cudaStream_t s) {
  k_up_bwd<<<gs((int64_t)B * C * m * m * m), 256, 0, s>>>(dy, dx, B, C, m, Cy, coff);
  return cudaGetLastError();
}
cudaError_t net_copy_ch(const float* src, float* dst, int B, int C, int64_t nv, int Cs, int soff,
                        int Cd, int doff, int accumulate, cudaStream_t s) {
  k_copy_ch<<<gs((int64_t)B * C * nv), 256, 0, s>>>(src, dst, B, C, nv, Cs, soff, Cd, doff,
                                                    accumulate);
  return cudaGetLastError();
}
cudaError_t net_mse(const float* p, const float* t, float* g, int64_t count, double* loss,
                    cudaStream_t s) {
  k_mse<<<gs(count), 256, 0, s>>>(p, t, g, count, loss);
  return cudaGetLastError();
}
cudaError_t net_adam(float* w, const float* g, float* m, float* v, void* wb, int64_t count,
                     float lr, float b1, float b2, float eps, int step, cudaStream_t s) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_adam<<<gs(count), 256, 0, s>>>(w, g, m, v, (__nv_bfloat16*)wb, count, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}
cudaError_t net_cast_bf16(const float* a, void* b, int64_t count, cudaStream_t s) {
  k_cast_bf16<<<gs(count), 256, 0, s>>>(a, (__nv_bfloat16*)b, count);
  return cudaGetLastError();
}

}  // namespace lddmm
