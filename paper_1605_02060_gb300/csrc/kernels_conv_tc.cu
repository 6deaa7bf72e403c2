// 3D convolution of the warm-start network on the tensor cores (tcgen05, sm_103a), as an
// implicit GEMM:
//     Y[b, co, v] = bias[co] + sum_{ci, t} X[b, ci, v + o(t)] W[co, ci, t]     (zero padding)
// with M = 128 consecutive output voxels of one sample (a tile), N = Co (padded to a multiple of
// 16) and K = Ci x taps walked as k-steps of 16 input channels at one tap t.
//
// The activations stay float32 [B][C][n^3]; the weights are bf16 [Co][Ci][taps].  Each k-step's
// A slice (128 voxels x 16 channels, shifted by the tap, zero outside the grid) is split into a
// bf16 hi and lo part (x = hi + lo to 16 mantissa bits), so the two products hi*W + lo*W give
// the FP32 activations times the bf16 weights to ~2^-17, the same numbers as the CUDA-core
// kernel up to rounding order; accumulation is FP32 in TMEM.
//
// Roles inside one CTA (one tile of 128 voxels, all Co):
//   warps 0-7   stage each k-step: thread (voxel m = tid % 128, half h = tid / 128) gathers 8
//               input channels of its shifted voxel and writes their hi/lo bf16 in the K-major
//               core-matrix layout; the same threads copy the k-step's weight slice [Co][16];
//               proxy fence, arrive on the stage's full barrier.  After the last k-step warps
//               0-3 read the accumulator (warp w owns TMEM lanes 32w..32w+31) and add the bias,
//               the optional old output and ReLU; warps 4-7 take the upper half of the columns.
//   warp 8      TMEM owner and MMA issuer (one thread): two MMAs per k-step, a commit frees the
//               stage, a final commit hands the accumulator to the epilogue.
// Every wait is bounded: a timeout sets *err and the CTA drains, frees TMEM and returns.
#include <cuda_bf16.h>

#include "kernels.h"
#include "tc_ptx.cuh"

namespace lddmm {

namespace {

constexpr int CV_THREADS = 288;     // 8 staging/epilogue warps + the MMA warp
constexpr int CV_STAGES = 4;
constexpr int CV_ABYTES = 128 * 16 * 2;   // one bf16 A operand (hi or lo)

__device__ __forceinline__ uint32_t cv_kmaj(int row, int kk) {
  return (uint32_t)((kk >> 3) * 128 + (row >> 3) * 256 + (row & 7) * 16 + (kk & 7) * 2);
}

__host__ __device__ inline int cv_stage_bytes(int Np) { return 2 * CV_ABYTES + Np * 32; }
__device__ __forceinline__ int q_of(int warp) { return warp & 3; }

__device__ __forceinline__ uint32_t pack_bf2(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__global__ void __launch_bounds__(CV_THREADS) k_conv_tc(const float* __restrict__ x,
                                                        const __nv_bfloat16* __restrict__ w,
                                                        const float* __restrict__ bias,
                                                        float* __restrict__ y, int Ci, int Co,
                                                        int Np, int n, int ks, int relu,
                                                        int accumulate, int tcols, int* err) {
  extern __shared__ __align__(128) uint8_t cv_smem[];
  __shared__ __align__(8) uint64_t b_full[CV_STAGES], b_empty[CV_STAGES], b_done;
  __shared__ uint32_t tmem_sh;
  __shared__ int abort_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = blockIdx.y;
  const long long nv = (long long)n * n * n;
  const long long v0 = (long long)blockIdx.x * 128;
  const int taps = ks * ks * ks;
  const int nkc = Ci / 16;                  // channel groups
  const int nsteps = nkc * taps;
  const int sb = cv_stage_bytes(Np);
  volatile int* abort = &abort_sh;

  if (warp == 8) {
    ptx::tmem_alloc(ptx::smem_u32(&tmem_sh), (uint32_t)tcols);
    ptx::tmem_relinquish();
  }
  if (tid == 0) {
    for (int s = 0; s < CV_STAGES; ++s) {
      ptx::mbar_init(ptx::smem_u32(&b_full[s]), 256);
      ptx::mbar_init(ptx::smem_u32(&b_empty[s]), 1);
    }
    ptx::mbar_init(ptx::smem_u32(&b_done), 1);
    ptx::fence_mbar_init();
    abort_sh = 0;
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = tmem_sh;

  if (warp < 8) {
    // ------------------------------------------------------------ staging
    const int m = tid & 127, h = tid >> 7;
    const long long v = v0 + m;
    const bool vin = v < nv;
    const int vx = (int)(v % n), vy = (int)((v / n) % n), vz = (int)(v / ((long long)n * n));
    const float* xb = x + (long long)b * Ci * nv;
    bool ok = true;
    for (int st = 0; st < nsteps && ok; ++st) {
      const int s = st % CV_STAGES;
      const uint32_t par = (uint32_t)((st / CV_STAGES) & 1);
      if (!ptx::mbar_wait_or_abort(ptx::smem_u32(&b_empty[s]), par ^ 1u, abort)) { ok = false; break; }
      const int kc = st / taps, t = st % taps;
      int ox = 0, oy = 0, oz = 0;
      if (ks == 3) { ox = t % 3 - 1; oy = (t / 3) % 3 - 1; oz = t / 9 - 1; }
      const int sx = vx + ox, sy = vy + oy, sz = vz + oz;
      const bool in = vin && sx >= 0 && sx < n && sy >= 0 && sy < n && sz >= 0 && sz < n;
      const long long off = ((long long)sz * n + sy) * n + sx;
      float xv[8];
#pragma unroll
      for (int j = 0; j < 8; ++j)
        xv[j] = in ? __ldg(xb + (long long)(kc * 16 + h * 8 + j) * nv + off) : 0.f;
      uint32_t hw[4], lw[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const __nv_bfloat162 hb = __floats2bfloat162_rn(xv[2 * j], xv[2 * j + 1]);
        const float2 hf = __bfloat1622float2(hb);
        hw[j] = *reinterpret_cast<const uint32_t*>(&hb);
        lw[j] = pack_bf2(xv[2 * j] - hf.x, xv[2 * j + 1] - hf.y);
      }
      uint8_t* stg = cv_smem + s * sb;
      *reinterpret_cast<uint4*>(stg + cv_kmaj(m, 8 * h)) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      *reinterpret_cast<uint4*>(stg + CV_ABYTES + cv_kmaj(m, 8 * h)) =
          make_uint4(lw[0], lw[1], lw[2], lw[3]);
      // weight slice: row co, k = 16 channels of group kc at tap t (zero rows past Co)
      uint8_t* bs = stg + 2 * CV_ABYTES;
      for (int r = tid; r < Np * 2; r += 256) {
        const int co = r >> 1, hh = r & 1;
        uint16_t e[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const __nv_bfloat16 wv = co < Co ? w[((long long)co * Ci + kc * 16 + hh * 8 + j) * taps + t]
                                           : __float2bfloat16_rn(0.f);
          e[j] = *reinterpret_cast<const uint16_t*>(&wv);
        }
        *reinterpret_cast<uint4*>(bs + cv_kmaj(co, 8 * hh)) =
            make_uint4(e[0] | ((uint32_t)e[1] << 16), e[2] | ((uint32_t)e[3] << 16),
                       e[4] | ((uint32_t)e[5] << 16), e[6] | ((uint32_t)e[7] << 16));
      }
      ptx::fence_proxy_async_smem();
      ptx::mbar_arrive(ptx::smem_u32(&b_full[s]));
    }
    // ------------------------------------------------------------ epilogue
    const bool done = ok && ptx::mbar_wait_or_abort(ptx::smem_u32(&b_done), 0u, abort);
    if (!done && warp < 4) {
      // a wait gave up: the tile's outputs are marked invalid (NaN) besides the error flag
      const long long vo = v0 + q_of(warp) * 32 + lane;
      if (vo < nv)
        for (int co = 0; co < Co; ++co) y[((long long)b * Co + co) * nv + vo] = __int_as_float(0x7fc00000);
    }
    if (done) {
      ptx::tc_fence_after();
      const int q = warp & 3, half = warp >> 2;
      const int nch = Np / 16, hc = (nch + 1) / 2;
      const int cb = half ? hc : 0, ce = half ? nch : hc;
      const long long vo = v0 + q * 32 + lane;
      for (int c = cb; c < ce; ++c) {
        float acc[16];
        ptx::tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(c * 16), acc);
        if (vo < nv) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int co = c * 16 + j;
            if (co < Co) {
              float* o = y + ((long long)b * Co + co) * nv + vo;
              float r = acc[j] + (bias ? bias[co] : 0.f);
              if (accumulate) r += *o;
              if (relu) r = fmaxf(r, 0.f);
              *o = r;
            }
          }
        }
      }
      ptx::tc_fence_before();
    }
  } else if (lane == 0) {
    // ------------------------------------------------------------ MMA issuer
    const uint32_t id = ptx::idesc_bf16(128, Np);
    const uint32_t base = ptx::smem_u32(cv_smem);
    int st = 0;
    for (; st < nsteps; ++st) {
      const int s = st % CV_STAGES;
      if (!ptx::mbar_wait_or_abort(ptx::smem_u32(&b_full[s]), (uint32_t)((st / CV_STAGES) & 1), abort))
        break;
      ptx::tc_fence_after();
      const uint32_t sa = base + (uint32_t)(s * sb);
      const uint64_t dAh = ptx::smem_desc(sa, 128, 256), dAl = ptx::smem_desc(sa + CV_ABYTES, 128, 256);
      const uint64_t dB = ptx::smem_desc(sa + 2 * CV_ABYTES, 128, 256);
      ptx::mma_bf16(tmem, dAh, dB, id, st > 0 ? 1u : 0u);
      ptx::mma_bf16(tmem, dAl, dB, id, 1u);
      ptx::mma_commit(ptx::smem_u32(&b_empty[s]));
    }
    ptx::mma_commit(ptx::smem_u32(&b_done));
  }
  // ------------------------------------------------------------ teardown
  __syncthreads();
  if (warp == 8) {
    if (lane == 0) {
      // all MMAs of this CTA have completed before TMEM is freed
      if (!ptx::mbar_wait(ptx::smem_u32(&b_done), 0u)) abort_sh = 1;
    }
    __syncwarp();
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, (uint32_t)tcols);
  }
  __syncthreads();
  if (tid == 0 && abort_sh && err) atomicExch(err, 3);
}

}  // namespace

bool conv_tc_supported(int Ci, int Co) { return Ci % 16 == 0 && Co >= 1 && Co <= 256; }

// Device flag a tensor-core convolution sets when one of its bounded waits gave up (its tile's
// outputs are then NaN); allocated once per process.
static int* conv_err_flag() {
  static int* f = nullptr;
  if (!f && cudaMalloc((void**)&f, sizeof(int)) == cudaSuccess) cudaMemset(f, 0, sizeof(int));
  else cudaGetLastError();
  return f;
}

cudaError_t conv_tc_fwd(const float* x, const void* w, const float* bias, float* y, int B, int Ci,
                        int Co, int n, int ks, int relu, int accumulate, cudaStream_t s) {
  int* err = conv_err_flag();
  const int Np = (Co + 15) / 16 * 16;
  int tcols = 32;
  while (tcols < Np) tcols <<= 1;
  const int smem = CV_STAGES * cv_stage_bytes(Np);
  static int limit = 0;   // only ever raised (a recorded launch may need more than this one)
  if (smem > limit) {
    cudaError_t e = cudaFuncSetAttribute(k_conv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    limit = smem;
  }
  const long long nv = (long long)n * n * n;
  dim3 grid((unsigned)((nv + 127) / 128), (unsigned)B);
  k_conv_tc<<<grid, CV_THREADS, smem, s>>>(x, (const __nv_bfloat16*)w, bias, y, Ci, Co, Np, n, ks,
                                           relu, accumulate, tcols, err);
  return cudaGetLastError();
}

}  // namespace lddmm
