// Per-axis real DFTs of the smoothing operator K (§2.4) as tensor-core GEMMs on sm_103a.
//
// One launch transforms every line of one axis of a field stack:
//     C(m, n) = sum_k A(m, k) B(k, n),   A(m, k) = field value k of line m,
// with B the (padded) orthonormal real DFT matrix or its transpose, so that K = R^T S R is
// five or six such passes (see kernels_dft.cu).  Lines are addressed through
// base(m) = (m / mdiv) * mhi + (m % mdiv) * mlo and element k of a line at base(m) + k * kstride,
// which covers x lines (contiguous) and y/z lines (strided, consecutive m contiguous).
//
// Per CTA: a 128-line tile, the full N = Npad output columns in TMEM (fp32 accumulators).
// A k-step of 16: 256 threads stage the fp32 field slice with cp.async, split each value into
// bf16 hi + lo (x = hi + lo to ~2^-17 relative) and write both into K-major core-matrix layout;
// the B slice (pre-split on the host, already in that layout) is copied by cp.async; one thread
// issues tcgen05.mma:  hi*hi + hi*lo + lo*hi  (split mode) or hi*hi (plain bf16).  Stages form an
// S-deep ring guarded by mbarriers that tcgen05.commit arrives on.  The epilogue reads TMEM with
// tcgen05.ld and stores (plain / times the K symbol / fused gradient-descent update).
// Every wait is bounded; a timeout sets *err, drains the issued MMAs and frees TMEM.
#include <cuda_bf16.h>

#include "kernels.h"
#include "tc_ptx.cuh"

namespace lddmm {

struct TcArgs {
  const float* in;
  float* out;
  const uint4* B;       // nk k-steps x [hi block | lo block], each Npad x 16 bf16, core-matrix layout
  int M;                // lines
  int L;                // transform length (valid k and n)
  int Npad;             // multiple of 16, >= L (also K padding)
  int nk;               // Npad / 16
  int mdiv;
  long long mhi, mlo, kstride;
  int epi;              // 0 plain, 1 times symbol, 2 update v -= eps (2 v - C)
  const float* lx;
  const float* ly;
  const float* lz;
  int nx, nxy;
  float alpha, gamma, eps;
  int split;            // 1: hi*hi + hi*lo + lo*hi, 0: hi*hi
  int vec;              // 16-byte cp.async legal for the A slices
  int tmem_cols;
  int* err;
};

constexpr int TC_THREADS = 256;
constexpr int TC_BM = 128;
constexpr int RAW_BYTES = TC_BM * 16 * 4;   // fp32 slice
constexpr int AOP_BYTES = TC_BM * 16 * 2;   // one bf16 operand slice (hi or lo)

__host__ __device__ inline int stage_bytes(int Npad) { return RAW_BYTES + 2 * AOP_BYTES + Npad * 64; }

// byte offset of (row, kk) inside one K-major no-swizzle slice of 16 columns
__device__ __forceinline__ uint32_t kmajor_off(int row, int kk) {
  return (uint32_t)((kk >> 3) * 128 + (row >> 3) * 256 + (row & 7) * 16 + (kk & 7) * 2);
}

__device__ __forceinline__ long long line_base(const TcArgs& a, int m) {
  return (long long)(m / a.mdiv) * a.mhi + (long long)(m % a.mdiv) * a.mlo;
}

// Stage k-step s of A (raw fp32) and B (bf16 hi/lo) into ring slot `slot`.
template <int LOADT>
__device__ __forceinline__ void issue_loads(const TcArgs& a, uint8_t* stage, int m0, int s) {
  const int tid = threadIdx.x;
  const uint32_t raw = ptx::smem_u32(stage);
  const int k0 = s * 16;
  if (LOADT == 0) {
    // x lines: raw[m][16] floats, element (m, k) at line_base(m) + k
    if (a.vec) {
      for (int q = tid; q < TC_BM * 4; q += TC_THREADS) {   // 4 x 16 B per line
        const int m = q >> 2, c = q & 3;
        const int gm = m0 + m, k = k0 + c * 4;
        const int valid = (gm < a.M) ? max(0, min(4, a.L - k)) : 0;
        const float* src = valid ? a.in + line_base(a, gm) + k : a.in;
        ptx::cp_async16(raw + (uint32_t)(m * 64 + c * 16), src, (uint32_t)valid * 4u);
      }
    } else {
      for (int q = tid; q < TC_BM * 16; q += TC_THREADS) {
        const int m = q >> 4, c = q & 15;
        const int gm = m0 + m, k = k0 + c;
        const int ok = (gm < a.M) && (k < a.L);
        const float* src = ok ? a.in + line_base(a, gm) + k : a.in;
        ptx::cp_async4(raw + (uint32_t)(m * 64 + c * 4), src, ok ? 4u : 0u);
      }
    }
  } else {
    // strided lines: raw[k][128] floats, element (m, k) at line_base(m) + k * kstride
    if (a.vec) {
      for (int q = tid; q < 16 * (TC_BM / 4); q += TC_THREADS) {
        const int kk = q / (TC_BM / 4), mq = q % (TC_BM / 4);
        const int gm = m0 + mq * 4, k = k0 + kk;
        const int valid = (k < a.L) ? max(0, min(4, a.M - gm)) : 0;
        const float* src = valid ? a.in + line_base(a, gm) + (long long)k * a.kstride : a.in;
        ptx::cp_async16(raw + (uint32_t)(kk * 512 + mq * 16), src, (uint32_t)valid * 4u);
      }
    } else {
      for (int q = tid; q < 16 * TC_BM; q += TC_THREADS) {
        const int kk = q / TC_BM, m = q % TC_BM;
        const int gm = m0 + m, k = k0 + kk;
        const int ok = (gm < a.M) && (k < a.L);
        const float* src = ok ? a.in + line_base(a, gm) + (long long)k * a.kstride : a.in;
        ptx::cp_async4(raw + (uint32_t)(kk * 512 + m * 4), src, ok ? 4u : 0u);
      }
    }
  }
  // B slice: contiguous Npad * 64 bytes
  const uint32_t bdst = raw + RAW_BYTES + 2 * AOP_BYTES;
  const uint4* bsrc = a.B + (size_t)s * (size_t)a.Npad * 4;
  for (int q = tid; q < a.Npad * 4; q += TC_THREADS)
    ptx::cp_async16(bdst + (uint32_t)q * 16u, bsrc + q, 16u);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo_elem, float hi_elem) {
  // two bf16 (round to nearest) in one 32-bit word, first element in the low half
  const __nv_bfloat16 a = __float2bfloat16_rn(lo_elem);
  const __nv_bfloat16 b = __float2bfloat16_rn(hi_elem);
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// raw fp32 slice -> bf16 hi and lo operand slices (K-major core matrices)
template <int LOADT>
__device__ __forceinline__ void convert_slice(uint8_t* stage, int split) {
  const int tid = threadIdx.x;
  int m, h;
  float x[8];
  const float* raw = reinterpret_cast<const float*>(stage);
  if (LOADT == 0) {
    m = tid >> 1;
    h = tid & 1;
    const float4* p = reinterpret_cast<const float4*>(raw + m * 16 + h * 8);
    const float4 u = p[0], w = p[1];
    x[0] = u.x; x[1] = u.y; x[2] = u.z; x[3] = u.w;
    x[4] = w.x; x[5] = w.y; x[6] = w.z; x[7] = w.w;
  } else {
    m = tid & (TC_BM - 1);
    h = tid >> 7;
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = raw[(h * 8 + i) * TC_BM + m];
  }
  float hi[8], lo[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    hi[i] = __bfloat162float(__float2bfloat16_rn(x[i]));
    lo[i] = x[i] - hi[i];
  }
  uint4 H, Lw;
  H.x = pack_bf16(hi[0], hi[1]); H.y = pack_bf16(hi[2], hi[3]);
  H.z = pack_bf16(hi[4], hi[5]); H.w = pack_bf16(hi[6], hi[7]);
  const uint32_t off = kmajor_off(m, h * 8);
  *reinterpret_cast<uint4*>(stage + RAW_BYTES + off) = H;
  if (split) {
    Lw.x = pack_bf16(lo[0], lo[1]); Lw.y = pack_bf16(lo[2], lo[3]);
    Lw.z = pack_bf16(lo[4], lo[5]); Lw.w = pack_bf16(lo[6], lo[7]);
    *reinterpret_cast<uint4*>(stage + RAW_BYTES + AOP_BYTES + off) = Lw;
  }
}

template <int LOADT, int S>
__global__ void __launch_bounds__(TC_THREADS, 1) k_dft_tc(TcArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ __align__(8) uint64_t bars[S + 1];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * TC_BM;
  const int sb = stage_bytes(a.Npad);
  const int nk = a.nk;

  if (warp == 0) {
    ptx::tmem_alloc(ptx::smem_u32(&tmem_base_sh), (uint32_t)a.tmem_cols);
    ptx::tmem_relinquish();
  }
  if (tid == 0) {
    for (int i = 0; i <= S; ++i) ptx::mbar_init(ptx::smem_u32(&bars[i]), 1);
    ptx::fence_mbar_init();
    abort_sh = 0;
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = tmem_base_sh;

  // prologue: k-steps 0 .. S-2
#pragma unroll
  for (int s = 0; s < S - 1; ++s) {
    if (s < nk) issue_loads<LOADT>(a, smem + s * sb, m0, s);
    ptx::cp_async_commit();
  }

  int issued = 0;   // MMA groups issued by thread 0
  for (int i = 0; i < nk; ++i) {
    const int slot = i % S;
    uint8_t* st = smem + slot * sb;
    ptx::cp_async_wait<S - 2>();
    __syncthreads();
    if (abort_sh) break;
    convert_slice<LOADT>(st, a.split);
    ptx::fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      ptx::tc_fence_after();
      const uint32_t sbase = ptx::smem_u32(st);
      const uint32_t a_hi = sbase + RAW_BYTES, a_lo = a_hi + AOP_BYTES;
      const uint32_t b_hi = sbase + RAW_BYTES + 2 * AOP_BYTES, b_lo = b_hi + a.Npad * 32;
      for (int n0 = 0; n0 < a.Npad; n0 += 256) {
        const int nc = min(256, a.Npad - n0);
        const uint32_t id = ptx::idesc_bf16(TC_BM, nc);
        const uint32_t boff = (uint32_t)(n0 / 8) * 256u;
        const uint32_t d = tmem + (uint32_t)n0;
        ptx::mma_bf16(d, ptx::smem_desc(a_hi, 128, 256), ptx::smem_desc(b_hi + boff, 128, 256), id,
                      i > 0 ? 1u : 0u);
        if (a.split) {
          ptx::mma_bf16(d, ptx::smem_desc(a_hi, 128, 256), ptx::smem_desc(b_lo + boff, 128, 256),
                        id, 1u);
          ptx::mma_bf16(d, ptx::smem_desc(a_lo, 128, 256), ptx::smem_desc(b_hi + boff, 128, 256),
                        id, 1u);
        }
      }
      ptx::mma_commit(ptx::smem_u32(&bars[slot]));
      ++issued;
    }
    // refill the slot used by step i-1 with step i+S-1 once its MMAs have read it
    const int nxt = i + S - 1;
    if (nxt < nk) {
      if (i >= 1) {
        const int ps = (i - 1) % S;
        if (!ptx::mbar_wait(ptx::smem_u32(&bars[ps]), (uint32_t)(((i - 1) / S) & 1))) {
          atomicExch(a.err, 1);
          abort_sh = 1;
        }
      }
      if (!abort_sh) issue_loads<LOADT>(a, smem + (nxt % S) * sb, m0, nxt);
    }
    ptx::cp_async_commit();
  }
  ptx::cp_async_wait<0>();
  // all MMAs issued by thread 0 complete -> bars[S]
  if (tid == 0) ptx::mma_commit(ptx::smem_u32(&bars[S]));
  __syncthreads();
  if (!ptx::mbar_wait(ptx::smem_u32(&bars[S]), 0u)) {
    atomicExch(a.err, 2);
    abort_sh = 1;
  }
  ptx::tc_fence_after();
  __syncthreads();
  (void)issued;

  if (!abort_sh) {
    // epilogue: warp w reads TMEM lanes 32*(w%4).., columns split between the two warp halves
    const int g = warp & 3, half = warp >> 2;
    const int m = m0 + g * 32 + lane;
    const int nch = a.Npad / 16;
    const int c_per = (nch + 1) / 2;
    const int c_begin = half * c_per, c_end = min(nch, c_begin + c_per);
    const bool mok = m < a.M;
    const long long base = mok ? line_base(a, m) : 0;
    int rx = 0, ry = 0;
    if (a.epi == 1 && mok) {
      const int r = m % a.nxy;
      ry = r / a.nx;
      rx = r % a.nx;
    }
    for (int c = c_begin; c < c_end; ++c) {
      float v[16];
      ptx::tmem_ld16(tmem + ((uint32_t)(g * 32) << 16) + (uint32_t)(c * 16), v);
      if (!mok) continue;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int n = c * 16 + j;
        if (n >= a.L) break;
        float val = v[j];
        const long long addr = base + (long long)n * a.kstride;
        if (a.epi == 1) {
          const float den = a.gamma + a.alpha * (a.lx[rx] + a.ly[ry] + a.lz[n]);
          val = val / (den * den);
          a.out[addr] = val;
        } else if (a.epi == 2) {
          const float vo = a.out[addr];
          a.out[addr] = vo - a.eps * (2.f * vo - val);
        } else {
          a.out[addr] = val;
        }
      }
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 0) ptx::tmem_dealloc(tmem, (uint32_t)a.tmem_cols);
}

// ---------------------------------------------------------------------------------------------

static int pow2_cols(int n) {
  int c = 32;
  while (c < n) c <<= 1;
  return c;
}

template <int LOADT, int S>
static cudaError_t launch_tc(const TcArgs& a, cudaStream_t s) {
  const int smem = S * stage_bytes(a.Npad);
  // the kernel's shared-memory limit only ever rises: an earlier launch (a recorded graph node)
  // may need more than this one
  static int limit = 0;
  if (smem > limit) {
    cudaError_t e = cudaFuncSetAttribute(k_dft_tc<LOADT, S>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    limit = smem;
  }
  const int grid = (a.M + TC_BM - 1) / TC_BM;
  if (grid > 0) k_dft_tc<LOADT, S><<<grid, TC_THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

// One axis pass.  axis 0: x lines, 1: y lines, 2: z lines of ncomp fields nx*ny*nz.
cudaError_t tc_axis_pass(const KPlan& kp, int axis, bool inverse, int split, const float* in,
                         float* out, int ncomp, int epi, float eps, cudaStream_t s) {
  TcArgs a{};
  const long long X = kp.nx, Y = kp.ny, Z = kp.nz, XY = X * Y, N = XY * Z;
  const int L = axis == 0 ? kp.nx : axis == 1 ? kp.ny : kp.nz;
  a.in = in;
  a.out = out;
  a.L = L;
  a.Npad = (L + 15) / 16 * 16;
  a.nk = a.Npad / 16;
  a.B = reinterpret_cast<const uint4*>(kp.tc[axis][inverse ? 1 : 0]);
  a.epi = epi;
  a.lx = kp.lx; a.ly = kp.ly; a.lz = kp.lz;
  a.nx = kp.nx; a.nxy = (int)XY;
  a.alpha = kp.alpha; a.gamma = kp.gamma; a.eps = eps;
  a.split = split;
  a.tmem_cols = pow2_cols(a.Npad);
  a.err = kp.err;
  const bool al = ((uintptr_t)in & 15) == 0;
  if (axis == 0) {
    a.M = (int)(ncomp * Y * Z);
    a.mdiv = a.M + 1;
    a.mhi = 0;
    a.mlo = X;
    a.kstride = 1;
    a.vec = al && (X % 4 == 0);
  } else if (axis == 1) {
    a.M = (int)(ncomp * Z * X);
    a.mdiv = (int)X;
    a.mhi = XY;
    a.mlo = 1;
    a.kstride = X;
    a.vec = al && (X % 4 == 0);
  } else {
    a.M = (int)(ncomp * XY);
    a.mdiv = (int)XY;
    a.mhi = N;
    a.mlo = 1;
    a.kstride = XY;
    a.vec = al && (XY % 4 == 0) && (N % 4 == 0);
  }
  if (axis == 0) {
    if (a.Npad > 256) return launch_tc<0, 4>(a, s);
    return launch_tc<0, 3>(a, s);
  }
  if (a.Npad > 192) return launch_tc<1, 3>(a, s);
  return launch_tc<1, 4>(a, s);
}

}  // namespace lddmm
