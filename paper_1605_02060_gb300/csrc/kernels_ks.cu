// Tensor-core axis pass over a pre-split field, for all six products of K (§2.4):
//     C(l, n) = sum_k A(l, k) B(k, n)       over all lines l of one axis,
// with B = R or R^T (the orthonormal real DFT basis of that axis).
//
// The field arrives already split into bf16 hi and lo planes (A = hi + lo to 16 mantissa bits),
// laid out [line][k] with the transformed axis contiguous (K-major).  A TMA load of a 64 k x
// 128 line box with the 128-byte swizzle therefore lands directly in the canonical swizzled
// operand layout of tcgen05.mma: there is no conversion step between the copy and the tensor
// cores.  The previous pass wrote the field that way: its epilogue stores its output transposed
// into the next axis's line order, split into hi and lo, so the only per-element work left is
// in the epilogues.  The split costs no extra bytes (2 x 2 bytes per fp32 value).
//
// Roles inside one CTA (one persistent CTA per SM, 448 threads):
//   warp 0      TMA producer: A hi/lo boxes into an AS-deep ring; B (bf16 hi/lo tables of the
//               axis, [Nc][Kp]) either resident (loaded once) or streamed per 64-k block;
//   warp 1      TMEM owner and MMA issuer (one thread): hi*hi + hi*lo + lo*hi per 16-k step into
//               a double-buffered TMEM accumulator (2 x Nc <= 512 columns);
//   warps 2-9   epilogue: tcgen05.ld of 16/32 columns (warp w reads TMEM lanes 32(w%4)..+31, the
//               two warps of a lane quadrant split the columns), optional K symbol or the
//               gradient-descent update, stores;
//   warps 10-13 x axis longer than 256: the output columns 256.. in FP32 on the CUDA cores,
//               one line per thread, read from the same A stages (hi + lo) as the MMA; an A
//               stage is free once the MMA has committed and these 128 threads have arrived.
//               Passes without such columns whose outputs are staged give these warps to
//               the epilogue (three warps per TMEM lane quadrant instead of two): the epilogue's
//               element-wise conversions and stores, not the tensor cores, set those passes'
//               pace, and more warps hide more of their latency.
// Every wait is bounded and observes a CTA-wide abort flag; on abort the kernel drains its
// copies and MMAs, frees TMEM and reports through *err.
#include <cuda.h>
#include <cuda_bf16.h>

#include "kernels.h"
#include "tc_ptx.cuh"

namespace lddmm {

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

constexpr int KS_NT = 448;
constexpr int KS_W_TMA = 0, KS_W_MMA = 1;  // epilogue: warps 2 .. 2 + 4 nparts - 1
constexpr int KS_ABOX = 128 * 128;         // one A box: 128 lines x 64 bf16 (16 KB)
constexpr int KS_MAXS = 6;                 // ring depths (A and streamed B) at most
// Lines longer than 256 (up to 272): the main product covers the output columns 0..239 (N = 240,
// two accumulators at TMEM columns 0 and 240) and a second product the columns 240.. (N = 32)
// into one accumulator at TMEM column 480, which the epilogue drains first in every tile.
constexpr int KS_NMAIN = 240, KS_TCOL = 480;
constexpr int KS_SMEM_CAP = 225 * 1024;    // dynamic shared memory of any pass, at most

struct KsArgs {
  int nlines;          // lines of the input field
  int L;               // transform length: valid k and valid output columns
  int Nc;              // output columns (L rounded up to 16, at most 272): B has Nc rows
  int Nm, Nt;          // widths of the main and the second product (Nc and 0, or 240 and Nc - 240)
  int nk, nkb;         // 16-wide k-steps and 64-wide k-blocks over the whole length
  int split;           // 1: three products (hi*hi + hi*lo + lo*hi), 0: hi*hi
  int AS, BS, bres;    // A ring depth; streamed B ring depth; 1: B resident (nkb blocks)
  int ntiles;          // 128-line tiles
  int nparts;          // epilogue column ranges (four warps each, one per TMEM lane quadrant)
  KsOut o;             // output addressing
  float eps;           // KS_OUT_UPD: step size
  const float* lx;     // symbol (o.sym): lambda per x, y, z frequency
  const float* ly;
  const float* lz;
  float alpha, gamma;
  int X, Y;            // symbol: line l = (c X + x) Y + y
  int* err;
  uint32_t poll;       // probes per pipeline wait before the CTA aborts
  int zz;              // the fused z pass: forward product, symbol, inverse product
  int ostore;          // staged outputs leave by TMA stores of the warps' 32-line groups (tmO)
};

__host__ __device__ inline int ks_abytes(int split) { return (split ? 2 : 1) * KS_ABOX; }
__host__ __device__ inline int ks_bbytes(int split, int Nc) { return (split ? 2 : 1) * Nc * 128; }
// per epilogue warp: 32 lines x 16 columns of fp32, rows padded to 17 (conflict-free transpose)
constexpr int KS_SROW = 17;
// transposed split outputs: per column range (2 or 3 of them), a tile of 16 columns x 128 lines
// of bf16 hi and lo, through which the four lane-quadrant warps of the range store runs of 128
// consecutive lines
constexpr int KS_CTILE = 2 * 16 * 128 * 2;
// (only when the output rows hold a multiple of 8 lines, so that the 8-line pieces are aligned:
// with other row lengths the per-lane stores measured faster)
__host__ __device__ inline bool ks_staged(const KsArgs& a) {
  return a.o.G != 1 && a.o.kind == KS_OUT_SPLIT && a.o.E % 8 == 0;
}
__host__ __device__ inline int ks_sbytes(const KsArgs& a) {
  if (a.o.G == 1) return 4 * a.nparts * 32 * KS_SROW * 4;   // row outputs: a tile per warp
  return ks_staged(a) ? a.nparts * KS_CTILE : 0;
}
__host__ __device__ inline int ks_smem(const KsArgs& a) {
  return 1024 + a.AS * ks_abytes(a.split) + (a.bres ? a.nkb : a.BS) * ks_bbytes(a.split, a.Nc) +
         ks_sbytes(a);
}
// rows of one B box (the TMA box is at most 256 rows: a 272-row table takes two)
__host__ __device__ inline int ks_brows(int Nc) { return Nc <= 256 ? Nc : Nc / 2; }

// tcgen05 shared-memory descriptor for a K-major operand in the 128-byte swizzled layout:
// rows of 128 bytes (64 bf16 of k), 8-row atoms of 1024 bytes (SBO), atoms 1024-byte aligned;
// a 16-k step inside the 128-byte row advances the start address by 32 bytes.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;                    // LBO (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;          // SBO: 8 rows x 128 bytes
  d |= (uint64_t)1 << 46;                    // descriptor version for tcgen05
  d |= (uint64_t)2 << 61;                    // layout: 128-byte swizzle
  return d;
}

__device__ __forceinline__ uint16_t bf16_bits(__nv_bfloat16 b) {
  return *reinterpret_cast<const uint16_t*>(&b);
}

// hi = bf16(x), lo = bf16(x - hi): x = hi + lo to 16 mantissa bits.
__device__ __forceinline__ void split1(float x, uint16_t& h, uint16_t& l) {
  const __nv_bfloat16 hb = __float2bfloat16_rn(x);
  h = bf16_bits(hb);
  l = bf16_bits(__float2bfloat16_rn(x - __bfloat162float(hb)));
}

// 8 bf16 (one 16-byte word, element 0 in the low half of the first word) added to x[0..7]
__device__ __forceinline__ void add_bf8(uint4 w, float* x) {
  const uint32_t u[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    x[2 * j] += __uint_as_float(u[j] << 16);
    x[2 * j + 1] += __uint_as_float(u[j] & 0xffff0000u);
  }
}

// Bulk prefetch of [p, p + bytes) into L2 (16-byte aligned, bytes a multiple of 16).
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
// The 16-byte-aligned part of [p, p + bytes) into L2 (nothing when it is empty).
__device__ __forceinline__ void prefetch_l2_inner(const void* p, uint32_t bytes) {
  const uintptr_t a = ((uintptr_t)p + 15u) & ~(uintptr_t)15u;
  const uintptr_t e = ((uintptr_t)p + bytes) & ~(uintptr_t)15u;
  if (e > a) prefetch_l2(reinterpret_cast<const void*>(a), (uint32_t)(e - a));
}

// Element offset of (line l, column 0): l = (a D + b) E + e -> (a F + b) P + e.
__device__ __forceinline__ long long out_base(const KsOut& o, long long l) {
  const long long e = l % o.E, t = l / o.E;
  return (t / o.D * o.F + t % o.D) * o.P + e;
}

// Store cnt (<= NMAX) consecutive output columns n0.. of one line, one element at a time
// (transposed outputs whose runs are not vector aligned, and the FP32 tail columns), split into
// bf16 hi/lo or plain fp32 (the update's tail columns are stored by the tail threads).  The loops
// are unrolled over NMAX so that vc stays in registers.
template <int NMAX>
__device__ __forceinline__ void store_scalar(const KsOut& o, int split, long long base, int n0,
                                             const float* vc, int cnt) {
  if (o.kind == KS_OUT_SPLIT) {
    uint16_t* oh = reinterpret_cast<uint16_t*>(o.out);
#pragma unroll
    for (int j = 0; j < NMAX; ++j) {
      if (j < cnt) {
        uint16_t h, lo;
        split1(vc[j], h, lo);
        const long long off = base + (long long)(n0 + j) * o.G;
        oh[off] = h;
        if (split) oh[o.plane + off] = lo;
      }
    }
  } else {
    float* of = reinterpret_cast<float*>(o.out);
#pragma unroll
    for (int j = 0; j < NMAX; ++j)
      if (j < cnt) of[base + (long long)(n0 + j) * o.G] = vc[j];
  }
}

__host__ __device__ inline bool is_upd_host(int kind) {
  return kind == KS_OUT_UPD || kind == KS_OUT_UPD_BF16;
}
__device__ __forceinline__ bool is_upd(int kind) { return is_upd_host(kind); }

// 4 consecutive bf16 (8 bytes) <-> float4
__device__ __forceinline__ float4 bf4_to_f4(uint2 u) {
  return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                     __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
}
__device__ __forceinline__ uint2 f4_to_bf4(float4 w) {
  const __nv_bfloat162 a = __floats2bfloat162_rn(w.x, w.y), b = __floats2bfloat162_rn(w.z, w.w);
  return make_uint2(*reinterpret_cast<const uint32_t*>(&a), *reinterpret_cast<const uint32_t*>(&b));
}

__device__ __forceinline__ uint32_t pack_bf16x2(uint16_t a, uint16_t b) {
  return (uint32_t)a | ((uint32_t)b << 16);
}

// Row-wise outputs (o.G == 1, line l at l * o.P): the 16 columns n0.. of the warp's 32 lines
// line0.. (lane = line on entry) leave through the warp's shared-memory tile, so that a lane
// writes 8 consecutive bf16 columns (split, 16-byte stores) or 4 consecutive fp32 columns
// (plain or the update, 16-byte loads and stores) of one line, and a store instruction covers
// 16 or 8 lines.  (Transposed outputs, consecutive lines = consecutive positions, are already
// coalesced across the lanes and are stored element by element from registers.)
// The old v that the update combines with the 16 columns n0.. of the warp's 32 lines, in the
// lane order store_rows uses (4 consecutive fp32 columns of one line per 16-byte load).
__device__ __forceinline__ void load_old_rows(const KsOut& o, int lane, long long line0,
                                              long long nlines, int n0, int ncols, float4* old) {
  const float* of = reinterpret_cast<const float*>(o.out);
  const uint16_t* ob = reinterpret_cast<const uint16_t*>(o.out);
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    const int idx = it * 32 + lane, r = idx >> 2, c4 = (idx & 3) * 4;
    const long long l = line0 + r;
    if (l < nlines && n0 + c4 + 4 <= ncols) {
      if (o.kind == KS_OUT_UPD_BF16)
        old[it] = bf4_to_f4(*reinterpret_cast<const uint2*>(ob + l * o.P + n0 + c4));
      else
        old[it] = *reinterpret_cast<const float4*>(of + l * o.P + n0 + c4);
    }
  }
}

__device__ __forceinline__ void store_rows(const KsOut& o, int split, float eps, float* sg,
                                           int lane, long long line0, long long nlines, int n0,
                                           int ncols, const float* vc, const float4* old) {
#pragma unroll
  for (int j = 0; j < 16; ++j) sg[lane * KS_SROW + j] = vc[j];
  __syncwarp();
  if (o.kind == KS_OUT_SPLIT) {
    uint16_t* oh = reinterpret_cast<uint16_t*>(o.out);
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      const int idx = it * 32 + lane, r = idx >> 1, c8 = (idx & 1) * 8;
      const long long l = line0 + r;
      if (l < nlines && n0 + c8 + 8 <= ncols) {
        uint16_t h[8], lo[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) split1(sg[r * KS_SROW + c8 + k], h[k], lo[k]);
        const long long off = l * o.P + n0 + c8;
        *reinterpret_cast<uint4*>(oh + off) =
            make_uint4(pack_bf16x2(h[0], h[1]), pack_bf16x2(h[2], h[3]), pack_bf16x2(h[4], h[5]),
                       pack_bf16x2(h[6], h[7]));
        if (split)
          *reinterpret_cast<uint4*>(oh + o.plane + off) =
              make_uint4(pack_bf16x2(lo[0], lo[1]), pack_bf16x2(lo[2], lo[3]),
                         pack_bf16x2(lo[4], lo[5]), pack_bf16x2(lo[6], lo[7]));
      }
    }
  } else {
    float* of = reinterpret_cast<float*>(o.out);
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int idx = it * 32 + lane, r = idx >> 2, c4 = (idx & 3) * 4;
      const long long l = line0 + r;
      if (l < nlines && n0 + c4 + 4 <= ncols) {
        const float* q = sg + r * KS_SROW + c4;
        float4 w = make_float4(q[0], q[1], q[2], q[3]);
        if (is_upd(o.kind)) {
          const float4 p = old[it];
          w = make_float4(p.x - eps * (2.f * p.x - w.x), p.y - eps * (2.f * p.y - w.y),
                          p.z - eps * (2.f * p.z - w.z), p.w - eps * (2.f * p.w - w.w));
        }
        if (o.kind == KS_OUT_UPD_BF16)
          *reinterpret_cast<uint2*>(reinterpret_cast<uint16_t*>(o.out) + l * o.P + n0 + c4) =
              f4_to_bf4(w);
        else
          *reinterpret_cast<float4*>(of + l * o.P + n0 + c4) = w;
      }
    }
  }
  __syncwarp();
}

// Epilogue kinds: each pass is compiled with only its own output path, so that the registers of
// the other paths do not count against it (the kernel runs at the 128-register limit of 448
// threads).
enum { EPI_T_STAGED = 0, EPI_T = 1, EPI_ROWS = 2, EPI_UPD = 3, EPI_ZZ = 4 };

__host__ __device__ inline int ks_epi(const KsArgs& a) {
  if (a.zz) return EPI_ZZ;
  if (is_upd_host(a.o.kind)) return EPI_UPD;
  if (a.o.G == 1) return EPI_ROWS;
  return ks_staged(a) ? EPI_T_STAGED : EPI_T;
}

template <int EPI>
__global__ void __launch_bounds__(KS_NT, 1) k_dft_ks(const __grid_constant__ CUtensorMap tmA,
                                                     const __grid_constant__ CUtensorMap tmB,
                                                     const __grid_constant__ CUtensorMap tmB2,
                                                     const __grid_constant__ CUtensorMap tmO,
                                                     KsArgs a) {
  constexpr bool ZZ = EPI == EPI_ZZ;
  extern __shared__ __align__(1024) uint8_t smem_dyn[];
  __shared__ __align__(8) uint64_t b_afull[KS_MAXS], b_aempty[KS_MAXS], b_bfull[KS_MAXS],
      b_bempty[KS_MAXS];
  __shared__ __align__(8) uint64_t b_tfull[2], b_tempty[2], b_fin;
  // the fused z pass: b_tfull[0] / [1] = forward / inverse accumulator full, b_tempty[1] = the
  // inverse accumulator drained, b_a2[kb] = 64-column block kb of the scaled spectrum (the second
  // product's A operand, in TMEM over the forward accumulator) converted
  __shared__ __align__(8) uint64_t b_a2[4];
  // the second product's accumulator (columns 240..) drained by the last epilogue part
  __shared__ __align__(8) uint64_t b_ttail;
  __shared__ uint32_t tmem_sh;
  __shared__ int abort_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nepi = 4 * a.nparts;                   // epilogue warps 2 .. 2 + nepi - 1
  uint8_t* smem = smem_dyn + ((1024u - (ptx::smem_u32(smem_dyn) & 1023u)) & 1023u);
  const int abytes = ks_abytes(a.split), bbytes = ks_bbytes(a.split, a.Nc);
  uint8_t* aring = smem;
  uint8_t* bring = smem + a.AS * abytes;
  float* stg = reinterpret_cast<float*>(bring + (a.bres ? a.nkb : a.BS) * bbytes);
  volatile int* abort = &abort_sh;

  if (warp == KS_W_MMA) {
    ptx::tmem_alloc(ptx::smem_u32(&tmem_sh), 512u);
    ptx::tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < a.AS; ++i) {
      ptx::mbar_init(ptx::smem_u32(&b_afull[i]), 1);
      ptx::mbar_init(ptx::smem_u32(&b_aempty[i]), 1);
    }
    for (int i = 0; i < KS_MAXS; ++i) {
      ptx::mbar_init(ptx::smem_u32(&b_bfull[i]), 1);
      ptx::mbar_init(ptx::smem_u32(&b_bempty[i]), 1);
    }
    for (int i = 0; i < 2; ++i) {
      ptx::mbar_init(ptx::smem_u32(&b_tfull[i]), 1);
      ptx::mbar_init(ptx::smem_u32(&b_tempty[i]), 32 * nepi);
    }
    ptx::mbar_init(ptx::smem_u32(&b_fin), 1);
    for (int i = 0; i < 4; ++i) ptx::mbar_init(ptx::smem_u32(&b_a2[i]), 32 * nepi);
    ptx::mbar_init(ptx::smem_u32(&b_ttail), 128);
    ptx::fence_mbar_init();
    abort_sh = 0;
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = tmem_sh;
  const int my_tiles =
      blockIdx.x < (unsigned)a.ntiles ? (a.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int nkb = a.nkb, AS = a.AS, BS = a.BS;

  if (warp == KS_W_TMA) {
    // ------------------------------------------------------------ producers
    // lane 0 loads the A boxes (and a resident B once); lane 1 streams B, so that neither ring's
    // refill waits behind the other's
    const int np = a.split ? 2 : 1;
    const int br = ks_brows(a.Nc);
    if (lane == 0) {
      ptx::prefetch_tmap(&tmA);
      ptx::prefetch_tmap(&tmB);
      if (ZZ) ptx::prefetch_tmap(&tmB2);
      if (a.bres && my_tiles > 0) {
        const uint32_t fb = ptx::smem_u32(&b_bfull[0]);
        ptx::mbar_arrive_expect_tx(fb, (uint32_t)(nkb * bbytes));
        for (int kb = 0; kb < nkb; ++kb)
          for (int pl = 0; pl < np; ++pl)
            for (int r = 0; r < a.Nc; r += br)
              ptx::tma_load_3d(ptx::smem_u32(bring + kb * bbytes + (pl * a.Nc + r) * 128), &tmB,
                               kb * 64, r, pl, fb);
      }
      uint32_t g = 0;
      for (int i = 0; i < my_tiles; ++i) {
        const int line0 = (blockIdx.x + i * gridDim.x) * 128;
        for (int kb = 0; kb < nkb; ++kb, ++g) {
          const int s = (int)(g % AS);
          if (!ptx::mbar_wait_or_abort(ptx::smem_u32(&b_aempty[s]), ((g / AS) & 1) ^ 1, abort, a.poll)) goto pa_done;
          const uint32_t fa = ptx::smem_u32(&b_afull[s]);
          ptx::mbar_arrive_expect_tx(fa, (uint32_t)abytes);
          for (int pl = 0; pl < np; ++pl)
            ptx::tma_load_3d(ptx::smem_u32(aring + s * abytes + pl * KS_ABOX), &tmA, kb * 64,
                             line0, pl, fa);
        }
      }
    pa_done:
      // copies still in flight (only after an abort can any remain unconsumed)
      for (uint32_t q = (g > (uint32_t)AS ? g - AS : 0u); q < g; ++q)
        ptx::mbar_wait(ptx::smem_u32(&b_afull[q % AS]), (q / AS) & 1);
      if (a.bres && my_tiles > 0) ptx::mbar_wait(ptx::smem_u32(&b_bfull[0]), 0u);
    } else if (lane == 1 && !a.bres) {
      // the tiles' B blocks in the order the MMA takes them (the fused z pass: the forward
      // table's blocks, then the inverse table's)
      uint32_t gb = 0;
      for (int i = 0; i < my_tiles; ++i) {
        for (int t = 0; t < (ZZ ? 2 : 1); ++t) {
          for (int kb = 0; kb < nkb; ++kb, ++gb) {
            const int sb = (int)(gb % BS);
            if (!ptx::mbar_wait_or_abort(ptx::smem_u32(&b_bempty[sb]), ((gb / BS) & 1) ^ 1, abort, a.poll)) goto pb_done;
            const uint32_t fb = ptx::smem_u32(&b_bfull[sb]);
            ptx::mbar_arrive_expect_tx(fb, (uint32_t)bbytes);
            for (int pl = 0; pl < np; ++pl)
              for (int r = 0; r < a.Nc; r += br)
                ptx::tma_load_3d(ptx::smem_u32(bring + sb * bbytes + (pl * a.Nc + r) * 128),
                                 t ? &tmB2 : &tmB, kb * 64, r, pl, fb);
          }
        }
      }
    pb_done:
      for (uint32_t q = (gb > (uint32_t)BS ? gb - BS : 0u); q < gb; ++q)
        ptx::mbar_wait(ptx::smem_u32(&b_bfull[q % BS]), (q / BS) & 1);
    }
  } else if (warp == KS_W_MMA) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t id = ptx::idesc_bf16(128, a.Nm);
      const uint32_t idt = a.Nt ? ptx::idesc_bf16(128, a.Nt) : 0u;
      const uint32_t a0 = ptx::smem_u32(aring), b0 = ptx::smem_u32(bring);
      const uint32_t blo = (uint32_t)a.Nc * 128u;               // B lo plane offset
      const uint32_t bto = (uint32_t)a.Nm * 128u;               // the second product's B rows
      uint32_t g = 0;
      if constexpr (ZZ) {
        // forward product into columns 0.. (A from the ring, B the forward table), then, block by
        // block as the epilogue converts it, the inverse product of the scaled spectrum (A in
        // TMEM over the forward accumulator, B the inverse table) into columns 256..
        uint32_t gb = 0;
        const uint32_t d2 = tmem + 256u;
        for (int i = 0; i < my_tiles; ++i) {
          // the forward accumulator still holds the previous tile's spectrum until the previous
          // inverse product has completed
          if (i > 0 && !ptx::mbar_wait_or_abort(ptx::smem_u32(&b_tfull[1]), (uint32_t)(i - 1) & 1u, abort, a.poll)) break;
          ptx::tc_fence_after();
          bool ok = true;
          for (int kb = 0; kb < nkb; ++kb, ++g, ++gb) {
            const int s = (int)(g % AS), sb = (int)(gb % BS);
            if (!ptx::mbar_wait_or_abort(ptx::smem_u32(&b_afull[s]), (g / AS) & 1, abort, a.poll) ||
                !ptx::mbar_wait_or_abort(ptx::smem_u32(&b_bfull[sb]), (gb / BS) & 1, abort, a.poll)) {
              ok = false;
              break;
            }
            ptx::tc_fence_after();
            const uint32_t as = a0 + (uint32_t)(s * abytes), bs = b0 + (uint32_t)(sb * bbytes);
            const int nst = min(4, a.nk - kb * 4);
            const uint64_t ah = desc_sw128(as), al = desc_sw128(as + (uint32_t)KS_ABOX);
            const uint64_t bh = desc_sw128(bs), bl = desc_sw128(bs + blo);
            for (int j = 0; j < nst; ++j) {
              const uint64_t o2 = 2u * (uint32_t)j;
              ptx::mma_bf16(tmem, ah + o2, bh + o2, id, (kb | j) ? 1u : 0u);
              if (a.split) {
                ptx::mma_bf16(tmem, ah + o2, bl + o2, id, 1u);
                ptx::mma_bf16(tmem, al + o2, bh + o2, id, 1u);
              }
            }
            ptx::mma_commit(ptx::smem_u32(&b_aempty[s]));
            ptx::mma_commit(ptx::smem_u32(&b_bempty[sb]));
          }
          if (!ok) break;
          ptx::mma_commit(ptx::smem_u32(&b_tfull[0]));
          if (!ptx::mbar_wait_or_abort(ptx::smem_u32(&b_tempty[1]), ((uint32_t)i & 1u) ^ 1u, abort, a.poll)) break;
          for (int kb = 0; kb < nkb; ++kb, ++gb) {
            const int sb = (int)(gb % BS);
            if (!ptx::mbar_wait_or_abort(ptx::smem_u32(&b_a2[kb]), (uint32_t)i & 1u, abort, a.poll) ||
                !ptx::mbar_wait_or_abort(ptx::smem_u32(&b_bfull[sb]), (gb / BS) & 1, abort, a.poll)) {
              ok = false;
              break;
            }
            ptx::tc_fence_after();
            const uint32_t bs = b0 + (uint32_t)(sb * bbytes);
            const int nst = min(4, a.nk - kb * 4);
            const uint64_t bh = desc_sw128(bs), bl = desc_sw128(bs + blo);
            for (int j = 0; j < nst; ++j) {
              const uint32_t ta = tmem + (uint32_t)(16 * (kb * 4 + j));   // hi at ta, lo at ta + 8
              const uint64_t o2 = 2u * (uint32_t)j;
              ptx::mma_bf16_ta(d2, ta, bh + o2, id, (kb | j) ? 1u : 0u);
              if (a.split) {
                ptx::mma_bf16_ta(d2, ta, bl + o2, id, 1u);
                ptx::mma_bf16_ta(d2, ta + 8u, bh + o2, id, 1u);
              }
            }
            ptx::mma_commit(ptx::smem_u32(&b_bempty[sb]));
          }
          if (!ok) break;
          ptx::mma_commit(ptx::smem_u32(&b_tfull[1]));
        }
        goto m_done;
      }
      if (a.bres && my_tiles > 0 &&
          !ptx::mbar_wait_or_abort(ptx::smem_u32(&b_bfull[0]), 0u, abort, a.poll)) goto m_done;
      for (int i = 0; i < my_tiles; ++i) {
        const int ab = i & 1;
        const uint32_t use = (uint32_t)(i >> 1);
        if (!ptx::mbar_wait_or_abort(ptx::smem_u32(&b_tempty[ab]), (use & 1) ^ 1, abort, a.poll)) break;
        ptx::tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(ab * (a.Nt ? KS_NMAIN : a.Nc));
        const uint32_t dt = tmem + (uint32_t)KS_TCOL;
        bool ok = true;
        for (int kb = 0; kb < nkb; ++kb, ++g) {
          const int s = (int)(g % AS);
          const int sb = a.bres ? kb : (int)(g % BS);
          if (!ptx::mbar_wait_or_abort(ptx::smem_u32(&b_afull[s]), (g / AS) & 1, abort, a.poll) ||
              (!a.bres && !ptx::mbar_wait_or_abort(ptx::smem_u32(&b_bfull[sb]), (g / BS) & 1, abort, a.poll))) {
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint32_t as = a0 + (uint32_t)(s * abytes), bs = b0 + (uint32_t)(sb * bbytes);
          const int nst = min(4, a.nk - kb * 4);
          // descriptors of the k-block's first 16-k step; a step advances the start address by
          // 32 bytes, i.e. the descriptor by 2
          const uint64_t ah = desc_sw128(as), al = desc_sw128(as + (uint32_t)KS_ABOX);
          const uint64_t bh = desc_sw128(bs), bl = desc_sw128(bs + blo);
          const uint64_t th = desc_sw128(bs + bto), tl = desc_sw128(bs + blo + bto);
          // the columns 240..: the epilogue drains the previous tile's first, before this tile's
          // second product starts; from then on the two products alternate step by step
          const bool tail_wait = a.Nt && kb == 0 && i > 0;
          for (int j = 0; j < nst; ++j) {
            const uint64_t o2 = 2u * (uint32_t)j;
            const uint32_t acc = (kb | j) ? 1u : 0u;
            ptx::mma_bf16(d, ah + o2, bh + o2, id, acc);
            if (a.split) {
              ptx::mma_bf16(d, ah + o2, bl + o2, id, 1u);
              ptx::mma_bf16(d, al + o2, bh + o2, id, 1u);
            }
            if (a.Nt && !tail_wait) {
              ptx::mma_bf16(dt, ah + o2, th + o2, idt, acc);
              if (a.split) {
                ptx::mma_bf16(dt, ah + o2, tl + o2, idt, 1u);
                ptx::mma_bf16(dt, al + o2, th + o2, idt, 1u);
              }
            }
          }
          if (tail_wait) {
            if (!ptx::mbar_wait_or_abort(ptx::smem_u32(&b_ttail), (uint32_t)(i - 1) & 1u, abort, a.poll)) {
              ok = false;
              break;
            }
            ptx::tc_fence_after();
            for (int j = 0; j < nst; ++j) {
              const uint64_t o2 = 2u * (uint32_t)j;
              ptx::mma_bf16(dt, ah + o2, th + o2, idt, j ? 1u : 0u);
              if (a.split) {
                ptx::mma_bf16(dt, ah + o2, tl + o2, idt, 1u);
                ptx::mma_bf16(dt, al + o2, th + o2, idt, 1u);
              }
            }
          }
          ptx::mma_commit(ptx::smem_u32(&b_aempty[s]));
          if (!a.bres) ptx::mma_commit(ptx::smem_u32(&b_bempty[sb]));
        }
        if (!ok) break;
        ptx::mma_commit(ptx::smem_u32(&b_tfull[ab]));
      }
    m_done:
      ptx::mma_commit(ptx::smem_u32(&b_fin));
    }
  } else if (warp < 2 + nepi) {
    // ------------------------------------------------------------ epilogue (warps 2-9 or 2-13)
    const int q = warp & 3;                          // TMEM lane quadrant of this warp
    const int part = (warp - 2) >> 2, nparts = nepi >> 2;   // column range of this warp
    const int nch = a.Nc / 16;
    const int cbeg = part * nch / nparts, cend = (part + 1) * nch / nparts;
    // This part's chunks in the order it drains them: the second product's (columns 240.., in
    // the last part) first, so that the next tile's second product may start, then the main
    // product's.  Chunk c lies at TMEM column 16 c of the accumulator, or 480 + 16 (c - 15).
    const int ntm = a.Nt ? KS_NMAIN / 16 : nch;      // chunks of the main product
    const int tb = cend > ntm ? max(cbeg, ntm) : cend;
    const int ntl = cend - tb;                       // second-product chunks of this part
    const int cnt = cend - cbeg;
    auto chunk_at = [&](int k) { return k < ntl ? tb + k : cbeg + (k - ntl); };
    const KsOut& o = a.o;
    const int Lc = min(a.L, a.Nc);                   // valid tensor-core output columns
    // columns written per line (row-wise split outputs stop at the row pitch)
    const int ncols = (o.G == 1 && o.kind == KS_OUT_SPLIT) ? min(a.Nc, (int)o.P) : Lc;
    float* sg = stg + (warp - 2) * (32 * KS_SROW);
    for (int i = 0; i < my_tiles; ++i) {
      // the fused z pass drains its one inverse accumulator (columns 256..) every tile
      const int ab = ZZ ? 1 : (i & 1);
      const uint32_t use = ZZ ? (uint32_t)i : (uint32_t)(i >> 1);
      const long long l = (long long)(blockIdx.x + i * gridDim.x) * 128 + q * 32 + lane;
      const bool valid = l < a.nlines;
      // output address of (line l, column 0) and the symbol's (x, y) part
      long long base = 0;
      float sxy = 1.f;
      if (valid) {
        base = out_base(o, l);
        if (o.sym || ZZ) {
          const int ry = (int)(l % a.Y), rx = (int)((l / a.Y) % a.X);
          sxy = a.gamma + a.alpha * (a.lx[rx] + a.ly[ry]);
        }
      }
      bool conv_ok = true;
      if constexpr (ZZ) {
        // Scaled spectrum: block kb of the forward accumulator (columns 64 kb..) is read, divided
        // by the symbol (gamma + alpha (lx + ly + lz))^2, split into bf16 hi/lo and written back
        // in place as the inverse product's A operand: per 16 columns, 8 columns of hi pairs
        // then 8 of lo pairs.  The 16-column chunks go round robin to the parts (chunk c to part
        // c % nparts), block by block; every epilogue thread arrives once per block, so block kb
        // is ready as soon as its few chunks are.  A thread whose wait gives up skips the
        // conversion but still reaches the drain's agreement below, where its part leaves
        // together.  (lz is zero padded to whole 16-column groups.)
        conv_ok = ptx::mbar_wait_or_abort(ptx::smem_u32(&b_tfull[0]), (uint32_t)i & 1u, abort, a.poll);
        ptx::tc_fence_after();
        const uint32_t t1 = tmem + ((uint32_t)(q * 32) << 16);
        for (int kb = 0; conv_ok && kb < nkb; ++kb) {
          const int c1 = min(4 * kb + 4, nch);
          for (int c = 4 * kb; c < c1; ++c) {
            if (c % nparts != part) continue;
            float vc[16];
            ptx::tmem_ld16(t1 + (uint32_t)(c * 16), vc);
            const float4* lz4 = reinterpret_cast<const float4*>(a.lz + c * 16);
            uint32_t hw[8], lw[8];
#pragma unroll
            for (int j4 = 0; j4 < 4; ++j4) {
              const float4 z4 = __ldg(lz4 + j4);
              const float zl[4] = {z4.x, z4.y, z4.z, z4.w};
#pragma unroll
              for (int jj = 0; jj < 2; ++jj) {
                const int j = 2 * j4 + jj;
                uint16_t h0, l0, h1, l1;
                const float d0 = fmaf(a.alpha, zl[2 * jj], sxy);
                const float d1 = fmaf(a.alpha, zl[2 * jj + 1], sxy);
                split1(__fdividef(vc[2 * j], d0 * d0), h0, l0);
                split1(__fdividef(vc[2 * j + 1], d1 * d1), h1, l1);
                hw[j] = pack_bf16x2(h0, h1);
                lw[j] = pack_bf16x2(l0, l1);
              }
            }
            ptx::tmem_st8(t1 + (uint32_t)(c * 16), hw);
            if (a.split) ptx::tmem_st8(t1 + (uint32_t)(c * 16 + 8), lw);
          }
          ptx::tmem_wait_st();
          ptx::tc_fence_before();
          ptx::mbar_arrive(ptx::smem_u32(&b_a2[kb]));
        }
      }
      const long long line0 = l - lane;
      // the update reads the old v of this warp's columns: start bringing it into L2 while the
      // tensor cores are still on the tile
      if (EPI == EPI_UPD && valid && cend * 16 > cbeg * 16) {
        const int c1 = min(cend * 16, Lc);
        const int es = o.kind == KS_OUT_UPD_BF16 ? 2 : 4;
        if (c1 > cbeg * 16)
          prefetch_l2_inner(reinterpret_cast<const char*>(o.out) + (l * o.P + cbeg * 16) * es,
                            (uint32_t)((c1 - cbeg * 16) * es));
      }
      // the update: the old v of the first pair of chunks is requested before the wait for the
      // accumulator, each later pair's just before its TMEM load (pairs never straddle the two
      // products: a part holds 0 or 2 chunks of the second)
      float4 oldv[8];
      if (EPI == EPI_UPD && cnt > 0) {
        load_old_rows(o, lane, line0, a.nlines, chunk_at(0) * 16, ncols, oldv);
        if (cnt > 1) load_old_rows(o, lane, line0, a.nlines, chunk_at(1) * 16, ncols, oldv + 4);
      }
      constexpr bool staged = EPI == EPI_T_STAGED || ZZ;
      int got = (conv_ok && ptx::mbar_wait_or_abort(ptx::smem_u32(&b_tfull[ab]), use & 1, abort, a.poll)) ? 1 : 0;
      if constexpr (staged) {
        // the four warps of a column range meet at named barriers below: they give up together
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.s32 p, %1, 0;\n\t"
            "bar.red.and.pred p, %2, 128, p;\n\tselp.s32 %0, 1, 0, p;\n\t}"
            : "=r"(got)
            : "r"(got), "r"(2 + part)
            : "memory");
      }
      if (!got) break;
      ptx::tc_fence_after();
      const uint32_t tlane = tmem + ((uint32_t)(q * 32) << 16);
      const uint32_t tbuf = ZZ ? 256u : (uint32_t)(ab * (a.Nt ? KS_NMAIN : a.Nc));
      auto tcol = [&](int c) -> uint32_t {
        return tlane + (c < ntm ? tbuf + 16u * (uint32_t)c : (uint32_t)KS_TCOL + 16u * (uint32_t)(c - ntm));
      };
      if (staged && a.ostore) {
        // Transposed split output by TMA: the output rows hold a multiple of 32 lines, so this
        // warp's 32 lines (one TMEM lane quadrant) lie in one row.  Per 16-column chunk the warp
        // writes its lines' hi and lo bf16 into its own 2 KB of the range's shared tile,
        // [plane][16 columns][32 lines], and one lane stores them as two boxes of a 5-D tensor
        // map over (line in row, row in block, column, block, plane).
        uint16_t* wt = reinterpret_cast<uint16_t*>(stg) + part * (KS_CTILE / 2) + q * (2 * 16 * 32);
        const uint32_t wts = ptx::smem_u32(wt);
        const bool gvalid = line0 < a.nlines;
        const long long t = line0 / o.E;
        const int e0 = (int)(line0 - t * o.E), r1 = (int)(t % o.D), r3 = (int)(t / o.D);
        for (int k = 0; k < cnt; ++k) {
          const int c = chunk_at(k);
          float vc[16];
          ptx::tmem_ld16(tcol(c), vc);
          if (k + 1 == ntl) {             // the second product's columns are read
            ptx::tc_fence_before();
            ptx::mbar_arrive(ptx::smem_u32(&b_ttail));
          }
          if (lane == 0) ptx::bulk_wait_read_all();   // the previous boxes have left the tile
          __syncwarp();
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            uint16_t h, lo;
            split1(vc[j], h, lo);
            wt[j * 32 + lane] = h;
            wt[512 + j * 32 + lane] = lo;
          }
          ptx::fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0 && gvalid) {
            ptx::tma_store_5d(&tmO, wts, e0, r1, c * 16, r3, 0);
            if (a.split) ptx::tma_store_5d(&tmO, wts + 1024u, e0, r1, c * 16, r3, 1);
            ptx::bulk_commit();
          }
        }
      } else if constexpr (staged) {
        // Transposed split output.  Per 16-column chunk the four quadrant warps of this column
        // range write their lines' hi/lo bf16 into the range's shared tile [plane][col][line];
        // then each of the 128 threads stores 16-byte pieces of 8 consecutive lines of one
        // column, so that a warp instruction writes two runs of 128 lines (256 bytes) instead
        // of 32 runs of one line.  A thread's line group g = its index % 16 is the same for
        // every piece it stores, so its output offset is found once per tile.
        uint16_t* tile = reinterpret_cast<uint16_t*>(stg) + part * (KS_CTILE / 2);
        const int tp = q * 32 + lane, grp = tp & 15;
        const long long lg0 = line0 - q * 32 + grp * 8;     // first line of this thread's group
        const long long gb = lg0 < a.nlines ? out_base(o, lg0) : 0;
        // 8 lines in one run: one 16-byte store when 16-byte aligned, else two of 8 bytes.  A
        // group that crosses the end of an output row (E lines) continues at the next row's
        // base nb from its line k on.
        const bool run = lg0 + 7 < a.nlines && out_base(o, lg0 + 7) == gb + 7;
        const int vec = !run ? 0 : ((gb & 7) == 0 ? 2 : ((gb & 3) == 0 ? 1 : 0));
        const int kcut = run ? 8 : (int)min((long long)8, o.E - lg0 % o.E);
        const long long nb = (!run && lg0 + kcut < a.nlines) ? out_base(o, lg0 + kcut) : 0;
        const int np = a.split ? 2 : 1;
        for (int k = 0; k < cnt; ++k) {
          const int c = chunk_at(k);
          float vc[16];
          ptx::tmem_ld16(tcol(c), vc);
          if (k + 1 == ntl) {             // the second product's columns are read
            ptx::tc_fence_before();
            ptx::mbar_arrive(ptx::smem_u32(&b_ttail));
          }
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            uint16_t h, lo;
            split1(vc[j], h, lo);
            tile[j * 128 + tp] = h;
            tile[(16 + j) * 128 + tp] = lo;
          }
          asm volatile("bar.sync %0, 128;" ::"r"(2 + part) : "memory");
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int k = tp + 128 * r, pl = k >> 8, j = (k >> 4) & 15, n = c * 16 + j;
            if (pl < np && n < Lc) {
              uint16_t* oh = reinterpret_cast<uint16_t*>(o.out) + (pl ? o.plane : 0);
              const uint16_t* src = tile + (pl * 16 + j) * 128 + grp * 8;
              if (vec == 2) {
                *reinterpret_cast<uint4*>(oh + gb + (long long)n * o.G) =
                    *reinterpret_cast<const uint4*>(src);
              } else if (vec == 1) {
                const uint4 w = *reinterpret_cast<const uint4*>(src);
                uint2* d = reinterpret_cast<uint2*>(oh + gb + (long long)n * o.G);
                d[0] = make_uint2(w.x, w.y);
                d[1] = make_uint2(w.z, w.w);
              } else {
                for (int e = 0; e < 8; ++e) {
                  if (lg0 + e < a.nlines) {
                    // rows shorter than 8 lines: a group can span several of them
                    const long long off = o.E < 8 ? out_base(o, lg0 + e)
                                                  : (e < kcut ? gb + e : nb + (e - kcut));
                    oh[off + (long long)n * o.G] = src[e];
                  }
                }
              }
            }
          }
          asm volatile("bar.sync %0, 128;" ::"r"(2 + part) : "memory");
        }
      } else {
      for (int k = 0; k < cnt; k += 2) {
        const int cp = chunk_at(k);
        const int npair = (k + 1 < cnt && k + 1 != ntl) ? 2 : 1;
        if (EPI == EPI_UPD && k > 0) {
          load_old_rows(o, lane, line0, a.nlines, cp * 16, ncols, oldv);
          if (npair == 2) load_old_rows(o, lane, line0, a.nlines, cp * 16 + 16, ncols, oldv + 4);
        }
        float v[32];
        if (npair == 2) ptx::tmem_ld32(tcol(cp), v);
        else ptx::tmem_ld16(tcol(cp), *reinterpret_cast<float(*)[16]>(v));
        if (k + npair == ntl) {           // the second product's columns are read
          ptx::tc_fence_before();
          ptx::mbar_arrive(ptx::smem_u32(&b_ttail));
        }
#pragma unroll
        for (int u2 = 0; u2 < 2; ++u2) {
          if (u2 >= npair) break;
          const int n0 = (cp + u2) * 16;
          float* vc = v + 16 * u2;
          if (o.sym && valid) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const float den = fmaf(a.alpha, __ldg(a.lz + min(n0 + j, a.L - 1)), sxy);
              vc[j] = __fdividef(vc[j], den * den);
            }
          }
          if constexpr (EPI == EPI_ROWS || EPI == EPI_UPD)   // whole warp
            store_rows(o, a.split, a.eps, sg, lane, line0, a.nlines, n0, ncols, vc, oldv + 4 * u2);
          else if (valid)
            store_scalar<16>(o, a.split, base, n0, vc, min(16, Lc - n0));
        }
      }
      }
      ptx::tc_fence_before();
      ptx::mbar_arrive(ptx::smem_u32(&b_tempty[ab]));
    }
    if (a.ostore && lane == 0) ptx::bulk_wait_all();   // this warp's stores have completed
  }

  // ------------------------------------------------------------ teardown
  __syncthreads();
  if (warp == KS_W_MMA) {
    if (lane == 0) {
      if (!ptx::mbar_wait(ptx::smem_u32(&b_fin), 0u)) abort_sh = 1;
    }
    __syncwarp();
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, 512u);
  }
  __syncthreads();   // abort_sh as the MMA warp left it
  if (threadIdx.x == 0 && abort_sh) atomicExch(a.err, 3);
}

int g_ks_sms = 0;

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

// fp32 rows [nrows][L] -> split field: one thread per (row, column), columns fastest.
__global__ void k_split_rows(const float* __restrict__ in, long long nrows, int L, int split,
                             KsOut o) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrows * L) return;
  const long long l = i / L;
  const int n = (int)(i - l * L);
  const long long off = out_base(o, l) + (long long)n * o.G;
  uint16_t h, lo;
  split1(in[i], h, lo);
  uint16_t* oh = reinterpret_cast<uint16_t*>(o.out);
  oh[off] = h;
  if (split) oh[o.plane + off] = lo;
}

}  // namespace

void* tma_encode_fn() { return reinterpret_cast<void*>(encode_fn()); }

int ks_pitch(int L) { return (L + 7) / 8 * 8; }

bool ks_supported(const KPlan& kp) {
  if (!tma_encode_fn() || !kp.ks[0][0] || !kp.ks[1][0] || !kp.ks[2][0]) return false;
  return kp.nx % 4 == 0 && kp.nx <= 264 && kp.ny <= 256 && kp.nz <= 256;
}

long long ks_field_floats(int nx, int ny, int nz, int ncomp) {
  const long long X = nx, Y = ny, Z = nz;
  const long long px = ks_pitch(nx), py = ks_pitch(ny), pz = ks_pitch(nz);
  long long m = X * Y * Z;                      // fp32 rows
  if (Z * Y * px > m) m = Z * Y * px;           // split [c][z][y][x] (x rows)
  if (X * pz * py > m) m = X * pz * py;         // [c][x'][Pz][y] and [c][z][x'][y']
  if (X * Y * pz > m) m = X * Y * pz;           // [c][x'][y'][z]
  return m * ncomp;                             // two bf16 planes = one float per value
}

cudaError_t ks_split_rows(const float* in, long long nrows, int L, int split, const KsOut& o,
                          cudaStream_t s) {
  const long long n = nrows * L;
  if (n > 0) k_split_rows<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, nrows, L, split, o);
  return cudaGetLastError();
}

// One pass of k_dft_ks over a split field `in` (hi plane, lo plane nlines*pitch elements later),
// lines of length L along `axis` (0: x, 1: y, 2: z) with row pitch ks_pitch(L), output as `o`
// says (eps: the update's step size for KS_OUT_UPD).  zz: the fused z pass (axis 2): forward
// product, symbol and inverse product of every line, output as the inverse pass's.
cudaError_t ks_axis_pass(const KPlan& kp, int axis, bool inverse, int split, const void* in,
                         long long nlines, const KsOut& o, float eps, cudaStream_t s, bool zz) {
  EncodeTiledFn enc = reinterpret_cast<EncodeTiledFn>(tma_encode_fn());
  if (!enc) return cudaErrorNotSupported;
  KsArgs a{};
  a.L = axis == 0 ? kp.nx : axis == 1 ? kp.ny : kp.nz;
  a.Nc = (a.L + 15) / 16 * 16;
  if (a.Nc > 272) return cudaErrorNotSupported;
  a.Nm = a.Nc <= 256 ? a.Nc : KS_NMAIN;
  a.Nt = a.Nc - a.Nm;
  a.nk = (a.L + 15) / 16;
  a.nkb = (a.L + 63) / 64;
  a.split = split;
  a.nlines = (int)nlines;
  a.ntiles = (int)((nlines + 127) / 128);
  a.o = o;
  a.eps = eps;
  // row-wise outputs: line l at l * P (P a multiple of 8 bf16 or 4 floats)
  if (o.G == 1 && (o.D != 1 || o.E != 1 || o.F != 1)) return cudaErrorInvalidValue;
  a.lx = kp.lx; a.ly = kp.ly; a.lz = kp.lz;
  a.alpha = kp.alpha; a.gamma = kp.gamma;
  a.X = kp.nx; a.Y = kp.ny;
  a.err = kp.err;
  a.poll = kp.poll_limit ? kp.poll_limit : (1u << 22);
  a.zz = zz ? 1 : 0;
  // the fused pass drains through the staging tiles: its output rows hold a multiple of 8 lines
  if (zz && (axis != 2 || o.sym || !ks_staged(a) || a.Nt)) return cudaErrorInvalidValue;
  const int P = ks_pitch(a.L);
  const int np = split ? 2 : 1;
  // A: [2 planes][nlines][P] bf16, box 64 k x 128 lines, 128-byte swizzle; k >= L and lines
  // beyond the field read as zero
  CUtensorMap tmA, tmB, tmB2;
  {
    cuuint64_t dims[3] = {(cuuint64_t)a.L, (cuuint64_t)nlines, (cuuint64_t)np};
    cuuint64_t strides[2] = {(cuuint64_t)P * 2, (cuuint64_t)nlines * P * 2};
    cuuint32_t box[3] = {64, 128, 1}, es[3] = {1, 1, 1};
    if (enc(&tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(in), dims, strides, box,
            es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  // B: [2 planes][Nc][Kp] bf16 (zero padded), box 64 k x Nc rows (two boxes of Nc / 2 rows past
  // 256; the fused z pass: the forward table, then the inverse one)
  for (int t = 0; t < (zz ? 2 : 1); ++t) {
    const int Kp = (a.L + 15) / 16 * 16;
    cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)a.Nc, 2};
    cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)a.Nc * Kp * 2};
    cuuint32_t box[3] = {64, (cuuint32_t)ks_brows(a.Nc), 1}, es[3] = {1, 1, 1};
    const int which = zz ? t : (inverse ? 1 : 0);
    if (enc(t ? &tmB2 : &tmB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, kp.ks[axis][which], dims,
            strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  if (!zz) tmB2 = tmB;
  // Staged outputs whose rows hold a multiple of 32 lines leave by TMA stores: a 5-D map over
  // (line in row e < E, row in block < D, column < Lc, block, plane), element
  // (t / D * F + t % D) * P + e + column * G (+ plane) for line t * E + e, boxes of 32 lines x 16
  // columns; the lines fill whole blocks of D rows, so every box lies inside the output.  Other
  // outputs (or addresses the map cannot describe) take the per-thread stores.
  CUtensorMap tmO = tmA;
  a.ostore = 0;
  if (ks_staged(a) && o.E % 32 == 0 && nlines % (o.E * o.D) == 0 &&
      (reinterpret_cast<uintptr_t>(o.out) & 15) == 0 &&
      o.P % 8 == 0 && o.G % 8 == 0 && (o.F * o.P) % 8 == 0 && (!split || o.plane % 8 == 0)) {
    const long long rows = (nlines + o.E - 1) / o.E;
    cuuint64_t dims[5] = {(cuuint64_t)o.E, (cuuint64_t)o.D, (cuuint64_t)min(a.L, a.Nc),
                          (cuuint64_t)((rows + o.D - 1) / o.D), (cuuint64_t)(split ? 2 : 1)};
    cuuint64_t strides[4] = {(cuuint64_t)o.P * 2, (cuuint64_t)o.G * 2, (cuuint64_t)(o.F * o.P) * 2,
                             (cuuint64_t)(split ? o.plane : o.F * o.P) * 2};
    cuuint32_t box[5] = {32, 1, 16, 1, 1}, es[5] = {1, 1, 1, 1, 1};
    if (enc(&tmO, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, o.out, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
      a.ostore = 1;
  }
  // Shared memory (<= 225 KB): B resident when all its k-blocks fit next to 2 A stages;
  // otherwise 3 A stages (2 when needed) and as many streamed B stages as fit (at least 2).
  // Staged and row outputs take 12 epilogue warps (three column ranges) when that still
  // leaves room for 2 A and 2 B stages, else 8.
  const int ab = ks_abytes(split), bb = ks_bbytes(split, a.Nc);
  bool fits = false;
  for (int parts = (ks_staged(a) || o.G == 1) ? 3 : 2; parts >= 2 && !fits; --parts) {
    a.nparts = parts;
    const int budget = KS_SMEM_CAP - 1024 - ks_sbytes(a);
    if (!zz && a.nkb * bb + 2 * ab <= budget) {
      a.bres = 1;
      a.AS = min(KS_MAXS, (budget - a.nkb * bb) / ab);
      a.BS = 1;
      fits = true;
    } else {
      a.bres = 0;
      a.AS = 3;
      a.BS = min(KS_MAXS, (budget - 3 * ab) / bb);
      if (a.BS < 2) {
        a.AS = 2;
        a.BS = min(KS_MAXS, (budget - 2 * ab) / bb);
      }
      fits = a.BS >= 2;
    }
  }
  if (!fits) return cudaErrorNotSupported;
  // the second product's chunks (15 and 16 of 17) must fall in one part, the last
  if (a.Nt && (a.nparts - 1) * (a.Nc / 16) / a.nparts > KS_NMAIN / 16) return cudaErrorNotSupported;
  const int smem = ks_smem(a);
  const int epi = ks_epi(a);
  auto kern = epi == EPI_T_STAGED ? k_dft_ks<EPI_T_STAGED>
            : epi == EPI_T        ? k_dft_ks<EPI_T>
            : epi == EPI_ROWS     ? k_dft_ks<EPI_ROWS>
            : epi == EPI_ZZ       ? k_dft_ks<EPI_ZZ>
                                  : k_dft_ks<EPI_UPD>;
  // The limit is set once per kernel, to the cap every pass stays under: a per-pass value would
  // lower it below what an earlier launch of the same kernel (a recorded graph node) needs.
  static bool limit_set[5] = {false, false, false, false, false};
  if (smem > KS_SMEM_CAP) return cudaErrorNotSupported;
  if (!limit_set[epi]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         KS_SMEM_CAP);
    if (e != cudaSuccess) return e;
    limit_set[epi] = true;
  }
  if (!g_ks_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_ks_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_ks_sms <= 0) g_ks_sms = 148;
  }
  const int grid = a.ntiles < g_ks_sms ? a.ntiles : g_ks_sms;
  if (grid > 0) kern<<<grid, KS_NT, smem, s>>>(tmA, tmB, tmB2, tmO, a);
  return cudaGetLastError();
}

}  // namespace lddmm
