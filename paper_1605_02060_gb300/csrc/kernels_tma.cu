// Persistent, warp-specialised tensor-core pass for the per-axis real DFTs of K (§2.4):
//     C(m, n) = sum_k A(m, k) B(k, n)   over all lines m of one axis of a field stack,
// with A the fp32 field (k runs along the transformed axis) and B the padded orthonormal real
// DFT matrix (or its transpose) pre-split into bf16 hi + lo on the host.
//
// Roles inside one CTA (one CTA per SM, 480 threads):
//   warp 12      A producer: one cp.async.bulk.tensor load per raw box of the 128-line fp32
//                slice covering kb k-steps (x pass: 2 k-steps in a 16 KB box with the 128-byte
//                swizzle; y and z passes: 4 k-steps in a 32 KB box) into a ring of raw slots;
//                large boxes matter: the copy rate of a CTA is set by the number of boxes in
//                flight, not by their bytes;
//   warp 13      B producer: one bulk copy of the k-step's B slice into the operand ring, or the
//                whole table once when it fits in shared memory (resident B);
//   warps 4-11   converters: raw fp32 slice -> bf16 hi + lo (packed round-to-nearest) in K-major
//                core-matrix layout in the operand ring, proxy fence, arrive;
//   warp 14      TMEM owner and MMA issuer (one thread): hi*hi + hi*lo + lo*hi (or hi*hi) per
//                k-step into the tile's TMEM accumulator; tcgen05.commit frees the operand slot,
//                and after the last k-step signals the epilogue;
//   warps 0-3    epilogue: tcgen05.ld (warp w owns TMEM lanes 32w..32w+31), optional symbol
//                scaling or fused update, stores straight from registers to global memory
//                (y and z: the 32 lanes are 32 consecutive positions, so every store is one
//                coalesced 128-byte row; x: each lane writes 16-byte pieces of its own line).
//                For the fused update the old v is prefetched by cp.async into a per-warp ring,
//                NBV chunks ahead.  The accumulator is double-buffered in TMEM when
//                2*Nc <= 512 columns (Nc = output columns on the tensor cores).
// Line tiles: x pass: 128 consecutive x-lines (rows); y pass: 32 x by 4 (component, z) planes;
// z pass: 128 consecutive (y,x) positions of one component.
// Every wait is bounded and observes a CTA-wide abort flag; on abort the kernel drains its
// copies and MMAs, frees TMEM and reports through *err.
#include <cuda.h>
#include <cuda_bf16.h>

#include "kernels.h"
#include "tc_ptx.cuh"

namespace lddmm {

namespace {

constexpr int NT = 608;
constexpr int W_CONV = 4, W_PA = 12, W_PB = 13, W_MMA = 14, W_EPI2 = 15;
constexpr int NEPI = 8;              // epilogue warps: 0-3 and 15-18
constexpr int NCONV = 256;
constexpr int OPB = 128 * 16 * 2;    // one bf16 operand slice (hi or lo)
constexpr int NBV = 4;               // update: v chunks in flight per epilogue warp
constexpr int VSLOT = 32 * 16 * 4;   // one v chunk of a warp: 32 lines x 16 columns fp32
constexpr int KBMAX = 4;             // k-steps per raw box (at most)

struct TmaArgs {
  float* out;          // output field; for the update, v (read and written)
  const uint4* B;
  int L, Npad, nk;     // transform length, its 16-padding (k extent), k-steps
  int Nc;              // output columns on the tensor cores (Npad, or 256 with an FP32 tail)
  const float* tail;   // x pass, 256 < L <= 264: B(k, 256 + j) as float [Npad][8]
  int tw;              // tail columns (0: none)
  int kind;            // 0 x, 1 y, 2 z
  int ntiles;
  int X, XY, rows, nxc, ncz, tpc;
  long long N;
  int epi;             // 0 plain, 1 symbol, 2 update
  const float* lx;
  const float* ly;
  const float* lz;
  float alpha, gamma, eps;
  int split;
  int dbuf;
  int kb;              // k-steps per raw box
  int rawb;            // bytes of one raw box
  int RS, PS;          // raw-ring and operand-ring depths (PS k-steps, a multiple of G)
  int G;               // k-steps per operand group: one MMA-side wait and one commit per group
  int bres;            // 1: the whole B table is loaded once and stays in shared memory
  int* err;
};

// operand slot: A hi and lo, plus the k-step's B slice unless B is resident
__host__ __device__ inline int op_slot_bytes(int Nc, int bres) {
  return 2 * OPB + (bres ? 0 : Nc * 64);
}
__host__ __device__ inline int vring_bytes(int epi) { return epi == 2 ? NEPI * NBV * VSLOT : 0; }
// 1 KB of slack aligns the raw ring to the 1024-byte period of the 128-byte swizzle
// x tail: the FP32 table [Npad][8] and a [128][8] exchange area for the two k halves of a line
__host__ __device__ inline int tail_bytes(const TmaArgs& a) {
  return a.tw ? a.Npad * 8 * 4 + 128 * 8 * 4 : 0;
}
__host__ __device__ inline int smem_bytes(const TmaArgs& a) {
  return 1024 + a.RS * a.rawb + a.PS * op_slot_bytes(a.Nc, a.bres) +
         (a.bres ? a.nk * a.Nc * 64 : 0) + vring_bytes(a.epi) + tail_bytes(a);
}

__device__ __forceinline__ uint32_t kmaj(int row, int kk) {
  return (uint32_t)((kk >> 3) * 128 + (row >> 3) * 256 + (row & 7) * 16 + (kk & 7) * 2);
}

__device__ __forceinline__ void split8(const float* x, uint4& H, uint4& Lw) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const __nv_bfloat162 hb = __floats2bfloat162_rn(x[2 * j], x[2 * j + 1]);
    const float2 hf = __bfloat1622float2(hb);
    const __nv_bfloat162 lb = __floats2bfloat162_rn(x[2 * j] - hf.x, x[2 * j + 1] - hf.y);
    h[j] = *reinterpret_cast<const uint32_t*>(&hb);
    l[j] = *reinterpret_cast<const uint32_t*>(&lb);
  }
  H = make_uint4(h[0], h[1], h[2], h[3]);
  Lw = make_uint4(l[0], l[1], l[2], l[3]);
}

// Packed FP32 pairs: fma.rn.f32x2 rounds each half like fmaf (one instruction for two).
__device__ __forceinline__ uint64_t pack2(float x, float y) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
  return r;
}
__device__ __forceinline__ float2 unpack2(uint64_t r) {
  float2 v;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
  return v;
}
__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// tile coordinates of the TMA box (c0 innermost, c1 outermost) for tile t
__device__ __forceinline__ void tile_coords(const TmaArgs& a, int t, int& c0, int& c1) {
  if (a.kind == 0) { c0 = 0; c1 = t * 128; }
  else if (a.kind == 1) { c0 = (t % a.nxc) * 32; c1 = (t / a.nxc) * 4; }
  else { c0 = (t % a.tpc) * 128; c1 = t / a.tpc; }
}

// The 8 values k = 16 ks + 8 h .. +7 of line m from a raw box.
__device__ __forceinline__ void raw_read8(const TmaArgs& a, const uint8_t* rs, int m, int ks,
                                          int h, float* x) {
  if (a.kind == 0) {
    // [128 rows][32 floats], 16-byte chunk c of row m stored at chunk c ^ (m & 7)
    const int c = ks * 4 + h * 2, sw = m & 7;
    const float4 u = *reinterpret_cast<const float4*>(rs + m * 128 + ((c ^ sw) << 4));
    const float4 w = *reinterpret_cast<const float4*>(rs + m * 128 + (((c + 1) ^ sw) << 4));
    x[0] = u.x; x[1] = u.y; x[2] = u.z; x[3] = u.w; x[4] = w.x; x[5] = w.y; x[6] = w.z; x[7] = w.w;
  } else if (a.kind == 1) {
    // [4 planes][64 k][32 x]
    const float* q = reinterpret_cast<const float*>(rs) + ((m >> 5) * 64 + ks * 16 + h * 8) * 32 + (m & 31);
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = q[j * 32];
  } else {
    // [64 k][128 positions]
    const float* q = reinterpret_cast<const float*>(rs) + (ks * 16 + h * 8) * 128 + m;
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = q[j * 128];
  }
}

__global__ void __launch_bounds__(NT, 1) k_dft_tma(const __grid_constant__ CUtensorMap tmA,
                                                   TmaArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_dyn[];
  __shared__ __align__(8) uint64_t b_rfull[8], b_rempty[8], b_pB[8], b_pconv[8], b_pempty[8];
  __shared__ __align__(8) uint64_t b_tfull[2], b_tempty[2], b_fin, b_bres, b_tail, b_xa, b_xb;
  __shared__ uint32_t tmem_sh;
  __shared__ int abort_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int RS = a.RS, PS = a.PS;
  uint8_t* smem = smem_dyn + ((1024u - (ptx::smem_u32(smem_dyn) & 1023u)) & 1023u);
  uint8_t* raw_ring = smem;
  uint8_t* op_ring = smem + RS * a.rawb;
  const int osb = op_slot_bytes(a.Nc, a.bres);
  uint8_t* barea = op_ring + PS * osb;                      // resident B (bres)
  uint8_t* vring = barea + (a.bres ? a.nk * a.Nc * 64 : 0);
  float* xtab = reinterpret_cast<float*>(vring + vring_bytes(a.epi));   // x tail table
  float* xsc = xtab + a.Npad * 8;                                          // x tail exchange
  volatile int* abort = &abort_sh;

  if (warp == W_MMA) {
    ptx::tmem_alloc(ptx::smem_u32(&tmem_sh), 512u);
    ptx::tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < RS; ++i) {
      ptx::mbar_init(ptx::smem_u32(&b_rfull[i]), 1);
      ptx::mbar_init(ptx::smem_u32(&b_rempty[i]), NCONV);
    }
    for (int i = 0; i < PS; ++i) ptx::mbar_init(ptx::smem_u32(&b_pconv[i]), NCONV);
    for (int i = 0; i < PS / a.G; ++i) {
      ptx::mbar_init(ptx::smem_u32(&b_pB[i]), 1);
      ptx::mbar_init(ptx::smem_u32(&b_pempty[i]), 1);
    }
    for (int i = 0; i < 2; ++i) {
      ptx::mbar_init(ptx::smem_u32(&b_tfull[i]), 1);
      ptx::mbar_init(ptx::smem_u32(&b_tempty[i]), 32 * NEPI);
    }
    ptx::mbar_init(ptx::smem_u32(&b_fin), 1);
    ptx::mbar_init(ptx::smem_u32(&b_bres), 1);
    ptx::mbar_init(ptx::smem_u32(&b_tail), 1);
    ptx::mbar_init(ptx::smem_u32(&b_xa), 128);
    ptx::mbar_init(ptx::smem_u32(&b_xb), 128);
    ptx::fence_mbar_init();
    abort_sh = 0;
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = tmem_sh;
  const int my_tiles =
      blockIdx.x < (unsigned)a.ntiles ? (a.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int nk = a.nk, kb = a.kb;
  const int nrb = (nk + kb - 1) / kb;   // raw boxes per tile
  const uint32_t total = (uint32_t)my_tiles * (uint32_t)nk;

  if (warp == W_PA) {
    // ------------------------------------------------------------ A producer (TMA tensor loads)
    if (lane == 0) {
      ptx::prefetch_tmap(&tmA);
      uint32_t gr = 0;
      for (int i = 0; i < my_tiles; ++i) {
        int c0, c1;
        tile_coords(a, blockIdx.x + i * gridDim.x, c0, c1);
        for (int rb = 0; rb < nrb; ++rb, ++gr) {
          const int r = (int)(gr % RS);
          if (!ptx::mbar_wait_or_abort(ptx::smem_u32(&b_rempty[r]), ((gr / RS) & 1) ^ 1, abort)) goto a_done;
          const uint32_t fb = ptx::smem_u32(&b_rfull[r]);
          const uint32_t dst = ptx::smem_u32(raw_ring + r * a.rawb);
          const int kc = rb * kb * 16;
          ptx::mbar_arrive_expect_tx(fb, (uint32_t)a.rawb);
          if (a.kind == 0) ptx::tma_load_2d(dst, &tmA, kc, c1, fb);
          else ptx::tma_load_3d(dst, &tmA, c0, kc, c1, fb);
        }
      }
    a_done:
      for (uint32_t q = (gr > (uint32_t)RS ? gr - RS : 0u); q < gr; ++q)
        ptx::mbar_wait(ptx::smem_u32(&b_rfull[q % RS]), (q / RS) & 1);
    }
  } else if (warp == W_PB) {
    // ------------------------------------------------------------ B producer (bulk copies)
    if (lane == 0 && a.tw) {
      const uint32_t fb = ptx::smem_u32(&b_tail);
      ptx::mbar_arrive_expect_tx(fb, (uint32_t)(a.Npad * 8 * 4));
      ptx::bulk_load(ptx::smem_u32(xtab), a.tail, (uint32_t)(a.Npad * 8 * 4), fb);
    }
    if (lane == 0 && a.bres) {
      // resident B: every k-step slice once, in the same per-step layout
      const uint32_t fb = ptx::smem_u32(&b_bres);
      ptx::mbar_arrive_expect_tx(fb, (uint32_t)(nk * a.Nc * 64));
      for (int s = 0; s < nk; ++s)
        ptx::bulk_load(ptx::smem_u32(barea + (size_t)s * a.Nc * 64), a.B + (size_t)s * a.Nc * 4,
                       (uint32_t)a.Nc * 64u, fb);
      ptx::mbar_wait(fb, 0u);
    } else if (lane == 0) {
      // streamed B: the slices of one operand group land on that group's barrier
      const int G = a.G, NG = PS / G;
      uint32_t q = 0, qpar = 0, issued = 0;
      for (uint32_t g0 = 0; g0 < total; g0 += G) {
        const uint32_t n = min((uint32_t)G, total - g0);
        if (!ptx::mbar_wait_or_abort(ptx::smem_u32(&b_pempty[q]), qpar ^ 1u, abort)) break;
        const uint32_t fb = ptx::smem_u32(&b_pB[q]);
        ptx::mbar_arrive_expect_tx(fb, n * (uint32_t)a.Nc * 64u);
        for (uint32_t k = 0; k < n; ++k) {
          const uint32_t g = g0 + k;
          const int sl = (int)(g % (uint32_t)nk), p = q * G + (int)k;
          ptx::bulk_load(ptx::smem_u32(op_ring + p * osb + 2 * OPB), a.B + (size_t)sl * a.Nc * 4,
                         (uint32_t)a.Nc * 64u, fb);
        }
        ++issued;
        if (++q == (uint32_t)NG) { q = 0; qpar ^= 1u; }
      }
      // drain: the last (up to NG) groups issued
      uint32_t dq = q, dpar = qpar;
      for (uint32_t k = 0; k < issued && k < (uint32_t)NG; ++k) {
        if (dq == 0) { dq = NG; dpar ^= 1u; }
        --dq;
        ptx::mbar_wait(ptx::smem_u32(&b_pB[dq]), dpar);
      }
    }
    if (lane == 0 && a.tw) ptx::mbar_wait(ptx::smem_u32(&b_tail), 0u);
  } else if (warp >= W_CONV && warp < W_CONV + 8) {
    // ------------------------------------------------------------ converters
    bool ok0 = true;
    // line m, k half h (8 values); a warp holds 32 lines of one half, so the x tail table is
    // read at one address per warp (broadcast)
    const int ct = threadIdx.x - W_CONV * 32;
    const int m = ct & 127, h = ct >> 7;
    if (a.tw && !ptx::mbar_wait_or_abort(ptx::smem_u32(&b_tail), 0u, abort)) ok0 = false;
    uint32_t p = 0, par = 0, r = 0, rpar = 0;
    bool ok = ok0;
    uint64_t tacc[4];                         // x tail columns 256.. as packed pairs
#pragma unroll
    for (int j = 0; j < 4; ++j) tacc[j] = 0ull;
    for (int i = 0; i < my_tiles && ok; ++i) {
      for (int rb = 0; rb < nrb; ++rb) {
        if (!ptx::mbar_wait_or_abort(ptx::smem_u32(&b_rfull[r]), rpar, abort)) { ok = false; break; }
        const int nks = min(kb, nk - rb * kb);
        const uint8_t* rs = raw_ring + r * a.rawb;
        float x[KBMAX][8];
#pragma unroll
        for (int ks = 0; ks < KBMAX; ++ks)
          if (ks < nks) raw_read8(a, rs, m, ks, h, x[ks]);
        ptx::mbar_arrive(ptx::smem_u32(&b_rempty[r]));   // raw slot consumed (values in registers)
        if (++r == (uint32_t)RS) { r = 0; rpar ^= 1u; }
#pragma unroll
        for (int ks = 0; ks < KBMAX; ++ks) {
          if (ks >= nks) break;
          if (a.tw) {
            // FP32 tail columns 256.. of this line: B(k, 256 + j) for the 8 k of (k-step, half)
            const int st = rb * kb + ks;
            const float4* bt = reinterpret_cast<const float4*>(xtab) + (st * 16 + h * 8) * 2;
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
              const float4 b0 = bt[2 * jj], b1 = bt[2 * jj + 1];
              const uint64_t x2 = pack2(x[ks][jj], x[ks][jj]);
              tacc[0] = ffma2(x2, pack2(b0.x, b0.y), tacc[0]);
              tacc[1] = ffma2(x2, pack2(b0.z, b0.w), tacc[1]);
              tacc[2] = ffma2(x2, pack2(b1.x, b1.y), tacc[2]);
              tacc[3] = ffma2(x2, pack2(b1.z, b1.w), tacc[3]);
            }
            if (st == nk - 1) {
              // line done: the upper half hands its partial sums to the lower half through the
              // exchange area (b_xa: written, b_xb: read and free again), which adds, stores
              float4* xl = reinterpret_cast<float4*>(xsc + m * 8);
              const float2 q0 = unpack2(tacc[0]), q1 = unpack2(tacc[1]), q2 = unpack2(tacc[2]),
                           q3 = unpack2(tacc[3]);
              const float ta[8] = {q0.x, q0.y, q1.x, q1.y, q2.x, q2.y, q3.x, q3.y};
              if (h == 1) {
                if (i > 0 && !ptx::mbar_wait_or_abort(ptx::smem_u32(&b_xb), (uint32_t)((i - 1) & 1), abort)) { ok = false; break; }
                xl[0] = make_float4(ta[0], ta[1], ta[2], ta[3]);
                xl[1] = make_float4(ta[4], ta[5], ta[6], ta[7]);
                ptx::mbar_arrive(ptx::smem_u32(&b_xa));
              } else {
                if (!ptx::mbar_wait_or_abort(ptx::smem_u32(&b_xa), (uint32_t)(i & 1), abort)) { ok = false; break; }
                const float4 u0 = xl[0], u1 = xl[1];
                ptx::mbar_arrive(ptx::smem_u32(&b_xb));
                const float t8[8] = {ta[0] + u0.x, ta[1] + u0.y, ta[2] + u0.z, ta[3] + u0.w,
                                     ta[4] + u1.x, ta[5] + u1.y, ta[6] + u1.z, ta[7] + u1.w};
                const int row = (blockIdx.x + i * gridDim.x) * 128 + m;
                if (row < a.rows) {
#pragma unroll
                  for (int g4 = 0; g4 < 2; ++g4) {
                    const int col = 256 + 4 * g4;
                    if (col + 4 > a.L) break;
                    float4* dst = reinterpret_cast<float4*>(a.out + (long long)row * a.X + col);
                    float4 w = make_float4(t8[4 * g4], t8[4 * g4 + 1], t8[4 * g4 + 2], t8[4 * g4 + 3]);
                    if (a.epi == 2) {
                      const float4 o = *dst;
                      w = make_float4(o.x - a.eps * (2.f * o.x - w.x), o.y - a.eps * (2.f * o.y - w.y),
                                      o.z - a.eps * (2.f * o.z - w.z), o.w - a.eps * (2.f * o.w - w.w));
                    }
                    *dst = w;
                  }
                }
              }
#pragma unroll
              for (int j = 0; j < 4; ++j) tacc[j] = 0ull;
            }
          }
          if (p % (uint32_t)a.G == 0 &&
              !ptx::mbar_wait_or_abort(ptx::smem_u32(&b_pempty[p / a.G]), par ^ 1u, abort)) { ok = false; break; }
          uint4 H, Lw;
          split8(x[ks], H, Lw);
          uint8_t* op = op_ring + p * osb;
          *reinterpret_cast<uint4*>(op + kmaj(m, 8 * h)) = H;
          if (a.split) *reinterpret_cast<uint4*>(op + OPB + kmaj(m, 8 * h)) = Lw;
          ptx::fence_proxy_async_smem();
          ptx::mbar_arrive(ptx::smem_u32(&b_pconv[p]));
          if (++p == (uint32_t)PS) { p = 0; par ^= 1u; }
        }
        if (!ok) break;
      }
    }
  } else if (warp == W_MMA) {
    // ------------------------------------------------------------ MMA issuer
    // One thread; tcgen05.mma issue stalls while the previous MMAs run, so the scalar work
    // between k-steps sits on the tensor pipe's critical path: slot and phase counters advance
    // incrementally and the shared-memory descriptors are built once and advanced by offsets
    // (the address field holds addr >> 4 in 14 bits; every operand lies below 256 KB).
    if (lane == 0) {
      uint32_t p = 0, par = 0, gk = 0;
      const int G = a.G;
      const uint64_t dA0 = ptx::smem_desc(ptx::smem_u32(op_ring), 128, 256);
      const uint64_t dR0 = a.bres ? ptx::smem_desc(ptx::smem_u32(barea), 128, 256) : 0ull;
      const uint32_t osb16 = (uint32_t)osb >> 4, opb16 = (uint32_t)OPB >> 4;
      const uint32_t bstep16 = (uint32_t)(a.Nc * 64) >> 4, blo16 = (uint32_t)(a.Nc * 32) >> 4;
      const int n1 = a.Nc > 256 ? a.Nc - 256 : 0;          // columns of the second MMA (x pass)
      const uint32_t id0 = ptx::idesc_bf16(128, a.Nc > 256 ? 256 : a.Nc);
      const uint32_t id1 = n1 ? ptx::idesc_bf16(128, n1) : 0u;
      const uint32_t b1off16 = (256u / 8u) * 256u >> 4;      // B rows 256.. (32 core-matrix groups)
      if (a.bres && !ptx::mbar_wait_or_abort(ptx::smem_u32(&b_bres), 0u, abort)) goto mma_done;
      for (int i = 0; i < my_tiles; ++i) {
        const int ab = a.dbuf ? (i & 1) : 0;
        const uint32_t use = a.dbuf ? (uint32_t)(i >> 1) : (uint32_t)i;
        if (!ptx::mbar_wait_or_abort(ptx::smem_u32(&b_tempty[ab]), (use & 1) ^ 1, abort)) break;
        ptx::tc_fence_after();
        const uint32_t d0 = tmem + (uint32_t)(ab * a.Nc);
        bool ok = true;
        uint64_t dRs = dR0;                                  // resident B of k-step s
        for (int s = 0; s < nk; ++s, ++gk) {
          const uint32_t pg = p % (uint32_t)G;
          if (pg == 0) {
            // the group's last k-step: converters arrive in k-step order, so it implies the rest
            const uint32_t last = p + min((uint32_t)G, total - gk) - 1u;
            if (!ptx::mbar_wait_or_abort(ptx::smem_u32(&b_pconv[last]), par, abort) ||
                (!a.bres && !ptx::mbar_wait_or_abort(ptx::smem_u32(&b_pB[p / G]), par, abort))) {
              ok = false;
              break;
            }
            ptx::tc_fence_after();
          }
          const uint64_t dA = dA0 + p * osb16, dAl = dA + opb16;
          const uint64_t dB = a.bres ? dRs : dA + 2 * opb16, dBl = dB + blo16;
          const uint32_t acc = s > 0 ? 1u : 0u;
          ptx::mma_bf16(d0, dA, dB, id0, acc);
          if (a.split) {
            ptx::mma_bf16(d0, dA, dBl, id0, 1u);
            ptx::mma_bf16(d0, dAl, dB, id0, 1u);
          }
          if (n1) {
            ptx::mma_bf16(d0 + 256u, dA, dB + b1off16, id1, acc);
            if (a.split) {
              ptx::mma_bf16(d0 + 256u, dA, dBl + b1off16, id1, 1u);
              ptx::mma_bf16(d0 + 256u, dAl, dB + b1off16, id1, 1u);
            }
          }
          if (pg == (uint32_t)G - 1u || gk + 1 == total) ptx::mma_commit(ptx::smem_u32(&b_pempty[p / G]));
          dRs += bstep16;
          if (++p == (uint32_t)PS) { p = 0; par ^= 1u; }
        }
        if (!ok) break;
        ptx::mma_commit(ptx::smem_u32(&b_tfull[ab]));
      }
    mma_done:
      ptx::mma_commit(ptx::smem_u32(&b_fin));
    }
  } else {
    // ------------------------------------------------------------ epilogue (warps 0-3, 15-18)
    // Warp w owns TMEM lanes 32(w%4)..+31, i.e. 32 lines of the tile (one line per lane); the
    // two warps of a lane quadrant split the output columns: the first takes chunks [0, nh), the
    // second [nh, nch) (16 columns a chunk).  Chunks are read from TMEM in pairs (32 columns,
    // one wait per pair).
    const int q = warp & 3;
    const int half = warp >= W_EPI2 ? 1 : 0;
    const int ew = half * 4 + q;                             // epilogue warp index 0..7
    const int nch = a.Nc / 16;
    const int nh = (nch + 1) / 2;
    const int cbeg = half ? nh : 0, cend = half ? nch : nh;
    uint8_t* vw = vring + ew * (NBV * VSLOT) + lane * 64;  // this lane's 64 bytes of each v slot
    const int vsw = (lane >> 1) & 3;                        // 16-byte unit swizzle (bank spread)
    for (int i = 0; i < my_tiles; ++i) {
      const int t = blockIdx.x + i * gridDim.x;
      const int ab = a.dbuf ? (i & 1) : 0;
      const uint32_t use = a.dbuf ? (uint32_t)(i >> 1) : (uint32_t)i;
      int c0, c1;
      tile_coords(a, t, c0, c1);
      // this lane's line: base address and the stride between output columns
      bool valid;
      float* gl;
      long long cs;
      if (a.kind == 0) {
        const int row = c1 + q * 32 + lane;
        valid = row < a.rows;
        gl = a.out + (long long)(valid ? row : 0) * a.X;
        cs = 1;
      } else if (a.kind == 1) {
        const int plane = c1 + q, xx = c0 + lane;
        valid = plane < a.ncz && xx < a.X;
        gl = a.out + (valid ? (long long)plane * a.XY + xx : 0);
        cs = a.X;
      } else {
        const int pos = c0 + q * 32 + lane;
        valid = pos < a.XY;
        gl = a.out + (valid ? (long long)c1 * a.N + pos : 0);
        cs = a.XY;
      }
      // update: the old v of this lane's line, chunk c (16 columns), into slot (c - cbeg) % NBV
      auto v_fetch = [&](int c) {
        if (c < cend) {
          uint8_t* dst = vw + ((c - cbeg) % NBV) * VSLOT;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int col = c * 16 + 4 * u;
            const bool in = valid && col + 4 <= a.L;
            ptx::cp_async16(ptx::smem_u32(dst + ((u ^ vsw) << 4)), in ? (const void*)(gl + col) : (const void*)a.out,
                            in ? 16u : 0u);
          }
        }
        ptx::cp_async_commit();
      };
      if (a.epi == 2)
        for (int c = cbeg; c < cbeg + NBV - 1; ++c) v_fetch(c);
      if (!ptx::mbar_wait_or_abort(ptx::smem_u32(&b_tfull[ab]), use & 1, abort)) break;
      ptx::tc_fence_after();
      float sxy = 0.f;
      if (a.kind == 2 && a.epi == 1) {
        const int r = c0 + q * 32 + lane;
        if (r < a.XY) {
          const int ry = r / a.X, rx = r - ry * a.X;
          sxy = a.gamma + a.alpha * (a.lx[rx] + a.ly[ry]);
        }
      }
      const uint32_t trow = tmem + (uint32_t)(ab * a.Nc) + ((uint32_t)(q * 32) << 16);
      for (int cp = cbeg; cp < cend; cp += 2) {
        const int npair = min(2, cend - cp);
        float v[32];
        if (npair == 2) ptx::tmem_ld32(trow + (uint32_t)(cp * 16), v);
        else {
          float* v16 = v;
          ptx::tmem_ld16(trow + (uint32_t)(cp * 16), *reinterpret_cast<float(*)[16]>(v16));
        }
#pragma unroll
        for (int u2 = 0; u2 < 2; ++u2) {
          if (u2 >= npair) break;
          const int c = cp + u2, n0 = c * 16;
          float* vc = v + 16 * u2;
          if (a.epi == 1) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const float den = fmaf(a.alpha, __ldg(a.lz + min(n0 + j, a.L - 1)), sxy);
              vc[j] = __fdividef(vc[j], den * den);
            }
          }
          if (a.epi == 2) {
            v_fetch(c + NBV - 1);
            ptx::cp_async_wait<NBV - 1>();     // chunk c has landed
            const uint8_t* src = vw + ((c - cbeg) % NBV) * VSLOT;
            if (valid) {
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int col = n0 + 4 * u;
                if (col + 4 <= a.L) {
                  float4 w = *reinterpret_cast<const float4*>(src + ((u ^ vsw) << 4));
                  w.x -= a.eps * (2.f * w.x - vc[4 * u]);
                  w.y -= a.eps * (2.f * w.y - vc[4 * u + 1]);
                  w.z -= a.eps * (2.f * w.z - vc[4 * u + 2]);
                  w.w -= a.eps * (2.f * w.w - vc[4 * u + 3]);
                  *reinterpret_cast<float4*>(gl + col) = w;
                }
              }
            }
          } else if (valid) {
            if (a.kind == 0) {
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int col = n0 + 4 * u;
                if (col + 4 <= a.L)
                  *reinterpret_cast<float4*>(gl + col) =
                      make_float4(vc[4 * u], vc[4 * u + 1], vc[4 * u + 2], vc[4 * u + 3]);
              }
            } else {
#pragma unroll
              for (int j = 0; j < 16; ++j)
                if (n0 + j < a.L) gl[(long long)(n0 + j) * cs] = vc[j];
            }
          }
        }
      }
      ptx::tc_fence_before();
      ptx::mbar_arrive(ptx::smem_u32(&b_tempty[ab]));
    }
    if (a.epi == 2) ptx::cp_async_wait<0>();
  }

  // ------------------------------------------------------------ teardown
  __syncthreads();
  if (warp == W_MMA) {
    if (lane == 0) {
      if (!ptx::mbar_wait(ptx::smem_u32(&b_fin), 0u)) abort_sh = 1;
    }
    __syncwarp();
    ptx::tc_fence_after();
    ptx::tmem_dealloc(tmem, 512u);
  }
  if (threadIdx.x == 0 && abort_sh) atomicExch(a.err, 3);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

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

int g_num_sms = 0;

}  // namespace

void* tma_encode_fn() { return reinterpret_cast<void*>(encode_fn()); }

bool tma_pass_supported(const KPlan& kp, int axis) {
  // TMA needs 16-byte row strides: the x extent (x and y passes) or the (y,x) plane (z pass)
  // must be a multiple of 4 floats.  Up to 512 accumulator columns (one TMEM buffer).
  if (!encode_fn()) return false;
  const int L = axis == 0 ? kp.nx : axis == 1 ? kp.ny : kp.nz;
  const long long XY = (long long)kp.nx * kp.ny;
  if (axis == 2) return XY % 4 == 0 && L <= 512;
  return kp.nx % 4 == 0 && L <= 512;
}

// One TMA/tcgen05 pass; the caller checked tma_pass_supported.
cudaError_t tma_axis_pass(const KPlan& kp, int axis, bool inverse, int split, const float* in,
                          float* out, int ncomp, int epi, float eps, cudaStream_t s) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  const long long X = kp.nx, Y = kp.ny, Z = kp.nz, XY = X * Y, N = XY * Z;
  TmaArgs a{};
  a.out = out;
  a.L = axis == 0 ? kp.nx : axis == 1 ? kp.ny : kp.nz;
  a.Npad = (a.L + 15) / 16 * 16;
  a.nk = a.Npad / 16;
  a.B = reinterpret_cast<const uint4*>(kp.tc[axis][inverse ? 1 : 0]);
  a.Nc = a.Npad;
  if (axis == 0 && kp.xtw > 0 && kp.tcx[inverse ? 1 : 0]) {
    // 256 < nx <= 264: 256 columns on the tensor cores (one MMA per product, TMEM double
    // buffer), the rest in FP32 by the converters
    a.Nc = 256;
    a.B = reinterpret_cast<const uint4*>(kp.tcx[inverse ? 1 : 0]);
    a.tail = kp.xtail[inverse ? 1 : 0];
    a.tw = kp.xtw;
  }
  a.kind = axis;
  a.X = (int)X;
  a.XY = (int)XY;
  a.N = N;
  a.epi = epi;
  a.lx = kp.lx; a.ly = kp.ly; a.lz = kp.lz;
  a.alpha = kp.alpha; a.gamma = kp.gamma; a.eps = eps;
  a.split = split;
  a.dbuf = (2 * a.Nc <= 512) ? 1 : 0;
  a.err = kp.err;
  cuuint64_t dims[3], strides[2];
  cuuint32_t box[3], es[3] = {1, 1, 1};
  cuuint32_t rank;
  CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_NONE;
  if (axis == 0) {
    // [rows][X]: box 32 k x 128 rows (16 KB, 2 k-steps), 128-byte rows swizzled so that the
    // converters' 16-byte reads of 8 consecutive rows fall in distinct banks
    a.rows = (int)(ncomp * Y * Z);
    a.ntiles = (a.rows + 127) / 128;
    a.kb = 2;
    rank = 2;
    dims[0] = X; dims[1] = a.rows;
    strides[0] = X * 4;
    box[0] = 32; box[1] = 128;
    swz = CU_TENSOR_MAP_SWIZZLE_128B;
  } else if (axis == 1) {
    // [ncomp*Z][Y][X]: box 32 x by 64 k by 4 planes (32 KB, 4 k-steps)
    a.nxc = (int)((X + 31) / 32);
    a.ncz = (int)(ncomp * Z);
    a.ntiles = a.nxc * ((a.ncz + 3) / 4);
    a.kb = 4;
    rank = 3;
    dims[0] = X; dims[1] = Y; dims[2] = a.ncz;
    strides[0] = X * 4; strides[1] = XY * 4;
    box[0] = 32; box[1] = 64; box[2] = 4;
  } else {
    // [ncomp][Z][XY]: box 128 positions by 64 k (32 KB, 4 k-steps)
    a.tpc = (int)((XY + 127) / 128);
    a.ntiles = a.tpc * ncomp;
    a.kb = 4;
    rank = 3;
    dims[0] = XY; dims[1] = Z; dims[2] = ncomp;
    strides[0] = XY * 4; strides[1] = N * 4;
    box[0] = 128; box[1] = 64; box[2] = 1;
  }
  a.rawb = (int)(box[0] * box[1] * (rank == 3 ? box[2] : 1) * 4);
  CUtensorMap tmA;
  CUresult r = enc(&tmA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, const_cast<float*>(in), dims,
                   strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  // Shared memory (<= 225 KB): B resident when its whole table fits (the y pass); about 96 KB
  // of raw boxes in flight (fewer when that would leave fewer than 4 operand slots); the rest
  // for operand slots (at most 8); the update's v ring.
  const int budget = 225 * 1024 - 1024;
  const int vr = vring_bytes(epi);
  const int bbytes = a.nk * a.Nc * 64;
  a.bres = (bbytes + 2 * a.rawb + 3 * 2 * OPB + vr + tail_bytes(a) <= budget) ? 1 : 0;
  const int osb = op_slot_bytes(a.Nc, a.bres);
  // Raw boxes in flight: 96 KB down to 48 KB, the first depth that leaves 6 operand slots (3
  // groups of G = 2 k-steps); else the shallowest, with what it leaves.
  a.G = 2;
  const int rs_max = (96 * 1024) / a.rawb, rs_min = (48 * 1024 + a.rawb - 1) / a.rawb;
  const int tb = tail_bytes(a);
  auto ps_for = [&](int rs) {
    int ps = (budget - rs * a.rawb - (a.bres ? bbytes : 0) - vr - tb) / osb;
    if (ps > 8) ps = 8;
    return ps - ps % a.G;
  };
  int RS = rs_max;
  while (RS > rs_min && ps_for(RS) < 6) --RS;
  const int PS = ps_for(RS);
  if (PS < 2 * a.G) return cudaErrorNotSupported;
  a.RS = RS;
  a.PS = PS;
  const int smem = smem_bytes(a);
  cudaError_t e = cudaFuncSetAttribute(k_dft_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  if (!g_num_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 148;
  }
  const int grid = a.ntiles < g_num_sms ? a.ntiles : g_num_sms;
  if (grid > 0) k_dft_tma<<<grid, NT, smem, s>>>(tmA, a);
  return cudaGetLastError();
}

}  // namespace lddmm
