// Persistent, warp-specialised tensor-core pass for the per-axis real DFTs of K (§2.4):
//     C(m, n) = sum_k A(m, k) B(k, n)   over all lines m of one axis of a field stack,
// with A the fp32 field (k runs along the transformed axis) and B the padded orthonormal real
// DFT matrix (or its transpose) pre-split into bf16 hi + lo on the host.
//
// Roles inside one CTA (one CTA per SM, 480 threads):
//   warp 12      A producer: per 16-wide k-step one cp.async.bulk.tensor load of the 128-line
//                fp32 slice (zero fill outside the field) into a deep ring of raw slots;
//   warp 13      B producer: one bulk copy of the k-step's B slice into the operand ring;
//   warps 4-11   converters: raw fp32 slice -> bf16 hi + lo (packed round-to-nearest) in K-major
//                core-matrix layout in the operand ring, proxy fence, arrive;
//   warp 14      TMEM owner and MMA issuer (one thread): hi*hi + hi*lo + lo*hi (or hi*hi) per
//                k-step into the tile's TMEM accumulator; tcgen05.commit frees the operand slot,
//                and after the last k-step signals the epilogue;
//   warps 0-3    epilogue: tcgen05.ld (warp w owns TMEM lanes 32w..32w+31), optional symbol
//                scaling or fused update, staging in shared memory, TMA tensor store.  The
//                accumulator is double-buffered in TMEM when 2*Npad <= 512 columns.
// Line tiles (the TMA box): x pass: 128 consecutive x-lines (rows) x 16 k; y pass: 32 x by 4
// (component, z) planes x 16 k; z pass: 128 consecutive (y,x) positions of one component x 16 k.
// Every wait is bounded and observes a CTA-wide abort flag; on abort the kernel drains its
// copies and MMAs, frees TMEM and reports through *err.
#include <cuda.h>
#include <cuda_bf16.h>

#include "kernels.h"
#include "tc_ptx.cuh"

namespace lddmm {

namespace {

constexpr int NT = 480;
constexpr int W_CONV = 4, W_PA = 12, W_PB = 13, W_MMA = 14;
constexpr int NCONV = 256;
constexpr int RAWB = 128 * 16 * 4;   // fp32 A slice
constexpr int OPB = 128 * 16 * 2;    // one bf16 operand slice (hi or lo)
constexpr int NBMAX = 4;            // staging buffers per epilogue warp (at most)
constexpr int WSTGB = 32 * 16 * 4;  // one staging buffer: 32 lines x 16 columns fp32

struct TmaArgs {
  const float* vupd;   // update epilogue: v (read), written through the store map
  const uint4* B;
  int L, Npad, nk;
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
  int RS, PS;          // raw-ring and operand-ring depths
  int bres;            // 1: the whole B table is loaded once and stays in shared memory
  int nb;              // staging buffers per epilogue warp (4 for the update, else 2)
  int* err;
};

// operand slot: A hi and lo, plus the k-step's B slice unless B is resident
__host__ __device__ inline int op_slot_bytes(int Npad, int bres) {
  return 2 * OPB + (bres ? 0 : Npad * 64);
}
__host__ __device__ inline int stage_bytes(int nb) { return 4 * nb * WSTGB; }
__host__ __device__ inline int smem_bytes(int Npad, int RS, int PS, int bres, int nb) {
  return RS * RAWB + PS * op_slot_bytes(Npad, bres) + (bres ? Npad * Npad * 4 : 0) + stage_bytes(nb);
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

__device__ __forceinline__ void named_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void tma_store_2d(const void* tmap, uint32_t src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];"
               ::"l"(tmap), "r"(x), "r"(y), "r"(src) : "memory");
}
__device__ __forceinline__ void tma_store_3d(const void* tmap, uint32_t src, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];"
      ::"l"(tmap), "r"(x), "r"(y), "r"(z), "r"(src) : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// at most n bulk store groups of this thread still reading shared memory (n is 0..3)
__device__ __forceinline__ void bulk_wait_read_le(int n) {
  if (n <= 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
  else if (n == 1) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
  else if (n == 2) asm volatile("cp.async.bulk.wait_group.read 2;" ::: "memory");
  else asm volatile("cp.async.bulk.wait_group.read 3;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// tile coordinates of the TMA box (c0 innermost, c1 outermost) for tile t
__device__ __forceinline__ void tile_coords(const TmaArgs& a, int t, int& c0, int& c1) {
  if (a.kind == 0) { c0 = 0; c1 = t * 128; }
  else if (a.kind == 1) { c0 = (t % a.nxc) * 32; c1 = (t / a.nxc) * 4; }
  else { c0 = (t % a.tpc) * 128; c1 = t / a.tpc; }
}

__global__ void __launch_bounds__(NT, 1) k_dft_tma(const __grid_constant__ CUtensorMap tmA,
                                                   const __grid_constant__ CUtensorMap tmO,
                                                   TmaArgs a) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ __align__(8) uint64_t b_rfull[16], b_rempty[16], b_pB[8], b_pconv[8], b_pempty[8];
  __shared__ __align__(8) uint64_t b_tfull[2], b_tempty[2], b_fin, b_v[4 * NBMAX], b_bres;
  __shared__ uint32_t tmem_sh;
  __shared__ int abort_sh;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int RS = a.RS, PS = a.PS;
  uint8_t* raw_ring = smem;
  uint8_t* op_ring = smem + RS * RAWB;
  const int osb = op_slot_bytes(a.Npad, a.bres);
  uint8_t* barea = op_ring + PS * osb;                      // resident B (bres)
  uint8_t* stage = barea + (a.bres ? a.Npad * a.Npad * 4 : 0);
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
    for (int i = 0; i < PS; ++i) {
      ptx::mbar_init(ptx::smem_u32(&b_pB[i]), 1);
      ptx::mbar_init(ptx::smem_u32(&b_pconv[i]), NCONV);
      ptx::mbar_init(ptx::smem_u32(&b_pempty[i]), 1);
    }
    for (int i = 0; i < 2; ++i) {
      ptx::mbar_init(ptx::smem_u32(&b_tfull[i]), 1);
      ptx::mbar_init(ptx::smem_u32(&b_tempty[i]), 128);
    }
    ptx::mbar_init(ptx::smem_u32(&b_fin), 1);
    ptx::mbar_init(ptx::smem_u32(&b_bres), 1);
    for (int i = 0; i < 4 * NBMAX; ++i) ptx::mbar_init(ptx::smem_u32(&b_v[i]), 1);
    ptx::fence_mbar_init();
    abort_sh = 0;
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = tmem_sh;
  const int my_tiles =
      blockIdx.x < (unsigned)a.ntiles ? (a.ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const int nk = a.nk;
  const uint32_t total = (uint32_t)my_tiles * (uint32_t)nk;

  if (warp == W_PA) {
    // ------------------------------------------------------------ A producer (TMA tensor loads)
    if (lane == 0) {
      ptx::prefetch_tmap(&tmA);
      uint32_t g = 0;
      for (int i = 0; i < my_tiles; ++i) {
        int c0, c1;
        tile_coords(a, blockIdx.x + i * gridDim.x, c0, c1);
        for (int s = 0; s < nk; ++s, ++g) {
          const int r = (int)(g % RS);
          if (!ptx::mbar_wait_or_abort(ptx::smem_u32(&b_rempty[r]), ((g / RS) & 1) ^ 1, abort)) goto a_done;
          const uint32_t fb = ptx::smem_u32(&b_rfull[r]);
          const uint32_t dst = ptx::smem_u32(raw_ring + r * RAWB);
          ptx::mbar_arrive_expect_tx(fb, (uint32_t)RAWB);
          if (a.kind == 0) ptx::tma_load_2d(dst, &tmA, s * 16, c1, fb);
          else ptx::tma_load_3d(dst, &tmA, c0, s * 16, c1, fb);
        }
      }
    a_done:
      for (uint32_t q = (g > (uint32_t)RS ? g - RS : 0u); q < g; ++q)
        ptx::mbar_wait(ptx::smem_u32(&b_rfull[q % RS]), (q / RS) & 1);
    }
  } else if (warp == W_PB) {
    // ------------------------------------------------------------ B producer (bulk copies)
    if (lane == 0 && a.bres) {
      // resident B: every k-step slice once, in the same per-step layout
      const uint32_t fb = ptx::smem_u32(&b_bres);
      ptx::mbar_arrive_expect_tx(fb, (uint32_t)(nk * a.Npad * 64));
      for (int s = 0; s < nk; ++s)
        ptx::bulk_load(ptx::smem_u32(barea + (size_t)s * a.Npad * 64), a.B + (size_t)s * a.Npad * 4,
                       (uint32_t)a.Npad * 64u, fb);
      ptx::mbar_wait(fb, 0u);
    } else if (lane == 0) {
      uint32_t g = 0;
      for (; g < total; ++g) {
        const int s = (int)(g % nk), p = (int)(g % PS);
        if (!ptx::mbar_wait_or_abort(ptx::smem_u32(&b_pempty[p]), ((g / PS) & 1) ^ 1, abort)) break;
        const uint32_t fb = ptx::smem_u32(&b_pB[p]);
        ptx::mbar_arrive_expect_tx(fb, (uint32_t)a.Npad * 64u);
        ptx::bulk_load(ptx::smem_u32(op_ring + p * osb + 2 * OPB), a.B + (size_t)s * a.Npad * 4,
                       (uint32_t)a.Npad * 64u, fb);
      }
      for (uint32_t q = (g > (uint32_t)PS ? g - PS : 0u); q < g; ++q)
        ptx::mbar_wait(ptx::smem_u32(&b_pB[q % PS]), (q / PS) & 1);
    }
  } else if (warp >= W_CONV && warp < W_CONV + 8) {
    // ------------------------------------------------------------ converters
    const int ct = threadIdx.x - W_CONV * 32;
    const int m = ct & 127, h = ct >> 7;     // line, k half (8 values)
    for (uint32_t g = 0; g < total; ++g) {
      const int r = (int)(g % RS), p = (int)(g % PS);
      if (!ptx::mbar_wait_or_abort(ptx::smem_u32(&b_rfull[r]), (g / RS) & 1, abort)) break;
      const float* raw = reinterpret_cast<const float*>(raw_ring + r * RAWB);
      float x[8];
      if (a.kind == 0) {
        const float4* q4 = reinterpret_cast<const float4*>(raw + m * 16 + h * 8);
        const float4 u = q4[0], w = q4[1];
        x[0] = u.x; x[1] = u.y; x[2] = u.z; x[3] = u.w; x[4] = w.x; x[5] = w.y; x[6] = w.z; x[7] = w.w;
      } else if (a.kind == 1) {
        const float* q1 = raw + (m >> 5) * 512 + h * 8 * 32 + (m & 31);
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = q1[j * 32];
      } else {
        const float* q2 = raw + h * 8 * 128 + m;
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = q2[j * 128];
      }
      ptx::mbar_arrive(ptx::smem_u32(&b_rempty[r]));   // raw slot consumed (values in registers)
      uint4 H, Lw;
      split8(x, H, Lw);
      if (!ptx::mbar_wait_or_abort(ptx::smem_u32(&b_pempty[p]), ((g / PS) & 1) ^ 1, abort)) break;
      uint8_t* op = op_ring + p * osb;
      *reinterpret_cast<uint4*>(op + kmaj(m, 8 * h)) = H;
      if (a.split) *reinterpret_cast<uint4*>(op + OPB + kmaj(m, 8 * h)) = Lw;
      ptx::fence_proxy_async_smem();
      ptx::mbar_arrive(ptx::smem_u32(&b_pconv[p]));
    }
  } else if (warp == W_MMA) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t g = 0;
      if (a.bres && !ptx::mbar_wait_or_abort(ptx::smem_u32(&b_bres), 0u, abort)) goto mma_done;
      for (int i = 0; i < my_tiles; ++i) {
        const int ab = a.dbuf ? (i & 1) : 0;
        const uint32_t use = a.dbuf ? (uint32_t)(i >> 1) : (uint32_t)i;
        if (!ptx::mbar_wait_or_abort(ptx::smem_u32(&b_tempty[ab]), (use & 1) ^ 1, abort)) break;
        ptx::tc_fence_after();
        const uint32_t dbase = tmem + (uint32_t)(ab * a.Npad);
        bool ok = true;
        for (int s = 0; s < nk; ++s, ++g) {
          const int p = (int)(g % PS);
          const uint32_t par = (g / PS) & 1;
          if (!ptx::mbar_wait_or_abort(ptx::smem_u32(&b_pconv[p]), par, abort) ||
              (!a.bres && !ptx::mbar_wait_or_abort(ptx::smem_u32(&b_pB[p]), par, abort))) {
            ok = false;
            break;
          }
          ptx::tc_fence_after();
          const uint32_t op = ptx::smem_u32(op_ring + p * osb);
          const uint32_t a_hi = op, a_lo = op + OPB;
          const uint32_t b_hi = a.bres ? ptx::smem_u32(barea + (size_t)s * a.Npad * 64) : op + 2 * OPB;
          const uint32_t b_lo = b_hi + (uint32_t)a.Npad * 32u;
          for (int n0 = 0; n0 < a.Npad; n0 += 256) {
            const int nc = min(256, a.Npad - n0);
            const uint32_t id = ptx::idesc_bf16(128, nc);
            const uint32_t boff = (uint32_t)(n0 / 8) * 256u;
            const uint32_t d = dbase + (uint32_t)n0;
            ptx::mma_bf16(d, ptx::smem_desc(a_hi, 128, 256), ptx::smem_desc(b_hi + boff, 128, 256),
                          id, s > 0 ? 1u : 0u);
            if (a.split) {
              ptx::mma_bf16(d, ptx::smem_desc(a_hi, 128, 256),
                            ptx::smem_desc(b_lo + boff, 128, 256), id, 1u);
              ptx::mma_bf16(d, ptx::smem_desc(a_lo, 128, 256),
                            ptx::smem_desc(b_hi + boff, 128, 256), id, 1u);
            }
          }
          ptx::mma_commit(ptx::smem_u32(&b_pempty[p]));
        }
        if (!ok) break;
        ptx::mma_commit(ptx::smem_u32(&b_tfull[ab]));
      }
    mma_done:
      ptx::mma_commit(ptx::smem_u32(&b_fin));
    }
  } else {
    // ------------------------------------------------------------ epilogue (warps 0-3)
    // Warp q owns TMEM lanes 32q..32q+31 (32 lines of the tile) and its own ring of NB staging
    // buffers (32 lines x 16 columns); lane 0 issues that warp's TMA stores (and, for the update,
    // the TMA loads of v that are prefetched NB-1 chunks ahead).
    const int q = warp;
    const int NB = a.nb;
    uint8_t* wst = stage + q * (NB * WSTGB);
    const uint32_t vbar0 = ptx::smem_u32(&b_v[q * NBMAX]);
    if (lane == 0) ptx::prefetch_tmap(&tmO);
    const int nch = a.Npad / 16;
    uint32_t cc = 0;      // chunks processed by this warp (ring position)
    uint32_t cl = 0;      // v chunks requested by this warp
    for (int i = 0; i < my_tiles; ++i) {
      const int t = blockIdx.x + i * gridDim.x;
      const int ab = a.dbuf ? (i & 1) : 0;
      const uint32_t use = a.dbuf ? (uint32_t)(i >> 1) : (uint32_t)i;
      int c0, c1;
      tile_coords(a, t, c0, c1);
      // store coordinates of this warp's 32 lines
      int s0, s2;
      if (a.kind == 0) { s0 = 0; s2 = c1 + q * 32; }
      else if (a.kind == 1) { s0 = c0; s2 = c1 + q; }
      else { s0 = c0 + q * 32; s2 = c1; }
      // update: prefetch the first NB-1 chunks of v for this tile
      if (a.epi == 2 && lane == 0) {
        for (int c = 0; c < nch && c < NB - 1; ++c, ++cl) {
          const int b = (int)(cl % NB);
          bulk_wait_read_le(0);   // every earlier store has finished reading its buffer
          ptx::mbar_arrive_expect_tx(vbar0 + 8u * b, (uint32_t)WSTGB);
          ptx::tma_load_2d(ptx::smem_u32(wst + b * WSTGB), &tmO, c * 16, s2, vbar0 + 8u * b);
        }
      }
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
      const uint32_t trow = tmem + (uint32_t)(ab * a.Npad) + ((uint32_t)(q * 32) << 16);
      bool ok = true;
      for (int c = 0; c < nch; ++c, ++cc) {
        const int n0 = c * 16;
        const int b = (int)(cc % NB);
        float* sg = reinterpret_cast<float*>(wst + b * WSTGB);
        float v[16];
        ptx::tmem_ld16(trow + (uint32_t)n0, v);
        if (a.epi == 1) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float den = fmaf(a.alpha, a.lz[min(n0 + j, a.L - 1)], sxy);
            v[j] = __fdividef(v[j], den * den);
          }
        }
        if (a.epi == 2) {
          // v chunk c sits in buffer b (requested in order, one per chunk)
          if (!ptx::mbar_wait_or_abort(vbar0 + 8u * b, (cc / NB) & 1, abort)) { ok = false; break; }
          float4* r4 = reinterpret_cast<float4*>(sg + lane * 16);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            float4 w = r4[j];
            w.x -= a.eps * (2.f * w.x - v[4 * j]);
            w.y -= a.eps * (2.f * w.y - v[4 * j + 1]);
            w.z -= a.eps * (2.f * w.z - v[4 * j + 2]);
            w.w -= a.eps * (2.f * w.w - v[4 * j + 3]);
            r4[j] = w;
          }
        } else {
          // buffer b is free once the store issued NB chunks ago finished reading it
          if (lane == 0) bulk_wait_read_le(NB - 1);
          __syncwarp();
          if (a.kind == 0) {
            float4* d4 = reinterpret_cast<float4*>(sg + lane * 16);
#pragma unroll
            for (int j = 0; j < 4; ++j) d4[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) sg[j * 32 + lane] = v[j];
          }
        }
        ptx::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          const uint32_t src = ptx::smem_u32(sg);
          if (a.kind == 0) tma_store_2d(&tmO, src, n0, s2);
          else tma_store_3d(&tmO, src, s0, n0, s2);
          bulk_commit();
          // update: request v chunk c + NB - 1 into the buffer freed NB-1 stores ago
          if (a.epi == 2 && c + NB - 1 < nch) {
            const int bn = (int)(cl % NB);
            bulk_wait_read_le(1);   // the store of chunk c-1 (same buffer) is done reading
            ptx::mbar_arrive_expect_tx(vbar0 + 8u * bn, (uint32_t)WSTGB);
            ptx::tma_load_2d(ptx::smem_u32(wst + bn * WSTGB), &tmO, (c + NB - 1) * 16, s2, vbar0 + 8u * bn);
            ++cl;
          }
        }
        __syncwarp();
      }
      if (!ok) break;
      ptx::tc_fence_before();
      ptx::mbar_arrive(ptx::smem_u32(&b_tempty[ab]));
    }
    if (lane == 0) bulk_wait_all();
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
  a.vupd = out;
  a.L = axis == 0 ? kp.nx : axis == 1 ? kp.ny : kp.nz;
  a.Npad = (a.L + 15) / 16 * 16;
  a.nk = a.Npad / 16;
  a.B = reinterpret_cast<const uint4*>(kp.tc[axis][inverse ? 1 : 0]);
  a.kind = axis;
  a.X = (int)X;
  a.XY = (int)XY;
  a.N = N;
  a.epi = epi;
  a.lx = kp.lx; a.ly = kp.ly; a.lz = kp.lz;
  a.alpha = kp.alpha; a.gamma = kp.gamma; a.eps = eps;
  a.split = split;
  a.dbuf = (2 * a.Npad <= 512) ? 1 : 0;
  a.err = kp.err;
  cuuint64_t dims[3], strides[2];
  cuuint32_t box[3], es[3] = {1, 1, 1};
  cuuint32_t rank;
  if (axis == 0) {
    a.rows = (int)(ncomp * Y * Z);
    a.ntiles = (a.rows + 127) / 128;
    rank = 2;
    dims[0] = X; dims[1] = a.rows;
    strides[0] = X * 4;
    box[0] = 16; box[1] = 128;
  } else if (axis == 1) {
    a.nxc = (int)((X + 31) / 32);
    a.ncz = (int)(ncomp * Z);
    a.ntiles = a.nxc * ((a.ncz + 3) / 4);
    rank = 3;
    dims[0] = X; dims[1] = Y; dims[2] = a.ncz;
    strides[0] = X * 4; strides[1] = XY * 4;
    box[0] = 32; box[1] = 16; box[2] = 4;
  } else {
    a.tpc = (int)((XY + 127) / 128);
    a.ntiles = a.tpc * ncomp;
    rank = 3;
    dims[0] = XY; dims[1] = Z; dims[2] = ncomp;
    strides[0] = XY * 4; strides[1] = N * 4;
    box[0] = 128; box[1] = 16; box[2] = 1;
  }
  CUtensorMap tmA, tmO;
  CUresult r = enc(&tmA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, const_cast<float*>(in), dims,
                   strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  // stores (and v loads of the update) move 32 lines x 16 columns per epilogue warp
  cuuint32_t obox[3];
  if (axis == 0) { obox[0] = 16; obox[1] = 32; }
  else if (axis == 1) { obox[0] = 32; obox[1] = 16; obox[2] = 1; }
  else { obox[0] = 32; obox[1] = 16; obox[2] = 1; }
  r = enc(&tmO, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, out, dims, strides, obox, es,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  // Shared memory (<= 225 KB): 6 raw slots for the TMA loads (measured: deeper raw rings at
  // the expense of operand slots are slower), 4 staging buffers per epilogue warp, B resident
  // when its whole table fits (the y pass) or streamed with the operand slots, and the rest of
  // the budget for operand slots (at most 8).
  const int budget = 225 * 1024;
  a.nb = 4;
  const int stg = stage_bytes(a.nb);
  const int bbytes = a.Npad * a.Npad * 4;
  a.RS = 6;
  a.bres = (a.RS * RAWB + bbytes + 3 * 2 * OPB + stg <= budget) ? 1 : 0;
  int PS = (budget - a.RS * RAWB - (a.bres ? bbytes : 0) - stg) / op_slot_bytes(a.Npad, a.bres);
  if (PS > 8) PS = 8;
  if (PS < 2) return cudaErrorNotSupported;
  a.PS = PS;
  const int smem = smem_bytes(a.Npad, a.RS, a.PS, a.bres, a.nb);
  cudaError_t e = cudaFuncSetAttribute(k_dft_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  if (!g_num_sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (g_num_sms <= 0) g_num_sms = 148;
  }
  const int grid = a.ntiles < g_num_sms ? a.ntiles : g_num_sms;
  if (grid > 0) k_dft_tma<<<grid, NT, smem, s>>>(tmA, tmO, a);
  return cudaGetLastError();
}

}  // namespace lddmm
