// The smoothing operator K = (gamma - alpha Lap_h)^-2 of §2.4 (K = (L^T L)^-1 for
// L = -alpha Lap + gamma), applied on the periodic grid as separable per-axis real DFTs.
//
// For an axis of length n, R is the orthonormal real Fourier basis (rows: constant, then
// cos/sin pairs of frequency k = 1.., then the Nyquist cosine when n is even).  The symbol of
// K depends on each frequency only through lambda(k) = sum_d (2 - 2 cos(2 pi k_d / n_d)) / h_d^2,
// which is the same for the cos and the sin row of a pair, so with R3 = Rz (x) Ry (x) Rx
//     K = R3^T diag((gamma + alpha lambda)^-2) R3.
// Each axis transform is a dense matrix product over all lines of that axis: a batched GEMM
// whose small operand is R (n x n) and whose large operand is the field.  The symbol scaling is
// fused into the epilogue of the forward z product.
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/lddmm.h"
#include "kernels.h"

namespace lddmm {

// ---------------------------------------------------------------------------------------------
// Table construction (host, double precision, angles reduced modulo n).
static void real_dft_matrix(int n, double h, std::vector<float>& R, std::vector<float>& lam) {
  R.assign((size_t)n * n, 0.f);
  lam.assign(n, 0.f);
  const double two_pi = 6.283185307179586476925286766559;
  for (int r = 0; r < n; ++r) {
    const int k = (r + 1) / 2;
    const bool is_sin = (r > 0) && (r % 2 == 0);
    const bool nyq = (n % 2 == 0) && (r == n - 1);
    const double scale = (r == 0 || nyq) ? std::sqrt(1.0 / n) : std::sqrt(2.0 / n);
    for (int m = 0; m < n; ++m) {
      const double ang = two_pi * (double)(((long long)k * m) % n) / (double)n;
      R[(size_t)r * n + m] = (float)(scale * (is_sin ? std::sin(ang) : std::cos(ang)));
    }
    lam[r] = (float)((2.0 - 2.0 * std::cos(two_pi * (double)k / (double)n)) / (h * h));
  }
}

void host_real_dft_tables(int n, double h, std::vector<float>& R, std::vector<float>& lam) {
  real_dft_matrix(n, h, R, lam);
}

static uint16_t bf16_rn(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;
  return (uint16_t)(u >> 16);
}
static float bf16_to_f(uint16_t b) {
  uint32_t u = (uint32_t)b << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

// Tensor-core operand table: B(k, n) = R[n][k] (forward) or R[k][n] (inverse) for the output
// columns n < rows (rows a multiple of 16; zero for n >= n_len), k zero-padded to ceil16(n_len);
// per 16-wide k-step a bf16 hi block then a bf16 lo block (B = hi + lo), each rows x 16 k in the
// K-major no-swizzle core-matrix order the MMA descriptors expect:
// element (row, kk) at byte (kk/8)*128 + (row/8)*256 + (row%8)*16 + (kk%8)*2.
static void tc_table(const std::vector<float>& R, int n, bool inverse, int rows,
                     std::vector<uint16_t>& t) {
  const int Kpad = (n + 15) / 16 * 16, nk = Kpad / 16;
  const size_t block = (size_t)rows * 16;  // elements per hi (or lo) block
  t.assign((size_t)nk * 2 * block, 0);
  for (int s = 0; s < nk; ++s) {
    uint16_t* hi = t.data() + (size_t)s * 2 * block;
    uint16_t* lo = hi + block;
    for (int row = 0; row < rows; ++row)
      for (int kk = 0; kk < 16; ++kk) {
        const int k = s * 16 + kk;
        float b = 0.f;
        if (k < n && row < n) b = inverse ? R[(size_t)k * n + row] : R[(size_t)row * n + k];
        const uint16_t bh = bf16_rn(b);
        const uint16_t bl = bf16_rn(b - bf16_to_f(bh));
        const size_t off = ((size_t)(kk / 8) * 128 + (size_t)(row / 8) * 256 + (row % 8) * 16 +
                            (kk % 8) * 2) / 2;
        hi[off] = bh;
        lo[off] = bl;
      }
  }
}

// Operand table of the pre-split pass: B(k, n) as bf16 [hi plane][lo plane], each [Nc][Kp]
// row-major (row n = output column, k contiguous), Nc = Kp = ceil16(n), zero for n >= n_len or
// k >= n_len.
static void ks_table(const std::vector<float>& R, int n, bool inverse, std::vector<uint16_t>& t) {
  const int Kp = (n + 15) / 16 * 16, Nc = Kp;
  const size_t plane = (size_t)Nc * Kp;
  t.assign(2 * plane, 0);
  for (int row = 0; row < n && row < Nc; ++row)
    for (int k = 0; k < n; ++k) {
      const float b = inverse ? R[(size_t)k * n + row] : R[(size_t)row * n + k];
      const uint16_t bh = bf16_rn(b);
      t[(size_t)row * Kp + k] = bh;
      t[plane + (size_t)row * Kp + k] = bf16_rn(b - bf16_to_f(bh));
    }
}

template <typename T>
static cudaError_t upload(T** dst, const std::vector<T>& src) {
  cudaError_t e = cudaMalloc((void**)dst, src.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

cudaError_t kplan_create(KPlan* kp, int nx, int ny, int nz, float hx, float hy, float hz,
                         float alpha, float gamma) {
  *kp = KPlan{};
  kp->nx = nx; kp->ny = ny; kp->nz = nz;
  kp->alpha = alpha; kp->gamma = gamma;
  const int n[3] = {nx, ny, nz};
  const double h[3] = {hx, hy, hz};
  float** Rs[3] = {&kp->Rx, &kp->Ry, &kp->Rz};
  float** ls[3] = {&kp->lx, &kp->ly, &kp->lz};
  for (int d = 0; d < 3; ++d) {
    std::vector<float> R, lam;
    real_dft_matrix(n[d], h[d], R, lam);
    lam.resize((size_t)(n[d] + 15) / 16 * 16, 0.f);   // zero padded: 16-column groups load whole
    cudaError_t e;
    if ((e = upload(Rs[d], R)) != cudaSuccess) return e;
    if ((e = upload(ls[d], lam)) != cudaSuccess) return e;
    for (int dir = 0; dir < 2; ++dir) {
      std::vector<uint16_t> t;
      tc_table(R, n[d], dir == 1, (n[d] + 15) / 16 * 16, t);
      if ((e = upload(&kp->tc[d][dir], t)) != cudaSuccess) return e;
    }
    if (n[d] <= (d == 0 ? 264 : 256)) {
      for (int dir = 0; dir < 2; ++dir) {
        std::vector<uint16_t> t;
        ks_table(R, n[d], dir == 1, t);
        if ((e = upload(&kp->ks[d][dir], t)) != cudaSuccess) return e;
      }
    }
  }
  cudaError_t e = cudaMalloc((void**)&kp->err, sizeof(int));
  if (e != cudaSuccess) return e;
  return cudaMemset(kp->err, 0, sizeof(int));
}

void kplan_destroy(KPlan* kp) {
  void* ps[] = {kp->Rx, kp->Ry, kp->Rz, kp->lx, kp->ly, kp->lz, kp->err};
  for (void* p : ps)
    if (p) cudaFree(p);
  for (int d = 0; d < 3; ++d)
    for (int dir = 0; dir < 2; ++dir)
      if (kp->tc[d][dir]) cudaFree(kp->tc[d][dir]);
  for (int dir = 0; dir < 2; ++dir) {
    for (int d = 0; d < 3; ++d)
      if (kp->ks[d][dir]) cudaFree(kp->ks[d][dir]);
  }
  *kp = KPlan{};
}

// ---------------------------------------------------------------------------------------------
// FP32 batched GEMM on the CUDA cores: C_b(m,n) = sum_k A_b(m,k) B_b(k,n), arbitrary strides.
// 64x64 output tile per block, k-slices of 16 staged in shared memory, 4x4 per thread.
struct GemmArgs {
  int M, N, K, batch;
  const float* A; long long sAb, sAm, sAk;
  const float* B; long long sBb, sBk, sBn;
  float* C; long long sCb, sCm, sCn;
  // optional symbol epilogue (forward z): C(m,n) *= (gamma + alpha (lz[m] + ly[n/nx] + lx[n%nx]))^-2
  const float* lx; const float* ly; const float* lz; int nx; float alpha, gamma;
};

constexpr int TBM = 64, TBN = 64, TBK = 16;

__global__ void __launch_bounds__(256) k_sgemm(GemmArgs a) {
  __shared__ float As[TBK][TBM + 4];
  __shared__ float Bs[TBK][TBN + 4];
  const int b = blockIdx.z;
  const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * TBN;
  const float* A = a.A + b * a.sAb;
  const float* B = a.B + b * a.sBb;
  float* C = a.C + b * a.sCb;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  float acc[4][4] = {};
  const bool a_kfast = (a.sAk == 1);
  const bool b_nfast = (a.sBn == 1);
  for (int k0 = 0; k0 < a.K; k0 += TBK) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int e = tid + i * 256;
      int mm, kk;
      if (a_kfast) { mm = e / TBK; kk = e % TBK; } else { kk = e / TBM; mm = e % TBM; }
      const int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < a.M && gk < a.K) ? A[gm * a.sAm + gk * a.sAk] : 0.f;
      int nn, kb;
      if (b_nfast) { kb = e / TBN; nn = e % TBN; } else { nn = e / TBK; kb = e % TBK; }
      const int gn = n0 + nn, gk2 = k0 + kb;
      Bs[kb][nn] = (gn < a.N && gk2 < a.K) ? B[gk2 * a.sBk + gn * a.sBn] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TBK; ++kk) {
      float av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= a.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= a.N) continue;
      float v = acc[i][j];
      if (a.lz) {
        const float lam = a.lz[gm] + a.ly[gn / a.nx] + a.lx[gn % a.nx];
        const float den = a.gamma + a.alpha * lam;
        v = v / (den * den);
      }
      C[gm * a.sCm + gn * a.sCn] = v;
    }
  }
}

static void sgemm(const GemmArgs& a, cudaStream_t s) {
  dim3 grid((a.N + TBN - 1) / TBN, (a.M + TBM - 1) / TBM, a.batch);
  k_sgemm<<<grid, 256, 0, s>>>(a);
}

static GemmArgs gemm_x(const KPlan& kp, int ncomp, const float* in, float* out, bool fwd) {
  // rows of length nx: out[row][n] = sum_k in[row][k] B(k,n); B(k,n) = R[n][k] (fwd) or R[k][n]
  const int L = kp.nx;
  GemmArgs a{};
  a.M = ncomp * kp.ny * kp.nz; a.N = L; a.K = L; a.batch = 1;
  a.A = in; a.sAm = L; a.sAk = 1;
  a.B = kp.Rx;
  if (fwd) { a.sBk = 1; a.sBn = L; } else { a.sBk = L; a.sBn = 1; }
  a.C = out; a.sCm = L; a.sCn = 1;
  return a;
}

static GemmArgs gemm_left(const float* R, int L, long long stride_k, long long ncols,
                          int batch, long long sbatch, const float* in, float* out, bool fwd) {
  // out_b[r][n] = sum_m A(r,m) in_b[m][n]; A = R (fwd) or R^T (inverse)
  GemmArgs a{};
  a.M = L; a.K = L; a.N = (int)ncols; a.batch = batch;
  a.A = R;
  if (fwd) { a.sAm = L; a.sAk = 1; } else { a.sAm = 1; a.sAk = L; }
  a.sAb = 0;
  a.B = in; a.sBb = sbatch; a.sBk = stride_k; a.sBn = 1;
  a.C = out; a.sCb = sbatch; a.sCm = stride_k; a.sCn = 1;
  return a;
}

static cudaError_t apply_K_fp32(const KPlan& kp, const float* in, float* out, float* work,
                                int ncomp, cudaStream_t s, const Hook& hook) {
  const long long nxy = (long long)kp.nx * kp.ny;
  const long long N = nxy * kp.nz;
  // forward x: in -> work
  hook(KID_KX_FWD, 0);
  sgemm(gemm_x(kp, ncomp, in, work, true), s);
  hook(KID_KX_FWD, 1);
  // forward y: work -> out   (batches: ncomp * nz planes of ny x nx)
  hook(KID_KY_FWD, 0);
  sgemm(gemm_left(kp.Ry, kp.ny, kp.nx, kp.nx, ncomp * kp.nz, nxy, work, out, true), s);
  hook(KID_KY_FWD, 1);
  // forward z with the symbol: out -> work (batches: ncomp volumes, nz x (ny nx))
  {
    GemmArgs a = gemm_left(kp.Rz, kp.nz, nxy, nxy, ncomp, N, out, work, true);
    a.lx = kp.lx; a.ly = kp.ly; a.lz = kp.lz; a.nx = kp.nx;
    a.alpha = kp.alpha; a.gamma = kp.gamma;
    hook(KID_KZ_SYM, 0);
    sgemm(a, s);
    hook(KID_KZ_SYM, 1);
  }
  // inverse z: work -> out
  hook(KID_KZ_INV, 0);
  sgemm(gemm_left(kp.Rz, kp.nz, nxy, nxy, ncomp, N, work, out, false), s);
  hook(KID_KZ_INV, 1);
  // inverse y: out -> work
  hook(KID_KY_INV, 0);
  sgemm(gemm_left(kp.Ry, kp.ny, kp.nx, kp.nx, ncomp * kp.nz, nxy, out, work, false), s);
  hook(KID_KY_INV, 1);
  // inverse x: work -> out
  hook(KID_KX_INV, 0);
  sgemm(gemm_x(kp, ncomp, work, out, false), s);
  hook(KID_KX_INV, 1);
  return cudaGetLastError();
}

// Tensor-core K over pre-split intermediate fields.  Every pass reads its input with the
// transformed axis contiguous and writes its output in the next pass's line order:
//   x fwd:  [c][z][y][x]  (split, x rows, pitch Px)  -> [c][x'][Pz][y] (split, y rows, pitch Py)
//   y fwd:                                            -> [c][x'][y'][z] (split, z rows, pitch Pz)
//   z fwd + symbol:                                   -> [c][x'][y'][z'] (split, same order)
//   z inv:                                            -> [c][z][x'][y'] (split, y rows, pitch Py)
//   y inv:                                            -> [c][z][y][x']  (split, x rows, pitch Px)
//   x inv:                                            -> fp32 [c][z][y][x], or the update of v
// The buffers alternate between work and out (in may alias out).  A plain fp32 input is first
// split into work; without the update the result then lands in work and is copied to out.
// The x forward output holds Pz (z rounded up to 8) planes per x' so that the y forward pass
// runs over Pz lines per output row: its 8-line output pieces then start 16-byte aligned (the
// staged epilogue).  Lines z >= nz are never written by the x pass and read whatever the buffer
// holds; the y pass stores their results into the pitch padding of the z rows, which no later
// pass reads (rows of a product are independent).
static cudaError_t apply_K_ks(const KPlan& kp, int split, const float* in, float* out,
                              float* work, int ncomp, cudaStream_t s, const Hook& hook,
                              void* v_upd, float eps, bool in_split, int upd_kind = KS_OUT_UPD) {
  const long long X = kp.nx, Y = kp.ny, Z = kp.nz, C = ncomp;
  const long long Px = ks_pitch(kp.nx), Py = ks_pitch(kp.ny), Pz = ks_pitch(kp.nz);
  cudaError_t e;
  float* bA = work;   // receives the x forward product
  float* bB = out;
  const void* src = in;
  if (!in_split) {
    const KsOut o0{KS_OUT_SPLIT, 0, work, C * Z * Y * Px, 1, 1, 1, Px, 1};
    if ((e = ks_split_rows(in, C * Z * Y, kp.nx, split, o0, s)) != cudaSuccess) return e;
    src = work;
    bA = out;
    bB = work;
  }
  // z forward, symbol and z inverse run as one fused pass when the z inverse output rows (y
  // lines) hold a multiple of 8 lines; its output then lands where the z inverse pass puts it
  const bool zz = Y % 8 == 0;
  struct Pass2 {
    int kid, axis;
    bool inv, zz;
    long long nlines;
    KsOut o;
  };
  const Pass2 ps[5] = {
      {KID_KX_FWD, 0, false, false, C * Z * Y, {KS_OUT_SPLIT, 0, bA, C * X * Pz * Py, Z, Y, X * Pz, Py, Pz * Py}},
      {KID_KY_FWD, 1, false, false, C * X * Pz, {KS_OUT_SPLIT, 0, bB, C * X * Y * Pz, 1, Pz, Y, Pz, Pz}},
      {KID_KZ_SYM, 2, false, false, C * X * Y, {KS_OUT_SPLIT, 1, bA, C * X * Y * Pz, 1, 1, 1, Pz, 1}},
      {zz ? KID_KZ_FUSED : KID_KZ_INV, 2, true, zz, C * X * Y,
       {KS_OUT_SPLIT, 0, zz ? bA : bB, C * Z * X * Py, X, Y, Z * X, Py, X * Py}},
      {KID_KY_INV, 1, true, false, C * Z * X, {KS_OUT_SPLIT, 0, zz ? bB : bA, C * Z * Y * Px, 1, X, Y, Px, Px}}};
  for (int p = 0; p < 5; ++p) {
    if (zz && p == 2) continue;
    hook(ps[p].kid, 0);
    e = ks_axis_pass(kp, ps[p].axis, ps[p].inv, split, src, ps[p].nlines, ps[p].o, 0.f, s,
                     ps[p].zz);
    hook(ps[p].kid, 1);
    if (e != cudaSuccess) return e;
    src = ps[p].o.out;
  }
  // x inverse: from the last output into v_upd (update) or fp32 rows in the other buffer
  void* dst = v_upd ? v_upd : (void*)(src == bA ? bB : bA);
  const KsOut o6{v_upd ? upd_kind : KS_OUT_F32, 0, dst, 0, 1, 1, 1, X, 1};
  hook(KID_KX_INV, 0);
  e = ks_axis_pass(kp, 0, true, split, src, C * Z * Y, o6, eps, s);
  hook(KID_KX_INV, 1);
  if (e != cudaSuccess) return e;
  if (!v_upd && dst != out)
    e = cudaMemcpyAsync(out, dst, (size_t)C * X * Y * Z * sizeof(float), cudaMemcpyDeviceToDevice, s);
  return e;
}

cudaError_t apply_K_update_bf16(const KPlan& kp, int mode, const float* in, float* work,
                                cudaStream_t s, const Hook& hook, void* v_bf16, float eps,
                                long long cap, bool in_split) {
  if (!ks_path(kp, mode, 3, cap)) return cudaErrorNotSupported;
  return apply_K_ks(kp, mode == LDDMM_K_BF16X3 ? 1 : 0, in, const_cast<float*>(in), work, 3, s,
                    hook, v_bf16, eps, in_split, KS_OUT_UPD_BF16);
}

bool ks_path(const KPlan& kp, int mode, int ncomp, long long cap) {
  if (mode != LDDMM_K_BF16X3 && mode != LDDMM_K_BF16) return false;
  const long long N = (long long)kp.nx * kp.ny * kp.nz;
  if (cap <= 0) cap = (long long)ncomp * N;
  return ks_supported(kp) && cap >= ks_field_floats(kp.nx, kp.ny, kp.nz, ncomp);
}

static cudaError_t apply_K_tc(const KPlan& kp, int split, const float* in, float* out,
                              float* work, int ncomp, cudaStream_t s, const Hook& hook,
                              float* v_upd, float eps, long long cap, bool in_split) {
  if (ks_path(kp, split ? LDDMM_K_BF16X3 : LDDMM_K_BF16, ncomp, cap))
    return apply_K_ks(kp, split, in, out, work, ncomp, s, hook, v_upd, eps, in_split);
  if (in_split) return cudaErrorInvalidValue;
  cudaError_t e;
#define TC_PASS(kid, axis, inv, src, dst, epi)                                         \
  do {                                                                                 \
    hook(kid, 0);                                                                      \
    e = tc_axis_pass(kp, axis, inv, split, src, dst, ncomp, epi, eps, s);              \
    hook(kid, 1);                                                                      \
    if (e != cudaSuccess) return e;                                                    \
  } while (0)
  TC_PASS(KID_KX_FWD, 0, false, in, work, 0);
  TC_PASS(KID_KY_FWD, 1, false, work, out, 0);
  TC_PASS(KID_KZ_SYM, 2, false, out, work, 1);
  TC_PASS(KID_KZ_INV, 2, true, work, out, 0);
  TC_PASS(KID_KY_INV, 1, true, out, work, 0);
  if (v_upd) TC_PASS(KID_KX_INV, 0, true, work, v_upd, 2);
  else TC_PASS(KID_KX_INV, 0, true, work, out, 0);
#undef TC_PASS
  return cudaSuccess;
}

cudaError_t apply_K(const KPlan& kp, int mode, const float* in, float* out, float* work,
                    int ncomp, cudaStream_t s, const Hook& hook, float* v_upd, float eps,
                    long long cap, bool in_split) {
  switch (mode) {
    case LDDMM_K_FP32: {
      if (in_split) return cudaErrorInvalidValue;
      cudaError_t e = apply_K_fp32(kp, in, out, work, ncomp, s, hook);
      if (e != cudaSuccess || !v_upd) return e;
      Grid g{kp.nx, kp.ny, kp.nz, kp.nx * kp.ny * kp.nz};
      hook(KID_UPDATE, 0);
      launch_update(g, v_upd, out, eps, s, 0);
      hook(KID_UPDATE, 1);
      return cudaGetLastError();
    }
    case LDDMM_K_BF16X3:
      return apply_K_tc(kp, 1, in, out, work, ncomp, s, hook, v_upd, eps, cap, in_split);
    case LDDMM_K_BF16:
      return apply_K_tc(kp, 0, in, out, work, ncomp, s, hook, v_upd, eps, cap, in_split);
    default:
      return cudaErrorNotSupported;
  }
}

}  // namespace lddmm
