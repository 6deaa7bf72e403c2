// Host-side launch wrappers for the liblddmm kernels (one translation unit per kernel family).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace lddmm {

// Accumulators written by the reduction kernels (device memory, reset per iteration).
struct Acc {
  double e_reg;       // sum_j sum_x |(gamma - alpha Lap_h) v_j|^2   (unscaled)
  double e_data;      // sum_x M (J0_T - I1)^2                       (unscaled)
  int min_det_ord;    // ordered-int encoding of min det D phi_{j,1}
  int nonfinite;      // set when a reduction saw NaN/Inf
};

// Optional timing hook: mark(user, kernel_id, 0) before and mark(user, kernel_id, 1) after
// every kernel launch (the host records CUDA events on the launching stream).
struct Hook {
  void (*mark)(void* user, int kernel_id, int phase) = nullptr;
  void* user = nullptr;
  void operator()(int id, int phase) const {
    if (mark) mark(user, id, phase);
  }
};

enum KernelId {
  KID_BACK_DISP = 0, KID_BACK_TERMS, KID_FWD_TERMS, KID_FWD_FLOW, KID_KX_FWD, KID_KY_FWD,
  KID_KZ_SYM, KID_KZ_INV, KID_KY_INV, KID_KX_INV, KID_UPDATE, KID_EREG, KID_KZ_FUSED,
  KID_FWD_FUSED, KID_J0_EDATA, KID_COUNT
};

// ---- flows (kernels_flow.cu) ----
// Velocity fields and images (vj, I0, I1, M) are stored as float (st = 0) or bf16 (st = 1);
// displacements, J1, W, b and all arithmetic are float.  Maps (displacements) are planar,
// [3][N], or, with quad = 1, [N] x (u_x, u_y, u_z, 0) (16 bytes a voxel): the iteration's
// backward sweep (launch_flow_back) and the map phi_{0,1} it leaves use the quad layout, the
// forward sweep (launch_fwd_fused) and phi_{1,0} the planar one.
// Backward sweep step j (quad maps): u_cur = dt v_j / h + u_next(x + dt v_j / h)
// (u_next == nullptr: id), then J1_j = I1 o phi, W_j = (M o phi) det(I + Du_cur), min det into
// acc.  IM holds I1 and M interleaved as pairs (launch_interleave).
void launch_flow_back(const Grid& g, const void* vj, const float* u_next, float* u_cur,
                      const void* IM, float* J1j, float* Wj, float dtx, float dty, float dtz,
                      Acc* acc, cudaStream_t s, const Hook& hook, int st, int rk = 0);
// out[i] = (a[i], b[i]) as storage-type pairs.
void launch_interleave(const void* a, const void* b, void* out, int64_t n, cudaStream_t s,
                       int st);
// Forward sweep step j: u_next = -dt v_j / h + u_cur(x - dt v_j / h) (u_cur == nullptr: id);
// if last, J0_T = I0 o (id + u_next) and E_data.
void launch_fwd_flow(const Grid& g, const void* vj, const float* u_cur, float* u_next,
                     float dtx, float dty, float dtz, bool last, const void* I0, const void* I1,
                     const void* M, float* J0T, Acc* acc, cudaStream_t s, int st, int rk = 0,
                     int quad = 0);
// Forward sweep step j (planar maps) in one pass over u_cur = phi_{j,0} - id (nullptr: id): the residual
// b = c W_j (J0_j - J1_j) grad J0_j / h with J0_j = I0 o (id + u_cur) (bsplit 0: b as 3 fp32
// fields; 1 / 2: b split for the pre-split K, bf16 hi plane / hi and lo planes, rows of pitch
// px), and u_next as launch_fwd_flow (without J0_T and E_data: launch_j0_edata gives them).
void launch_fwd_fused(const Grid& g, const void* vj, const float* u_cur, float* u_next,
                      float dtx, float dty, float dtz, const void* I0, const float* J1j,
                      const float* Wj, float* b, float c, float ihx, float ihy, float ihz,
                      int bsplit, int px, cudaStream_t s, int st, int rk = 0);
// J0_T = I0 o (id + u) and E_data = sum M (J0_T - I1)^2 into acc, from the planar map u = u_T.
void launch_j0_edata(const Grid& g, const float* u, const void* I0, const void* I1,
                     const void* M, float* J0T, Acc* acc, cudaStream_t s, int st);
// E_reg of all T fields v[T][3][N] into acc->e_reg (unscaled sum of |(gamma - alpha Lap_h) v|^2).
void launch_ereg(const Grid& g, const void* v, int T, float alpha, float gamma, float ihx2,
                 float ihy2, float ihz2, Acc* acc, cudaStream_t s, int st);
// v_j <- v_j - eps (2 v_j - Kb), 3 components.
void launch_update(const Grid& g, void* vj, const float* Kb, float eps, cudaStream_t s, int st);
// Displacement of phi_{1,0} / phi_{0,1} only (flows without the residual), to refresh maps.
// rk = 1: RK4 along each step (v_j held over the step) instead of one lookup.
void launch_flow_only_fwd(const Grid& g, const void* vj, const float* u_cur, float* u_next,
                          float dtx, float dty, float dtz, cudaStream_t s, int st, int rk = 0,
                          int quad = 0);
void launch_flow_only_back(const Grid& g, const void* vj, const float* u_next, float* u_cur,
                           float dtx, float dty, float dtz, cudaStream_t s, int st, int rk = 0,
                           int quad = 0);
// A map in the quad layout ([N] x (u_x, u_y, u_z, 0), the iteration's sweeps) to the planar one
// ([3][N]).
void launch_quad_to_planar(const float* quad, float* planar, int64_t n, cudaStream_t s);
void launch_warp(const Grid& g, const float* src, const float* u, float* dst, cudaStream_t s);
void launch_labels(const Grid& g, const uint16_t* L0, const float* u, uint16_t* dst,
                   cudaStream_t s);
void launch_downsample(const Grid& fine, const Grid& coarse, int factor, const float* src,
                       void* dst, cudaStream_t s, int st);
void launch_upsample(const Grid& coarse, const Grid& fine, float ratio, const void* src,
                     void* dst, int nfields, cudaStream_t s, int st);
void launch_to_storage(const float* src, void* dst, int64_t n, cudaStream_t s, int st);
void launch_from_storage(const void* src, float* dst, int64_t n, cudaStream_t s, int st);
// *flag |= bit when a[0..n) holds a NaN or an infinity.
void launch_check_finite(const float* a, int64_t n, int* flag, cudaStream_t s, int bit = 1);
void launch_fill(float* a, int64_t n, float value, cudaStream_t s);
void launch_dice_hist(const uint16_t* A, const uint16_t* B, int64_t n,
                      unsigned long long* hist /* 3 x 65536 */, cudaStream_t s);

// ---- registration-quality measures of §2.7 (kernels_metrics.cu) ----
// Surface voxels of mask m appended to list as (x, y, z, 0); *count receives their number
// (entries past cap are counted but not written, so cap = 0 only counts).
cudaError_t surface_list(const Grid& g, const uint8_t* m, int4* list, unsigned* count,
                         unsigned cap, cudaStream_t s);
// d[i] = distance (physical units) from src[i] to the nearest point of dst.
cudaError_t nearest_distances(const int4* src, unsigned ns, const int4* dst, unsigned nd,
                              float hx, float hy, float hz, double* d, cudaStream_t s);
// out[0] = max of d[0..n), out[1] = k1-th, out[2] = k2-th smallest (0-based); one block.
cudaError_t order_stats(const double* d, unsigned n, unsigned k1, unsigned k2, double* out,
                        cudaStream_t s);
// e[k] = |(x_k + u01(x_k) - y_k) h| for n points (float [n][3], voxel coordinates).
cudaError_t landmark_errors(const Grid& g, const float* u01, const float* xk, const float* yk,
                            int n, float hx, float hy, float hz, double* e, cudaStream_t s);

// ---- preprocessing of §2.2 (kernels_preprocess.cu) ----
// st[0], st[1]: min and max of I over M > 0.5 (ordered-int encoding), st[2]: their count.
cudaError_t masked_range(const float* I, const float* M, int64_t n, int* st, cudaStream_t s);
// counts[bins]: histogram of I over M > 0.5 on [min, max] from st.
cudaError_t masked_hist(const float* I, const float* M, int64_t n, const int* st, int bins,
                        unsigned long long* counts, cudaStream_t s);
// nodes: points + 2 source intensities, then points + 2 reference intensities (FP64).
cudaError_t match_nodes(const int* st0, const unsigned long long* c0, const int* st1,
                        const unsigned long long* c1, int bins, int points, double* nodes,
                        cudaStream_t s);
// out = the piecewise-linear map of I0 through the nodes where M0 > 0.5, else 0.
cudaError_t apply_match(const float* I0, const float* M0, int64_t n, const double* nodes,
                        int points, float* out, cudaStream_t s);
cudaError_t threshold_mask(const float* I, int64_t n, float t, uint8_t* out, cudaStream_t s);
// Erosion (erode) or dilation by the ball of radius r; beyond the grid is background.
cudaError_t ball_op(const Grid& g, const uint8_t* in, int r, bool erode, uint8_t* out,
                    cudaStream_t s);

// ---- geodesic shooting (kernels_shoot.cu) ----
// m = |D phi| (D phi)^T (m0 o phi), phi = id + u (u in voxels), 3 components of N each.
cudaError_t transport_momentum(const Grid& g, const float* m0, const float* u, float hx,
                               float hy, float hz, float* m, cudaStream_t s);

// ---- exact gradient of the discrete energy (kernels_adjoint.cu) ----
void launch_adj_init(const Grid& g, const float* uT, const float* I0, const float* I1,
                     const float* M, float* gT, float scale, cudaStream_t s);
void launch_adj_step(const Grid& g, const float* vj, const float* uj, const float* gnext,
                     float* gcur, float* gradj, float dtx, float dty, float dtz, cudaStream_t s);
void launch_apply_L3(const Grid& g, const float* src, float* dst, float alpha, float gamma,
                     float ihx2, float ihy2, float ihz2, float scale, bool accumulate,
                     cudaStream_t s);

// ---- smoothing operator K (kernels_dft.cu) ----
struct KPlan {
  int nx, ny, nz;
  float alpha, gamma;
  // per-axis orthonormal real DFT matrices R (row k = frequency basis vector), row-major
  float* Rx; float* Ry; float* Rz;
  // per-axis discrete-Laplacian eigenvalue of each row, lambda_d(row) / h_d^2 folded in
  float* lx; float* ly; float* lz;
  // tensor-core operand tables per axis (x, y, z) and direction (0 forward, 1 inverse):
  // nk = Npad/16 k-steps, each [hi | lo] bf16 blocks of Npad x 16 in K-major core-matrix order
  uint16_t* tc[3][2];
  // operand tables of the pre-split pass (kernels_ks.cu) per axis and direction: bf16
  // [2][Nc][Kp] (hi plane, lo plane), row n = output column, k contiguous (Nc = Kp =
  // ceil16(n)), zero beyond the axis length
  uint16_t* ks[3][2];
  int* err;  // device flag set by a tensor-core kernel whose bounded wait timed out
  // probes per pipeline wait in the pre-split tensor-core pass (0: the default, 2^22)
  uint32_t poll_limit;
};
// Build device tables for one grid (allocates; free with kplan_destroy).
cudaError_t kplan_create(KPlan* kp, int nx, int ny, int nz, float hx, float hy, float hz,
                         float alpha, float gamma);
void kplan_destroy(KPlan* kp);
// out = K in for `ncomp` scalar fields stored back to back (each nx*ny*nz); work needs
// ncomp*N floats.  in and out may alias.  mode: LDDMM_K_*.
// If v_upd != nullptr the result is not stored: instead v_upd <- v_upd - eps (2 v_upd - K in)
// (the gradient-descent update, fused into the last pass on the tensor-core path).
// cap: floats available in out and in work (0: ncomp*N); the tensor-core modes take the
// pre-split path when cap >= ks_field_floats (intermediate fields with padded rows).
cudaError_t apply_K(const KPlan& kp, int mode, const float* in, float* out, float* work,
                    int ncomp, cudaStream_t s, const Hook& hook = Hook(),
                    float* v_upd = nullptr, float eps = 0.f, long long cap = 0,
                    bool in_split = false);
// Output addressing of a pre-split pass: line l = (a D + b) E + e is written at column n to
// element (a F + b) P + e + n G, as bf16 hi/lo planes `plane` elements apart (KS_OUT_SPLIT), as
// fp32 (KS_OUT_F32), or as the update out <- out - eps (2 out - C) of fp32 rows (KS_OUT_UPD) or
// of bf16 rows (KS_OUT_UPD_BF16, arithmetic in FP32, one rounding);
// sym: scale by the K symbol of the z-forward product.
enum { KS_OUT_SPLIT = 0, KS_OUT_F32 = 1, KS_OUT_UPD = 2, KS_OUT_UPD_BF16 = 3 };
struct KsOut {
  int kind;
  int sym;
  void* out;
  long long plane;
  long long D, E, F, P, G;
};
// cuTensorMapEncodeTiled from the driver, as void* (nullptr when unavailable).
void* tma_encode_fn();
// The pre-split path (all six products on k_dft_ks).  Row pitch of a split line (elements),
// support test, and the floats a buffer needs for any intermediate field of ncomp components.
int ks_pitch(int L);
bool ks_supported(const KPlan& kp);
long long ks_field_floats(int nx, int ny, int nz, int ncomp);
cudaError_t ks_axis_pass(const KPlan& kp, int axis, bool inverse, int split, const void* in,
                         long long nlines, const KsOut& o, float eps, cudaStream_t s,
                         bool zz = false);
// True when apply_K(kp, mode, ..., ncomp, cap) takes the pre-split path; its input may then be
// given already split (in_split): bf16 hi/lo planes [ncomp][nz][ny][ks_pitch(nx)].
bool ks_path(const KPlan& kp, int mode, int ncomp, long long cap);
// The pre-split K of `in` (3 components, on the pre-split path only) with the update fused into
// its last product for a velocity stored in bf16: v <- bf16(v - eps (2 v - K in)), the
// arithmetic in FP32.  cudaErrorNotSupported when the pre-split path does not apply.
cudaError_t apply_K_update_bf16(const KPlan& kp, int mode, const float* in, float* work,
                                cudaStream_t s, const Hook& hook, void* v_bf16, float eps,
                                long long cap, bool in_split);
// fp32 rows [nrows][L] -> split field at the addresses `o` gives (line = row, column = n).
cudaError_t ks_split_rows(const float* in, long long nrows, int L, int split, const KsOut& o,
                          cudaStream_t s);
// One tensor-core axis pass (kernels_tc.cu): epi 0 plain, 1 times the K symbol, 2 update.
cudaError_t tc_axis_pass(const KPlan& kp, int axis, bool inverse, int split, const float* in,
                         float* out, int ncomp, int epi, float eps, cudaStream_t s);

}  // namespace lddmm
