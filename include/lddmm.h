/*
 * liblddmm — masked LDDMM registration of 3D volumes on one GB300 GPU (sm_103a).
 *
 * Method: Kutten et al., "Deformably registering and annotating whole CLARITY brains to an
 * atlas via masked LDDMM" (SPIE 2016).  §2.4 defines the energy
 *     E(v) = int_0^1 ||L v_t||^2 dt + sigma^-2 ||J0 o phi_10 - J1||^2,  L = (-alpha Lap + gamma) I3,
 * minimised by gradient descent over a time-varying velocity field v; §2.3 (Mask-LDDMM) passes
 * the brain masks as the images; §2.5 pulls the atlas labels back through phi_10.  The gradient
 * and the update are those of Beg et al. 2005 (cited in §2.4):
 *     v_t <- v_t - eps (2 v_t - K[(2/sigma^2) (M o phi_t1) |D phi_t1| (J0_t - J1_t) grad J0_t]),
 *     K = (gamma - alpha Lap_h)^-2 on the periodic grid.
 *
 * Discretisation used by every entry point (the paper gives only the continuous method):
 *   - grid nx x ny x nz, C order [z][y][x] (x fastest), spacing (hx, hy, hz);
 *   - T time steps, dt = 1/T; velocity v laid out [T][3][nz][ny][nx] float32, components (x,y,z),
 *     in physical units (voxel spacing units per unit time);
 *   - first-order semi-Lagrangian flows, one trilinear lookup per step:
 *       phi_{j,1}(x) = phi_{j+1,1}(x + dt v_j(x)),  phi_{j+1,0}(x) = phi_{j,0}(x - dt v_j(x));
 *   - maps are returned as displacements u = phi - id, [3][nz][ny][nx] float32, in voxels;
 *   - trilinear interpolation with clamp-to-edge coordinates; gradients and D phi by central
 *     differences inside, one-sided at the faces; Lap_h the periodic 7-point Laplacian;
 *   - E = hx hy hz [dt sum_j sum_x |(gamma - alpha Lap_h) v_j|^2
 *                   + sigma^-2 sum_x M (I0 o phi_10 - I1)^2].
 *
 * Memory: every pointer argument may address device memory or host memory (pinned or
 * pageable): data moves with cudaMemcpyAsync(cudaMemcpyDefault) on the context's stream.  The
 * caller owns every pointer it passes; the library copies inputs in and writes only the
 * destination buffers it is given.  The context owns its device buffers until lddmm_destroy.
 * Work is enqueued on the context's stream; a call that returns scalars or writes host memory
 * waits for that stream (bounded wait: LDDMM_ERR_TIMEOUT after params.timeout_s seconds).
 * Errors: a negative status; lddmm_last_error(ctx) describes the last failure of that context,
 * and lddmm_last_error(NULL) the last failure on the calling thread of a call without one.
 * No exception crosses this interface.  After LDDMM_ERR_CUDA the context must be destroyed;
 * after any other error it stays usable.  One context may be used by one host thread at a time.
 * LDDMM_ERR_TIMEOUT also reports a bounded wait inside a tensor-core pass that gave up: the
 * kernel drains its copies and returns, that iteration's v is not valid, and the context stays
 * usable once v is set again.
 * Test hooks, read from the environment by lddmm_create (unset in normal use):
 *   LDDMM_TEST_FAIL_ALLOC=k   the k-th device allocation of that call fails as out of memory;
 *   LDDMM_TEST_POLL_LIMIT=n   each pipeline wait of the pre-split DFT pass gives up after n probes.
 */
#ifndef LDDMM_H
#define LDDMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lddmm_ctx lddmm_ctx;

enum {
  LDDMM_OK = 0,
  LDDMM_ERR_INVALID_ARG = -1,
  LDDMM_ERR_OOM = -2,
  LDDMM_ERR_CUDA = -3,
  LDDMM_ERR_NONFINITE = -4,
  LDDMM_ERR_STATE = -5,
  LDDMM_ERR_TIMEOUT = -6
};

/* How K is applied (per-axis real DFTs written as dense matrix products). */
enum {
  LDDMM_K_FP32 = 0,    /* FP32 products on the CUDA cores (reference form)            */
  LDDMM_K_BF16X3 = 1,  /* tensor cores, split bf16 x3 products, FP32 accumulation      */
  LDDMM_K_BF16 = 2     /* tensor cores, plain bf16 products, FP32 accumulation         */
};

/* What lddmm_get_field returns. */
enum {
  LDDMM_FIELD_U10 = 0, /* phi_{1,0} - id, [3][nz][ny][nx] voxels (template -> target pull-back) */
  LDDMM_FIELD_U01 = 1, /* phi_{0,1} - id, [3][nz][ny][nx] voxels                                */
  LDDMM_FIELD_J0 = 2,  /* deformed template I0 o phi_{1,0}, [nz][ny][nx]                         */
  LDDMM_FIELD_I0 = 3,  /* template at the current level                                          */
  LDDMM_FIELD_I1 = 4,  /* target at the current level                                            */
  LDDMM_FIELD_M = 5    /* weight mask at the current level                                       */
};

/* Problem parameters (§2.4: alpha, gamma, sigma; time steps; gradient-descent step). */
typedef struct {
  int nx, ny, nz;            /* finest grid (each >= 2 at every level)                      */
  float hx, hy, hz;          /* finest voxel spacing (> 0)                                   */
  int T;                     /* time steps (>= 1)                                            */
  float alpha, gamma, sigma; /* L = (-alpha Lap + gamma), sigma of the data term (> 0)       */
  float epsilon;             /* gradient-descent step size (> 0)                             */
  int iterations;            /* iterations per level for lddmm_register (>= 0)               */
  int num_levels;            /* 1..4                                                         */
  int level_factor[4];       /* coarse -> fine downsampling factors, last must be 1, e.g. 4,2,1 */
  int k_mode;                /* LDDMM_K_*                                                    */
  int flags;                 /* bit 0: halve epsilon and retry when the energy increases;
                                bit 1: checkpoint the forward maps in lddmm_energy_grad;
                                bit 2: integrate each time step by RK4 along the characteristic
                                (v_j held over the step, read by trilinear lookups at the
                                stages; the paper's integrator, §2.4) instead of one lookup.
                                lddmm_energy_grad rejects bit 2.                             */
  float timeout_s;           /* bound on every host wait for the stream (<= 0: 600 s)        */
  int storage;               /* 0: v and images stored float32; 1: stored bf16 (FP32 arithmetic,
                                FP64 reductions; the precision form)                          */
} lddmm_params;

/* Energy of the velocity field at the start of an iteration (§2.4), FP64 reductions. */
typedef struct {
  double total, reg, data;   /* E = reg + data                                              */
  double min_det;            /* min over j, x of det D phi_{j,1} (fold check: <= 0 folds)    */
  int iter, level, fold;     /* iteration index, level index, 1 if min_det <= 0              */
  int pad;
} lddmm_energy;

/* Fill p with the defaults used by the tests: h = 1, T = 10, alpha = 0.02, gamma = 1,
 * sigma = 0.1, eps = 1e-3, 20 iterations, one level, K by FP32 DFT products (LDDMM_K_FP32), fp32 storage, timeout 600 s. */
int lddmm_default_params(lddmm_params* p, int nx, int ny, int nz);

/* Create a context: validates p, allocates device buffers for all levels, copies I0
 * (template), I1 (target) and M (weight mask, NULL = all ones; each nx*ny*nz float32) in,
 * builds the image pyramid and sets v = 0 at the coarsest level.  stream: the cudaStream_t all
 * work of this context is enqueued on (NULL = the legacy default stream); device outputs are
 * ready once that stream reaches the call's work.  Returns LDDMM_ERR_NONFINITE if an input holds
 * NaN/Inf, LDDMM_ERR_CUDA if no GPU is usable. */
int lddmm_create(const lddmm_params* p, const float* I0, const float* I1, const float* M,
                 void* stream, lddmm_ctx** out);

/* Replace the images at the finest level (and rebuild the pyramid), keeping v. */
int lddmm_set_images(lddmm_ctx* ctx, const float* I0, const float* I1, const float* M);

/* One gradient-descent iteration at the current level (Beg update).  out = NULL: fully
 * asynchronous; otherwise waits and fills *out with the energy of v before the update. */
int lddmm_step(lddmm_ctx* ctx, lddmm_energy* out);

/* Full schedule: for each remaining level, `iterations` steps, then upsample v to the next
 * level.  trace (NULL or room for num_levels*iterations entries) receives every energy. */
int lddmm_register(lddmm_ctx* ctx, lddmm_energy* trace, int trace_len);

/* Move to level `level` (0 = coarsest), carrying v over by trilinear resampling. */
int lddmm_set_level(lddmm_ctx* ctx, int level);
/* Grid of the current level. */
int lddmm_grid(lddmm_ctx* ctx, int* nx, int* ny, int* nz, int* level);

/* dst = src o phi_{1,0} (direction 0, template into target space) or src o phi_{0,1}
 * (direction 1), trilinear, on the current level grid (§2.4, §2.7). */
int lddmm_warp(lddmm_ctx* ctx, const float* src, float* dst, int direction);

/* dst = L0 o phi_{1,0} by nearest neighbour: index floor(x + u + 0.5) per axis in float32,
 * clamped to the grid (§2.5).  uint16 labels, nx*ny*nz each, current level grid. */
int lddmm_transfer_labels(lddmm_ctx* ctx, const uint16_t* L0, uint16_t* dst);

/* Velocity field of the current level, [T][3][nz][ny][nx] float32. */
int lddmm_get_velocity(lddmm_ctx* ctx, float* dst);
int lddmm_set_velocity(lddmm_ctx* ctx, const float* src);

/* One of LDDMM_FIELD_*, for the current v (flows are recomputed if v changed). */
int lddmm_get_field(lddmm_ctx* ctx, int which, float* dst);

/* dst = K src for one scalar field on the current level grid, using params.k_mode. */
int lddmm_apply_K(lddmm_ctx* ctx, const float* src, float* dst);

/* Energy of the current v without updating it. */
int lddmm_energy_eval(lddmm_ctx* ctx, lddmm_energy* out);

/* Exact Euclidean gradient of the discrete energy above with respect to v, by reverse-mode
 * differentiation of the forward sweep (§2.4 energy; the adjoint of the trilinear interpolation
 * is a scatter-add).  v: [T][3][nz][ny][nx] float32 of the current level (NULL = the context's
 * current v; otherwise it becomes the current v); grad: same layout, written; E: energy of v.
 * Forward maps are stored for all T+1 steps, or, with params.flags bit 1, kept every
 * ceil(sqrt(T)) steps and recomputed per segment during the reverse sweep.  The scatter uses
 * float atomics: results vary at FP32 rounding between runs. */
int lddmm_energy_grad(lddmm_ctx* ctx, const float* v, float* grad, double* E);

/* Mean Dice overlap over labels > 0 present in A or B (uint16, n voxels each). */
int lddmm_dice(lddmm_ctx* ctx, const uint16_t* A, const uint16_t* B, int64_t n, double* out);

/* Surface distances between two binary masks on the current level's grid (§2.7: the Hausdorff
 * distance d_H and the median surface distance d_M between the deformed-template surface
 * S(1) = boundary(M0 o phi^-1) and the target surface S1 = boundary(M1)).
 * A, B: uint8 [nz][ny][nx] (nonzero = inside), device or host memory, read only.  A surface
 * voxel is a mask voxel with a face neighbour outside the mask (outside the grid counts).
 * Distances are Euclidean between voxel centres in physical units (the level's spacing).
 * out[0] = d_H = max of both directed maxima; out[1] = d_M = median of the union of the directed
 * distances of S_A to S_B and of S_B to S_A (mean of the two middle values for an even count);
 * out[2], out[3] = the number of surface voxels of A and of B.  Host memory.
 * Allocates scratch for the surface lists and distances for the duration of the call and waits
 * for the result (bounded).  LDDMM_ERR_INVALID_ARG when a mask has no surface voxel. */
int lddmm_surface_distance(lddmm_ctx* ctx, const uint8_t* A, const uint8_t* B, double out[4]);

/* Landmark errors e_k = |phi(x_k) - y_k| (§2.7) for the current v: phi(x) = x + u01(x) carries
 * a template point to the target point it lands on (u01 = phi_{0,1} - id interpolated
 * trilinearly, clamp to edge).  xk, yk: n points as float [n][3] = (x, y, z) in voxel
 * coordinates of the current level; err: n doubles, physical units.  Any pointer may be device
 * or host memory; a host err is written before the call returns. */
int lddmm_landmark_error(lddmm_ctx* ctx, const float* xk, const float* yk, int n, double* err);

/* Geodesic shooting (EPDiff; LDDMM's minimisers are geodesics, Beg et al. 2005 cited in §2.4;
 * the paper has no shooting step): replaces the context's v_j, j = 0..T-1, by the geodesic from
 * v0.  The momentum m_0 = L^T L v0 is transported by the flow, m_j = |D phi| (D phi)^T (m_0 o phi)
 * with phi = phi_{j,0} from the same semi-Lagrangian steps as the forward sweep, and
 * v_j = K m_j with the context's K.  v0: float [3][nz][ny][nx] of the current level, device or
 * host memory, in physical units.  Needs float storage (params.storage = 0) and the one-lookup
 * flow (flags bit 2 clear). */
int lddmm_shoot(lddmm_ctx* ctx, const float* v0);

/* Image-LDDMM preprocessing (§2.2): the masks are applied to the images and the masked I0 is
 * histogram-matched to the masked I1.  Each image gets a `bins`-bin histogram (the paper: 32) of
 * its voxels with M > 0.5 over [min, max] of those voxels; `points` quantiles (the paper: 8) at
 * k / (points + 1) are read off the cumulative counts, interpolated inside the bin that reaches
 * the fraction.  out = the piecewise-linear map sending min to min, max to max and each quantile
 * of I0 to the same quantile of I1 (end segments continued beyond), applied to I0 where
 * M0 > 0.5, and 0 elsewhere.  I0, M0, I1, M1, out: n floats of device memory (out may alias
 * I0); bins in [1, 1024], points in [0, 64].  Work is enqueued on `stream` (NULL: the legacy
 * default stream); the call allocates a few hundred bytes of scratch and waits for the nodes
 * (bounded) to report an empty mask as LDDMM_ERR_INVALID_ARG.  No context. */
int lddmm_histogram_match(const float* I0, const float* M0, const float* I1, const float* M1,
                          int64_t n, int bins, int points, float* out, void* stream);

/* Mask generation (§2.2): out = [I > threshold] opened with the ball of radius r_open voxels
 * (erosion, then dilation), then closed with the ball of radius r_close (dilation, then
 * erosion); ball = offsets with dx^2 + dy^2 + dz^2 <= r^2; voxels beyond the grid count as
 * background (the paper: 50 um and 125 um radii).  I: float [nz][ny][nx], out: uint8, device
 * memory.  r_open, r_close in [0, 16] (0 skips that step).  Allocates one scratch volume for
 * the duration of the call and waits for it (bounded).  No context. */
int lddmm_mask_morphology(const float* I, int nx, int ny, int nz, float threshold, int r_open,
                          int r_close, uint8_t* out, void* stream);

/* Per-kernel device time, summed over the launches since lddmm_profile_start. */
typedef struct {
  char name[32];
  int launches;
  int pad;
  double total_ms;
} lddmm_kernel_stat;

/* Record a pair of CUDA events on the context stream around each of the next max_launches
 * kernel launches of lddmm_step (timing only; the computation is unchanged). */
int lddmm_profile_start(lddmm_ctx* ctx, int max_launches);
/* Stop recording, wait for the stream and sum device time per kernel into out[0..max_out);
 * *n_out = number of distinct kernels seen.  LDDMM_ERR_STATE if max_launches was too small. */
int lddmm_profile_stop(lddmm_ctx* ctx, lddmm_kernel_stat* out, int max_out, int* n_out);

/* The paper has no counterpart of this entry point.  dst = K src (K = (gamma - alpha Lap_h)^-2,
 * FP32 per-axis real-DFT products, the same arithmetic as lddmm_apply_K with LDDMM_K_FP32) for
 * one scalar field of nx*ny*nz float32 on a grid of spacing (hx, hy, hz), enqueued on `stream`
 * (NULL = legacy default stream), WITHOUT allocating any memory.  It serves callers that cannot
 * call cudaMalloc: a host callback, a real-time loop that must not stall on the allocator, a
 * process whose GPU memory another framework's pool has reserved up front.  Its scratch (the
 * intermediate field and the DFT tables) is one file-scope __device__ array of ~11.5 MB, which
 * every GPU that loads the library holds until the process exits.  Limits: nx*ny*nz <= 2^21,
 * each axis in [2, 512]; larger grids give LDDMM_ERR_INVALID_ARG.  src and dst must be device
 * pointers (LDDMM_ERR_INVALID_ARG otherwise); dst may equal src.  The first call on a device
 * looks up the array's device address with that device current; make it before any stream
 * capture.  The tables are generated on the device, and again only when (n, h) of an axis
 * changes; everything else in the array is rewritten before it is read, so nothing needs to
 * start at zero.  All calls share the array: calls that overlap on the GPU (other streams, other
 * host threads) race, so issue them on one stream.  LDDMM_ERR_CUDA on a CUDA failure; the reason
 * of any failure is in lddmm_last_error(NULL) on the calling thread. */
int lddmm_apply_K_noalloc(const float* src, float* dst, int nx, int ny, int nz, float hx,
                          float hy, float hz, float alpha, float gamma, void* stream);

/* ---- Learned warm start: kernels of a 3D convolutional encoder-decoder that predicts an initial
 * velocity from a mask pair (no counterpart in the paper: §2.4 optimises from v = 0).  All pointers are device
 * pointers; work is enqueued on `stream` (NULL = legacy default stream); LDDMM_ERR_INVALID_ARG
 * on a bad shape, LDDMM_ERR_CUDA on a launch failure.  Layout: activations [B][C][n][n][n]
 * float32; weights [Co][Ci][k^3] bf16 (k = 3, zero padding 1, or k = 1); FP32 accumulation. */
/* y (+)= conv(x, w) + bias (bias may be NULL), then ReLU if relu. */
int lddmm_net_conv3d_fwd(const float* x, const void* w_bf16, const float* bias, float* y, int B,
                         int Ci, int Co, int n, int ksize, int relu, int accumulate, void* stream);
/* dx = data gradient of the convolution for output gradient dy; wT_scratch holds Ci*Co*k^3
 * bf16 (the transposed, flipped kernel). */
int lddmm_net_conv3d_dgrad(const float* dy, const void* w_bf16, void* wT_scratch, float* dx, int B,
                           int Ci, int Co, int n, int ksize, void* stream);
/* Floats of scratch that lddmm_net_conv3d_wgrad needs for this shape (LDDMM_ERR_INVALID_ARG on
 * a bad shape). */
int64_t lddmm_net_conv3d_wgrad_scratch(int B, int Ci, int Co, int n, int ksize);
/* dw += weight gradient (float32 [Co][Ci][k^3]), db += bias gradient (NULL: skipped).  The sums
 * run in a fixed order through partial sums in `scratch` (device, scratch_floats >= the size
 * lddmm_net_conv3d_wgrad_scratch gives, else LDDMM_ERR_INVALID_ARG), so repeated calls on the same
 * inputs give the same bits. */
int lddmm_net_conv3d_wgrad(const float* x, const float* dy, float* dw, float* db, float* scratch,
                           int64_t scratch_floats, int B, int Ci, int Co, int n, int ksize,
                           void* stream);
/* dy[i] = 0 where y[i] <= 0 (ReLU backward on the stored output). */
int lddmm_net_relu_bwd(float* dy, const float* y, int64_t count, void* stream);
/* 2x average pooling of BC volumes of n^3 (backward: src = coarse gradient, dst = fine). */
int lddmm_net_pool2(const float* src, float* dst, int64_t BC, int n, int backward, void* stream);
/* 2x nearest upsampling of [B][C][m^3] into channels [coff, coff+C) of a [B][Cy][(2m)^3]
 * buffer (backward: sums the 8 children back). */
int lddmm_net_up2(const float* src, float* dst, int B, int C, int m, int Cy, int coff, int backward,
                  void* stream);
/* dst[b][doff+c] (+)= src[b][soff+c] for c < C, nv voxels per channel (concatenation). */
int lddmm_net_copy_channels(const float* src, float* dst, int B, int C, int64_t nv, int Cs,
                            int soff, int Cd, int doff, int accumulate, void* stream);
/* *loss_dev += sum (pred - target)^2 (FP64); grad = 2 (pred - target) / count (NULL: skipped). */
int lddmm_net_mse(const float* pred, const float* target, float* grad, int64_t count,
                  double* loss_dev, void* stream);
/* Adam step `step` (>= 1) on FP32 master weights w with moments m, v; refreshes the bf16 copy. */
int lddmm_net_adam(float* w, const float* g, float* m, float* v, void* w_bf16, int64_t count,
                   float lr, float beta1, float beta2, float eps, int step, void* stream);
int lddmm_net_cast_bf16(const float* a, void* b, int64_t count, void* stream);

/* Resampling between two grids over the same box (the warm start's coarse network grid and the
 * registration grid; the paper has no counterpart): dst = trilinear interpolation of src at
 * cell-centred coordinates q_d = (i_d + 0.5) s_d / d_d - 0.5 (source voxels, clamped to the
 * source grid), for nfields fields [nfields][sz][sy][sx] -> [nfields][dz][dy][dx] (x fastest);
 * field f is multiplied by (s0, s1, s2)[f % ncomp] (ncomp = 1 for scalar fields, 3 for vector
 * fields [..][3][..] whose components change units with the grid).  Device pointers; src and
 * dst must not overlap; enqueued on `stream`; LDDMM_ERR_INVALID_ARG on a bad shape. */
int lddmm_resample(const float* src, int sx, int sy, int sz, float* dst, int dx, int dy, int dz,
                   int nfields, int ncomp, float s0, float s1, float s2, void* stream);
/* x <- c x for count floats of device memory, enqueued on `stream`. */
int lddmm_scale(float* x, int64_t count, float c, void* stream);

/* Change the bound on host waits for this context (seconds, <= 0: 600 s). */
int lddmm_set_timeout(lddmm_ctx* ctx, float seconds);

const char* lddmm_last_error(lddmm_ctx* ctx);
void lddmm_destroy(lddmm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* LDDMM_H */
