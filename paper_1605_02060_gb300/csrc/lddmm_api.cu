// C ABI of liblddmm: context, buffers, the multiscale schedule and one gradient-descent
// iteration of masked LDDMM (§2.4 of Kutten et al., SPIE 2016; Beg et al. 2005 update).
// Host code only; every step of the computation runs in the kernels of kernels_*.cu.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/lddmm.h"
#include "kernels.h"

using namespace lddmm;

namespace {

thread_local std::string g_global_error;

struct Level {
  Grid g;
  int factor;
  float hx, hy, hz;
  float *I0 = nullptr, *I1 = nullptr, *M = nullptr;
  float* IM = nullptr;   // I1 and M interleaved as pairs (backward-sweep lookups)
  KPlan kp{};
};

}  // namespace

struct lddmm_ctx {
  lddmm_params p{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<Level> levels;
  int cur = 0;
  int64_t Nmax = 0;
  int64_t kcap = 0;         // floats in b and work (K's intermediate fields may pad rows)
  // working buffers, sized for the finest level
  float* v = nullptr;       // [T][3][N]
  float* v_tmp = nullptr;   // [T][3][N] resampling / backtracking copy
  float* v_prev = nullptr;  // [T][3][N] v before the last accepted update (backtracking)
  bool have_prev = false;
  float* uB[2] = {nullptr, nullptr};
  float* uF[2] = {nullptr, nullptr};
  float* J1 = nullptr;      // [T][N]
  float* W = nullptr;       // [T][N]
  float* b = nullptr;       // [3][N]
  float* work = nullptr;    // [3][N]
  float* J0T = nullptr;     // [N]
  float* stage = nullptr;   // [3][N] staging for host inputs / outputs
  Acc* acc = nullptr;
  Acc* acc_init = nullptr;  // the accumulators' start value (device copy, written at creation)
  Acc* acc_host = nullptr;  // pinned
  int* flag = nullptr;      // device int
  unsigned long long* hist = nullptr;  // 3 x 65536
  // map state
  const float* u10 = nullptr;
  const float* u01 = nullptr;
  bool maps_valid = false;
  bool j0_valid = false;
  int iter = 0;
  double last_E = -1.0;
  float eps = 0.f;
  int st = 0;               // storage of v and images: 0 float, 1 bf16
  size_t es = 4;            // bytes per stored element
  std::string err;
  // timing of every kernel launch (lddmm_profile_start / lddmm_profile_stop)
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_ev;   // 2 per launch
  std::vector<int> prof_kid;
  size_t prof_used = 0;
  bool prof_overflow = false;
  int prof_open = -1;
  // exact-gradient path (allocated on first use)
  float* uall = nullptr;    // stored forward maps u_0..u_T (or checkpoints)
  float* gA = nullptr;      // dE/du_{j+1}
  float* gB = nullptr;      // dE/du_j
  float* seg = nullptr;     // recomputed segment of maps (checkpoint mode)
  int uall_slots = 0, seg_slots = 0;
  // One iteration's launches recorded as a CUDA graph and replayed while the level, the step
  // size and the velocity buffer are those it was recorded with (the kernels' arguments are
  // part of the graph); the maps it leaves are the recorded ones.
  cudaGraphExec_t step_graph = nullptr;
  cudaStream_t cap_stream = nullptr;   // the graph is recorded on this stream (any context stream,
                                       // the legacy one included, can then launch it)
  int g_cur = -1;
  float g_eps = 0.f;
  const void* g_v = nullptr;
  const float* g_u10 = nullptr;
  const float* g_u01 = nullptr;
};

namespace {

int fail(lddmm_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  else g_global_error = msg;
  return code;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? LDDMM_ERR_OOM : LDDMM_ERR_CUDA,      \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                        \
  } while (0)

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int wait_stream(lddmm_ctx* ctx) {
  const double limit = ctx->p.timeout_s > 0 ? ctx->p.timeout_s : 600.0;
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaStreamQuery(ctx->stream);
    if (e == cudaSuccess) return LDDMM_OK;
    if (e != cudaErrorNotReady)
      return fail(ctx, LDDMM_ERR_CUDA, std::string("stream: ") + cudaGetErrorString(e));
    const double el =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el > limit) return fail(ctx, LDDMM_ERR_TIMEOUT, "timed out waiting for the GPU stream");
    std::this_thread::sleep_for(std::chrono::microseconds(el < 0.01 ? 5 : 200));
  }
}

void prof_mark(void* user, int kid, int phase) {
  lddmm_ctx* ctx = static_cast<lddmm_ctx*>(user);
  if (!ctx->prof_on) return;
  if (phase == 0) {
    if (ctx->prof_used >= ctx->prof_kid.size()) { ctx->prof_overflow = true; ctx->prof_open = -1; return; }
    cudaEventRecord(ctx->prof_ev[2 * ctx->prof_used], ctx->stream);
    ctx->prof_open = kid;
  } else if (ctx->prof_open == kid) {
    cudaEventRecord(ctx->prof_ev[2 * ctx->prof_used + 1], ctx->stream);
    ctx->prof_kid[ctx->prof_used++] = kid;
    ctx->prof_open = -1;
  }
}

Hook hook_of(lddmm_ctx* ctx) {
  Hook h;
  if (ctx->prof_on) { h.mark = prof_mark; h.user = ctx; }
  return h;
}

const char* kernel_name(int kid) {
  static const char* names[KID_COUNT] = {"flow_back_disp", "flow_back_terms", "fwd_residual",
                                         "fwd_flow", "K_x_fwd", "K_y_fwd", "K_z_symbol",
                                         "K_z_inv", "K_y_inv", "K_x_inv_update", "update", "ereg",
                                         "K_z_fused", "fwd_fused", "fwd_J0T_Edata"};
  return (kid >= 0 && kid < KID_COUNT) ? names[kid] : "?";
}

int validate(const lddmm_params* p, std::string& why) {
  if (!p) { why = "params is NULL"; return LDDMM_ERR_INVALID_ARG; }
  if (p->nx < 2 || p->ny < 2 || p->nz < 2) { why = "grid sizes must be >= 2"; return LDDMM_ERR_INVALID_ARG; }
  const int64_t N = (int64_t)p->nx * p->ny * p->nz;
  if (N * 3 >= (int64_t)1 << 31) { why = "grid too large (3*nx*ny*nz must be < 2^31)"; return LDDMM_ERR_INVALID_ARG; }
  if (!(p->hx > 0 && p->hy > 0 && p->hz > 0)) { why = "spacing must be > 0"; return LDDMM_ERR_INVALID_ARG; }
  if (p->T < 1 || p->T > 1000) { why = "T must be in [1, 1000]"; return LDDMM_ERR_INVALID_ARG; }
  if (!(p->alpha >= 0 && std::isfinite(p->alpha))) { why = "alpha must be >= 0"; return LDDMM_ERR_INVALID_ARG; }
  if (!(p->gamma > 0 && std::isfinite(p->gamma))) { why = "gamma must be > 0"; return LDDMM_ERR_INVALID_ARG; }
  if (!(p->sigma > 0 && std::isfinite(p->sigma))) { why = "sigma must be > 0"; return LDDMM_ERR_INVALID_ARG; }
  if (!(p->epsilon > 0 && std::isfinite(p->epsilon))) { why = "epsilon must be > 0"; return LDDMM_ERR_INVALID_ARG; }
  if (p->iterations < 0) { why = "iterations must be >= 0"; return LDDMM_ERR_INVALID_ARG; }
  if (p->num_levels < 1 || p->num_levels > 4) { why = "num_levels must be in [1, 4]"; return LDDMM_ERR_INVALID_ARG; }
  for (int l = 0; l < p->num_levels; ++l) {
    const int f = p->level_factor[l];
    if (f < 1 || f > 64) { why = "level factors must be in [1, 64]"; return LDDMM_ERR_INVALID_ARG; }
    if (l > 0 && f >= p->level_factor[l - 1]) { why = "level factors must decrease"; return LDDMM_ERR_INVALID_ARG; }
    if ((p->nx + f - 1) / f < 2 || (p->ny + f - 1) / f < 2 || (p->nz + f - 1) / f < 2) {
      why = "a level grid has an axis shorter than 2"; return LDDMM_ERR_INVALID_ARG;
    }
  }
  if (p->level_factor[p->num_levels - 1] != 1) { why = "the last level factor must be 1"; return LDDMM_ERR_INVALID_ARG; }
  if (p->k_mode < LDDMM_K_FP32 || p->k_mode > LDDMM_K_BF16) { why = "unknown k_mode"; return LDDMM_ERR_INVALID_ARG; }
  if (p->k_mode != LDDMM_K_FP32 && (p->nx > 512 || p->ny > 512 || p->nz > 512)) {
    why = "tensor-core K needs every axis <= 512 (TMEM columns)"; return LDDMM_ERR_INVALID_ARG;
  }
  if (p->flags & ~7) { why = "unknown flag bits"; return LDDMM_ERR_INVALID_ARG; }
  if (p->storage != 0 && p->storage != 1) { why = "storage must be 0 (float) or 1 (bf16)"; return LDDMM_ERR_INVALID_ARG; }
  return LDDMM_OK;
}

// Test hook (environment LDDMM_TEST_FAIL_ALLOC=k, read by lddmm_create): the k-th device
// allocation of that create call fails as if the device were out of memory, so that the
// clean-up path can be checked without exhausting a GPU.  0 or unset: no injection.
thread_local int g_fail_alloc_countdown = 0;

template <typename T>
cudaError_t dalloc(T** p, int64_t n) {
  if (g_fail_alloc_countdown > 0 && --g_fail_alloc_countdown == 0) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc((void**)p, (size_t)n * sizeof(T));
}

int env_int(const char* name) {
  const char* v = std::getenv(name);
  return v ? std::atoi(v) : 0;
}

const float* field_src(lddmm_ctx* ctx, const float* user, int64_t n, float* stage, int* rc) {
  // Device pointers are used in place; host pointers are copied to the staging buffer.
  *rc = LDDMM_OK;
  if (is_device_ptr(user)) return user;
  cudaError_t e = cudaMemcpyAsync(stage, user, n * sizeof(float), cudaMemcpyDefault, ctx->stream);
  if (e != cudaSuccess) {
    *rc = fail(ctx, LDDMM_ERR_CUDA, cudaGetErrorString(e));
    return nullptr;
  }
  return stage;
}

int check_finite(lddmm_ctx* ctx, const float* d, int64_t n, const char* what) {
  CK(cudaMemsetAsync(ctx->flag, 0, sizeof(int), ctx->stream));
  launch_check_finite(d, n, ctx->flag, ctx->stream);
  int h = 0;
  CK(cudaMemcpyAsync(&h, ctx->flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  int rc = wait_stream(ctx);
  if (rc) return rc;
  if (h) return fail(ctx, LDDMM_ERR_NONFINITE, std::string(what) + " holds NaN or Inf");
  return LDDMM_OK;
}

int load_images(lddmm_ctx* ctx, const float* I0, const float* I1, const float* M) {
  Level& F = ctx->levels.back();
  const int64_t N = F.g.N;
  // inputs are float32: stage them (I0 | I1 | M), check them, store them in the storage type
  float* s0 = ctx->stage;
  float* s1 = ctx->stage + N;
  float* s2 = ctx->stage + 2 * N;
  CK(cudaMemcpyAsync(s0, I0, N * sizeof(float), cudaMemcpyDefault, ctx->stream));
  CK(cudaMemcpyAsync(s1, I1, N * sizeof(float), cudaMemcpyDefault, ctx->stream));
  if (M) CK(cudaMemcpyAsync(s2, M, N * sizeof(float), cudaMemcpyDefault, ctx->stream));
  else launch_fill(s2, N, 1.0f, ctx->stream);
  CK(cudaGetLastError());
  // the three images checked with one wait: bit 1 I0, bit 2 I1, bit 4 M
  CK(cudaMemsetAsync(ctx->flag, 0, sizeof(int), ctx->stream));
  launch_check_finite(s0, N, ctx->flag, ctx->stream, 1);
  launch_check_finite(s1, N, ctx->flag, ctx->stream, 2);
  launch_check_finite(s2, N, ctx->flag, ctx->stream, 4);
  int h = 0;
  CK(cudaMemcpyAsync(&h, ctx->flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  int rc = wait_stream(ctx);
  if (rc) return rc;
  if (h) return fail(ctx, LDDMM_ERR_NONFINITE, std::string((h & 1) ? "I0" : (h & 2) ? "I1" : "M") +
                                                   " holds NaN or Inf");
  launch_to_storage(s0, F.I0, N, ctx->stream, ctx->st);
  launch_to_storage(s1, F.I1, N, ctx->stream, ctx->st);
  launch_to_storage(s2, F.M, N, ctx->stream, ctx->st);
  for (size_t l = 0; l + 1 < ctx->levels.size(); ++l) {
    Level& L = ctx->levels[l];
    launch_downsample(F.g, L.g, L.factor, s0, L.I0, ctx->stream, ctx->st);
    launch_downsample(F.g, L.g, L.factor, s1, L.I1, ctx->stream, ctx->st);
    launch_downsample(F.g, L.g, L.factor, s2, L.M, ctx->stream, ctx->st);
  }
  for (Level& L : ctx->levels) launch_interleave(L.I1, L.M, L.IM, L.g.N, ctx->stream, ctx->st);
  CK(cudaGetLastError());
  ctx->maps_valid = false;
  ctx->j0_valid = false;
  return LDDMM_OK;
}

void release(lddmm_ctx* ctx) {
  for (Level& L : ctx->levels) {
    cudaFree(L.I0); cudaFree(L.I1); cudaFree(L.M); cudaFree(L.IM);
    kplan_destroy(&L.kp);
  }
  void* ps2[] = {ctx->uall, ctx->gA, ctx->gB, ctx->seg};
  for (void* p : ps2)
    if (p) cudaFree(p);
  if (ctx->step_graph) cudaGraphExecDestroy(ctx->step_graph);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  void* ps[] = {ctx->v, ctx->v_tmp, ctx->v_prev, ctx->uB[0], ctx->uB[1], ctx->uF[0], ctx->uF[1], ctx->J1,
                ctx->W, ctx->b, ctx->work, ctx->J0T, ctx->stage, ctx->acc, ctx->acc_init, ctx->flag,
                ctx->hist};
  for (void* p : ps)
    if (p) cudaFree(p);
  if (ctx->acc_host) cudaFreeHost(ctx->acc_host);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
}

inline float dtv(const lddmm_ctx* ctx, float h) { return 1.0f / (float)ctx->p.T / h; }

// flags bit 2: RK4 along each time step instead of one lookup
inline int rk_of(const lddmm_ctx* ctx) { return (ctx->p.flags >> 2) & 1; }

// v_j in the storage type (3 components of N elements each)
inline void* vptr(const lddmm_ctx* ctx, int j, int64_t N) {
  return reinterpret_cast<char*>(ctx->v) + (size_t)j * 3 * N * ctx->es;
}

Acc acc_start() {
  Acc a{};
  a.min_det_ord = 0x7f7fffff;  // +FLT_MAX in the ordered encoding
  return a;
}

int reset_acc(lddmm_ctx* ctx) {
  CK(cudaMemcpyAsync(ctx->acc, ctx->acc_init, sizeof(Acc), cudaMemcpyDeviceToDevice, ctx->stream));
  return LDDMM_OK;
}

double ordered_to_float(int i) {
  const int b = i >= 0 ? i : i ^ 0x7fffffff;
  float f;
  std::memcpy(&f, &b, 4);
  return (double)f;
}

int read_energy(lddmm_ctx* ctx, lddmm_energy* out, bool with_det) {
  const Level& L = ctx->levels[ctx->cur];
  CK(cudaMemcpyAsync(ctx->acc_host, ctx->acc, sizeof(Acc), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(&ctx->acc_host->nonfinite, L.kp.err, sizeof(int), cudaMemcpyDeviceToHost,
                     ctx->stream));
  int rc = wait_stream(ctx);
  if (rc) return rc;
  if (ctx->acc_host->nonfinite) {
    // a bounded wait inside a tensor-core pass gave up: that pass's output (and so v) is not
    // valid.  The kernel drained its copies and freed its resources, so the context stays
    // usable once the flag is cleared.
    CK(cudaMemsetAsync(L.kp.err, 0, sizeof(int), ctx->stream));
    return fail(ctx, LDDMM_ERR_TIMEOUT,
                "a tensor-core pipeline wait on the GPU gave up: this iteration's result is invalid "
                "(set the velocity again)");
  }
  const double h3 = (double)L.hx * L.hy * L.hz;
  const double s = ctx->p.sigma;
  out->reg = ctx->acc_host->e_reg * h3 / (double)ctx->p.T;
  out->data = ctx->acc_host->e_data * h3 / (s * s);
  out->total = out->reg + out->data;
  out->min_det = with_det ? ordered_to_float(ctx->acc_host->min_det_ord) : 1.0;
  out->fold = with_det && out->min_det <= 0.0;
  out->iter = ctx->iter - 1;
  out->level = ctx->cur;
  out->pad = 0;
  if (!std::isfinite(out->total)) return fail(ctx, LDDMM_ERR_NONFINITE, "energy is not finite");
  return LDDMM_OK;
}

// One iteration: backward sweep, forward sweep with K and the update per time step.
int record_step(lddmm_ctx* ctx) {
  const Level& L = ctx->levels[ctx->cur];
  const Grid& g = L.g;
  const int T = ctx->p.T;
  const int64_t N = g.N;
  cudaStream_t s = ctx->stream;
  const float dtx = dtv(ctx, L.hx), dty = dtv(ctx, L.hy), dtz = dtv(ctx, L.hz);
  const Hook hk = hook_of(ctx);
  int rc = reset_acc(ctx);
  if (rc) return rc;
  // backward sweep j = T-1 .. 0
  const float* un = nullptr;
  int pb = 0;
  for (int j = T - 1; j >= 0; --j) {
    float* uc = ctx->uB[pb];
    launch_flow_back(g, vptr(ctx, j, N), un, uc, L.IM, ctx->J1 + j * N, ctx->W + j * N, dtx,
                     dty, dtz, ctx->acc, s, hk, ctx->st, rk_of(ctx));
    un = uc;
    pb ^= 1;
  }
  ctx->u01 = un;
  // E_reg of the velocity at the start of the iteration (before the forward sweep updates it)
  hk(KID_EREG, 0);
  launch_ereg(g, ctx->v, T, ctx->p.alpha, ctx->p.gamma, 1.0f / (L.hx * L.hx),
              1.0f / (L.hy * L.hy), 1.0f / (L.hz * L.hz), ctx->acc, s, ctx->st);
  hk(KID_EREG, 1);
  // forward sweep j = 0 .. T-1 with smoothing and update; on the pre-split K path the residual
  // is written already split into bf16 hi/lo planes (the layout K's first product reads)
  const float c = 2.0f / (ctx->p.sigma * ctx->p.sigma);
  const bool ks = ks_path(L.kp, ctx->p.k_mode, 3, ctx->kcap);
  const int bsplit = ks ? (ctx->p.k_mode == LDDMM_K_BF16X3 ? 2 : 1) : 0;
  const float* uc = nullptr;
  int pf = 0;
  for (int j = 0; j < T; ++j) {
    void* vj = vptr(ctx, j, N);
    float* unx = ctx->uF[pf];
    // the residual b_j and the map of step j + 1 in one pass over u_j
    hk(KID_FWD_FUSED, 0);
    launch_fwd_fused(g, vj, uc, unx, dtx, dty, dtz, L.I0, ctx->J1 + j * N, ctx->W + j * N,
                     ctx->b, c, 1.0f / L.hx, 1.0f / L.hy, 1.0f / L.hz, bsplit, ks_pitch(g.nx), s,
                     ctx->st, rk_of(ctx));
    hk(KID_FWD_FUSED, 1);
    if (j == T - 1) {     // J0_T = I0 o phi_{1,0} and E_data
      hk(KID_J0_EDATA, 0);
      launch_j0_edata(g, unx, L.I0, L.I1, L.M, ctx->J0T, ctx->acc, s, ctx->st);
      hk(KID_J0_EDATA, 1);
    }
    // K b_j and the update v_j <- v_j - eps (2 v_j - K b_j): fused into the last DFT pass (for
    // bf16 storage on the pre-split path too), else a separate pass
    if (ctx->st == 0) {
      CK(apply_K(L.kp, ctx->p.k_mode, ctx->b, ctx->b, ctx->work, 3, s, hk, (float*)vj, ctx->eps,
                 ctx->kcap, ks));
    } else if (ks) {
      CK(apply_K_update_bf16(L.kp, ctx->p.k_mode, ctx->b, ctx->work, s, hk, vj, ctx->eps,
                             ctx->kcap, ks));
    } else {
      CK(apply_K(L.kp, ctx->p.k_mode, ctx->b, ctx->b, ctx->work, 3, s, hk, nullptr, 0.f,
                 ctx->kcap, ks));
      hk(KID_UPDATE, 0);
      launch_update(g, vj, ctx->b, ctx->eps, s, ctx->st);
      hk(KID_UPDATE, 1);
    }
    uc = unx;
    pf ^= 1;
  }
  ctx->u10 = uc;
  CK(cudaGetLastError());
  // The maps and J0_T describe the velocity before the update.
  ctx->maps_valid = false;
  ctx->j0_valid = false;
  return LDDMM_OK;
}

// LDDMM_STEP_GRAPH=0 in the environment launches every iteration's kernels one by one.
bool step_graph_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("LDDMM_STEP_GRAPH");
    return !(v && v[0] == '0');
  }();
  return on;
}

// One iteration, replayed from the recorded graph when it still applies (per-kernel timing
// records each launch instead).  The graph saves the launch gaps between the ~100 kernels.
int run_step(lddmm_ctx* ctx) {
  if (ctx->prof_on || !step_graph_enabled()) return record_step(ctx);
  if (!ctx->step_graph || ctx->g_cur != ctx->cur || ctx->g_eps != ctx->eps || ctx->g_v != ctx->v) {
    if (ctx->step_graph) {
      cudaGraphExecDestroy(ctx->step_graph);
      ctx->step_graph = nullptr;
    }
    if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
    CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeRelaxed));
    cudaStream_t user = ctx->stream;
    ctx->stream = ctx->cap_stream;
    const int rc = record_step(ctx);
    ctx->stream = user;
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    CK(e);
    const cudaError_t ei = cudaGraphInstantiate(&ctx->step_graph, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      ctx->step_graph = nullptr;
      CK(ei);
    }
    ctx->g_cur = ctx->cur;
    ctx->g_eps = ctx->eps;
    ctx->g_v = ctx->v;
    ctx->g_u10 = ctx->u10;
    ctx->g_u01 = ctx->u01;
  }
  CK(cudaGraphLaunch(ctx->step_graph, ctx->stream));
  ctx->u10 = ctx->g_u10;
  ctx->u01 = ctx->g_u01;
  ctx->maps_valid = false;
  ctx->j0_valid = false;
  return LDDMM_OK;
}

// Recompute phi_{1,0}, phi_{0,1} (and optionally J0_T, the energy) for the current v.
int refresh_maps(lddmm_ctx* ctx, bool energy) {
  const Level& L = ctx->levels[ctx->cur];
  const Grid& g = L.g;
  const int T = ctx->p.T;
  const int64_t N = g.N;
  cudaStream_t s = ctx->stream;
  const float dtx = dtv(ctx, L.hx), dty = dtv(ctx, L.hy), dtz = dtv(ctx, L.hz);
  int rc = reset_acc(ctx);
  if (rc) return rc;
  const float* un = nullptr;
  int pb = 0;
  for (int j = T - 1; j >= 0; --j) {
    float* uc = ctx->uB[pb];
    launch_flow_only_back(g, vptr(ctx, j, N), un, uc, dtx, dty, dtz, s, ctx->st, rk_of(ctx), 1);
    un = uc;
    pb ^= 1;
  }
  ctx->u01 = un;
  launch_ereg(g, ctx->v, T, ctx->p.alpha, ctx->p.gamma, 1.0f / (L.hx * L.hx),
              1.0f / (L.hy * L.hy), 1.0f / (L.hz * L.hz), ctx->acc, s, ctx->st);
  const float* uc = nullptr;
  int pf = 0;
  for (int j = 0; j < T; ++j) {
    float* unx = ctx->uF[pf];
    launch_fwd_flow(g, vptr(ctx, j, N), uc, unx, dtx, dty, dtz, j == T - 1, L.I0, L.I1, L.M,
                    ctx->J0T, ctx->acc, s, ctx->st, rk_of(ctx), 0);
    uc = unx;
    pf ^= 1;
  }
  ctx->u10 = uc;
  CK(cudaGetLastError());
  ctx->maps_valid = true;
  ctx->j0_valid = true;
  (void)energy;
  return LDDMM_OK;
}

// The iteration leaves phi_{0,1} in the quad layout (phi_{1,0} is planar); entry points that
// read it (the inverse warp, landmarks, the map getter) take a planar copy in the K work buffer,
// which is free between iterations.
const float* planar_map(lddmm_ctx* ctx, const float* quad) {
  launch_quad_to_planar(quad, ctx->work, ctx->levels[ctx->cur].g.N, ctx->stream);
  return ctx->work;
}

int copy_out(lddmm_ctx* ctx, void* dst, const void* src, size_t bytes) {
  CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, ctx->stream));
  if (!is_device_ptr(dst)) return wait_stream(ctx);
  return LDDMM_OK;
}

int change_level(lddmm_ctx* ctx, int level) {
  if (level == ctx->cur) return LDDMM_OK;
  const Level& A = ctx->levels[ctx->cur];
  const Level& B = ctx->levels[level];
  const int T = ctx->p.T;
  launch_upsample(A.g, B.g, (float)B.factor / (float)A.factor, ctx->v, ctx->v_tmp, 3 * T,
                  ctx->stream, ctx->st);
  CK(cudaGetLastError());
  std::swap(ctx->v, ctx->v_tmp);
  ctx->cur = level;
  ctx->maps_valid = false;
  ctx->j0_valid = false;
  ctx->last_E = -1.0;
  ctx->have_prev = false;
  return LDDMM_OK;
}

int do_step(lddmm_ctx* ctx, lddmm_energy* out) {
  // flags bit 0: backtracking.  If E(v_k) > E(v_{k-1}), the previous update overshot: go back
  // to v_{k-1} (kept in v_prev), halve the step and redo that iteration.
  const bool backtrack = (ctx->p.flags & 1) != 0;
  const Level& L = ctx->levels[ctx->cur];
  const size_t vbytes = (size_t)ctx->p.T * 3 * L.g.N * ctx->es;
  for (int attempt = 0; attempt < 30; ++attempt) {
    if (backtrack) CK(cudaMemcpyAsync(ctx->v_tmp, ctx->v, vbytes, cudaMemcpyDeviceToDevice, ctx->stream));
    int rc = run_step(ctx);
    if (rc) return rc;
    ++ctx->iter;  // counts enqueued iterations, also when a later wait times out
    if (!out && !backtrack) return LDDMM_OK;
    lddmm_energy e{};
    rc = read_energy(ctx, &e, true);
    if (rc) return rc;
    if (backtrack && ctx->have_prev && e.total > ctx->last_E) {
      CK(cudaMemcpyAsync(ctx->v, ctx->v_prev, vbytes, cudaMemcpyDeviceToDevice, ctx->stream));
      ctx->eps *= 0.5f;
      ctx->have_prev = false;
      --ctx->iter;
      continue;
    }
    if (backtrack) { std::swap(ctx->v_prev, ctx->v_tmp); ctx->have_prev = true; }
    ctx->last_E = e.total;
    if (out) *out = e;
    return LDDMM_OK;
  }
  return fail(ctx, LDDMM_ERR_STATE, "backtracking did not find a decreasing step");
}

}  // namespace

namespace lddmm {
// The message lddmm_last_error(NULL) returns on this thread (entry points without a context).
void set_context_free_error(const char* msg) { g_global_error = msg; }
}  // namespace lddmm

extern "C" {

int lddmm_default_params(lddmm_params* p, int nx, int ny, int nz) {
  if (!p) return fail(nullptr, LDDMM_ERR_INVALID_ARG, "params is NULL");
  std::memset(p, 0, sizeof(*p));
  p->nx = nx; p->ny = ny; p->nz = nz;
  p->hx = p->hy = p->hz = 1.0f;
  p->T = 10;
  p->alpha = 0.02f; p->gamma = 1.0f; p->sigma = 0.1f;
  p->epsilon = 1e-3f;
  p->iterations = 20;
  p->num_levels = 1;
  p->level_factor[0] = 1;
  p->k_mode = LDDMM_K_FP32;
  p->flags = 0;
  p->timeout_s = 600.0f;
  return LDDMM_OK;
}

int lddmm_create(const lddmm_params* p, const float* I0, const float* I1, const float* M,
                 void* stream, lddmm_ctx** out) {
  if (!out) return fail(nullptr, LDDMM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  std::string why;
  int rc = validate(p, why);
  if (rc) return fail(nullptr, rc, why);
  if (!I0 || !I1) return fail(nullptr, LDDMM_ERR_INVALID_ARG, "I0 and I1 are required");
  lddmm_ctx* ctx = new (std::nothrow) lddmm_ctx();
  if (!ctx) return fail(nullptr, LDDMM_ERR_OOM, "host allocation failed");
  g_fail_alloc_countdown = env_int("LDDMM_TEST_FAIL_ALLOC");
  // Test hook (environment LDDMM_TEST_POLL_LIMIT=n): each pipeline wait of the pre-split
  // tensor-core pass gives up after n probes, so that the abort path can be exercised.
  const int poll_limit = env_int("LDDMM_TEST_POLL_LIMIT");
  ctx->p = *p;
  ctx->eps = p->epsilon;
  ctx->st = p->storage;
  ctx->es = p->storage ? 2 : 4;
  auto bail = [&](int code) {
    std::string msg = ctx->err;
    release(ctx);
    delete ctx;
    return fail(nullptr, code, msg);
  };
  ctx->stream = (cudaStream_t)stream;  // NULL: the legacy default stream
  {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
      cudaGetLastError();
      ctx->err = "no usable CUDA device";
      return bail(LDDMM_ERR_CUDA);
    }
  }
  const int nl = p->num_levels;
  ctx->levels.resize(nl);
  for (int l = 0; l < nl; ++l) {
    Level& L = ctx->levels[l];
    L.factor = p->level_factor[l];
    L.g.nx = (p->nx + L.factor - 1) / L.factor;
    L.g.ny = (p->ny + L.factor - 1) / L.factor;
    L.g.nz = (p->nz + L.factor - 1) / L.factor;
    L.g.N = L.g.nx * L.g.ny * L.g.nz;
    L.hx = p->hx * L.factor; L.hy = p->hy * L.factor; L.hz = p->hz * L.factor;
  }
  const int64_t N = ctx->levels.back().g.N;
  ctx->Nmax = N;
  ctx->kcap = 3 * N;
  for (int l = 0; l < nl; ++l) {
    const Grid& g = ctx->levels[l].g;
    ctx->kcap = std::max<int64_t>(ctx->kcap, ks_field_floats(g.nx, g.ny, g.nz, 3));
  }
  const int64_t T = p->T;
  auto A = [&](cudaError_t e) {
    if (e != cudaSuccess) {
      ctx->err = std::string("device allocation: ") + cudaGetErrorString(e);
      return false;
    }
    return true;
  };
  bool ok = true;
  for (int l = 0; l < nl && ok; ++l) {
    Level& L = ctx->levels[l];
    const int64_t ie = (L.g.N * (int64_t)ctx->es + 3) / 4;   // image storage, in floats
    ok = A(dalloc(&L.I0, ie)) && A(dalloc(&L.I1, ie)) && A(dalloc(&L.M, ie)) &&
         A(dalloc(&L.IM, 2 * ie)) &&
         A(kplan_create(&L.kp, L.g.nx, L.g.ny, L.g.nz, L.hx, L.hy, L.hz, p->alpha, p->gamma));
    L.kp.poll_limit = poll_limit > 0 ? (uint32_t)poll_limit : 0u;
  }
  const int64_t ve = (T * 3 * N * (int64_t)ctx->es + 3) / 4;  // velocity storage, in floats
  ok = ok && A(dalloc(&ctx->v, ve)) && A(dalloc(&ctx->v_tmp, ve)) &&
       A(dalloc(&ctx->uB[0], 4 * N)) && A(dalloc(&ctx->uB[1], 4 * N)) &&
       A(dalloc(&ctx->uF[0], 4 * N)) && A(dalloc(&ctx->uF[1], 4 * N)) &&
       A(dalloc(&ctx->J1, T * N)) && A(dalloc(&ctx->W, T * N)) && A(dalloc(&ctx->b, ctx->kcap)) &&
       A(dalloc(&ctx->work, ctx->kcap)) && A(dalloc(&ctx->J0T, N)) && A(dalloc(&ctx->stage, 3 * N)) &&
       A(dalloc(&ctx->acc, 1)) && A(dalloc(&ctx->acc_init, 1)) && A(dalloc(&ctx->flag, 1)) &&
       A(dalloc(&ctx->hist, 3 * 65536)) &&
       A(cudaMallocHost((void**)&ctx->acc_host, sizeof(Acc)));
  if (ok && (p->flags & 1)) ok = A(dalloc(&ctx->v_prev, ve));
  g_fail_alloc_countdown = 0;
  if (!ok) return bail(LDDMM_ERR_OOM);
  if (cudaMemsetAsync(ctx->v, 0, (size_t)ve * sizeof(float), ctx->stream) != cudaSuccess) {
    ctx->err = "memset failed";
    return bail(LDDMM_ERR_CUDA);
  }
  // the accumulators' start value, copied from pinned memory in stream order (the pinned block
  // is next written by the first energy read, which the stream orders after this copy)
  *ctx->acc_host = acc_start();
  if (cudaMemcpyAsync(ctx->acc_init, ctx->acc_host, sizeof(Acc), cudaMemcpyHostToDevice,
                      ctx->stream) != cudaSuccess) {
    ctx->err = "copy of the accumulator start value failed";
    return bail(LDDMM_ERR_CUDA);
  }
  rc = load_images(ctx, I0, I1, M);
  if (rc) return bail(rc);
  ctx->cur = 0;
  *out = ctx;
  return LDDMM_OK;
}

int lddmm_set_images(lddmm_ctx* ctx, const float* I0, const float* I1, const float* M) {
  if (!ctx || !I0 || !I1) return fail(ctx, LDDMM_ERR_INVALID_ARG, "NULL argument");
  return load_images(ctx, I0, I1, M);
}

int lddmm_step(lddmm_ctx* ctx, lddmm_energy* out) {
  if (!ctx) return fail(nullptr, LDDMM_ERR_INVALID_ARG, "ctx is NULL");
  return do_step(ctx, out);
}

int lddmm_register(lddmm_ctx* ctx, lddmm_energy* trace, int trace_len) {
  if (!ctx) return fail(nullptr, LDDMM_ERR_INVALID_ARG, "ctx is NULL");
  if (trace_len < 0 || (trace_len > 0 && !trace)) return fail(ctx, LDDMM_ERR_INVALID_ARG, "bad trace");
  int k = 0;
  for (int l = ctx->cur; l < (int)ctx->levels.size(); ++l) {
    int rc = change_level(ctx, l);
    if (rc) return rc;
    for (int it = 0; it < ctx->p.iterations; ++it) {
      lddmm_energy e{};
      rc = do_step(ctx, k < trace_len ? &e : nullptr);
      if (rc) return rc;
      if (k < trace_len) trace[k] = e;
      ++k;
    }
  }
  return wait_stream(ctx);
}

int lddmm_set_level(lddmm_ctx* ctx, int level) {
  if (!ctx) return fail(nullptr, LDDMM_ERR_INVALID_ARG, "ctx is NULL");
  if (level < 0 || level >= (int)ctx->levels.size()) return fail(ctx, LDDMM_ERR_INVALID_ARG, "bad level");
  return change_level(ctx, level);
}

int lddmm_grid(lddmm_ctx* ctx, int* nx, int* ny, int* nz, int* level) {
  if (!ctx) return fail(nullptr, LDDMM_ERR_INVALID_ARG, "ctx is NULL");
  const Grid& g = ctx->levels[ctx->cur].g;
  if (nx) *nx = g.nx;
  if (ny) *ny = g.ny;
  if (nz) *nz = g.nz;
  if (level) *level = ctx->cur;
  return LDDMM_OK;
}

int lddmm_warp(lddmm_ctx* ctx, const float* src, float* dst, int direction) {
  if (!ctx || !src || !dst) return fail(ctx, LDDMM_ERR_INVALID_ARG, "NULL argument");
  if (direction != 0 && direction != 1) return fail(ctx, LDDMM_ERR_INVALID_ARG, "direction must be 0 or 1");
  int rc;
  if (!ctx->maps_valid && (rc = refresh_maps(ctx, false))) return rc;
  const Grid& g = ctx->levels[ctx->cur].g;
  const float* s = field_src(ctx, src, g.N, ctx->stage, &rc);
  if (rc) return rc;
  const bool dev = is_device_ptr(dst);
  float* d = dev ? dst : ctx->stage + g.N;
  launch_warp(g, s, direction == 0 ? ctx->u10 : planar_map(ctx, ctx->u01), d, ctx->stream);
  CK(cudaGetLastError());
  if (!dev) return copy_out(ctx, dst, d, g.N * sizeof(float));
  return LDDMM_OK;
}

int lddmm_transfer_labels(lddmm_ctx* ctx, const uint16_t* L0, uint16_t* dst) {
  if (!ctx || !L0 || !dst) return fail(ctx, LDDMM_ERR_INVALID_ARG, "NULL argument");
  int rc;
  if (!ctx->maps_valid && (rc = refresh_maps(ctx, false))) return rc;
  const Grid& g = ctx->levels[ctx->cur].g;
  const uint16_t* s = L0;
  uint16_t* st = reinterpret_cast<uint16_t*>(ctx->stage);
  if (!is_device_ptr(L0)) {
    CK(cudaMemcpyAsync(st, L0, g.N * sizeof(uint16_t), cudaMemcpyDefault, ctx->stream));
    s = st;
  }
  const bool dev = is_device_ptr(dst);
  uint16_t* d = dev ? dst : st + g.N;
  launch_labels(g, s, ctx->u10, d, ctx->stream);
  CK(cudaGetLastError());
  if (!dev) return copy_out(ctx, dst, d, g.N * sizeof(uint16_t));
  return LDDMM_OK;
}

int lddmm_get_velocity(lddmm_ctx* ctx, float* dst) {
  if (!ctx || !dst) return fail(ctx, LDDMM_ERR_INVALID_ARG, "NULL argument");
  const Grid& g = ctx->levels[ctx->cur].g;
  if (ctx->st == 0) return copy_out(ctx, dst, ctx->v, (size_t)ctx->p.T * 3 * g.N * sizeof(float));
  // bf16 storage: convert one time step at a time through the staging buffer
  for (int j = 0; j < ctx->p.T; ++j) {
    launch_from_storage(vptr(ctx, j, g.N), ctx->stage, 3 * (int64_t)g.N, ctx->stream, ctx->st);
    int rc = copy_out(ctx, dst + (size_t)j * 3 * g.N, ctx->stage, (size_t)3 * g.N * sizeof(float));
    if (rc) return rc;
  }
  return wait_stream(ctx);
}

int lddmm_set_velocity(lddmm_ctx* ctx, const float* src) {
  if (!ctx || !src) return fail(ctx, LDDMM_ERR_INVALID_ARG, "NULL argument");
  const Grid& g = ctx->levels[ctx->cur].g;
  const int64_t n = (int64_t)ctx->p.T * 3 * g.N;
  int rc;
  if (ctx->st == 0) {
    CK(cudaMemcpyAsync(ctx->v, src, n * sizeof(float), cudaMemcpyDefault, ctx->stream));
    if ((rc = check_finite(ctx, ctx->v, n, "velocity"))) return rc;
  } else {
    for (int j = 0; j < ctx->p.T; ++j) {
      CK(cudaMemcpyAsync(ctx->stage, src + (size_t)j * 3 * g.N, (size_t)3 * g.N * sizeof(float),
                         cudaMemcpyDefault, ctx->stream));
      if ((rc = check_finite(ctx, ctx->stage, 3 * (int64_t)g.N, "velocity"))) return rc;
      launch_to_storage(ctx->stage, vptr(ctx, j, g.N), 3 * (int64_t)g.N, ctx->stream, ctx->st);
    }
  }
  ctx->maps_valid = false;
  ctx->j0_valid = false;
  ctx->last_E = -1.0;
  return LDDMM_OK;
}

int lddmm_get_field(lddmm_ctx* ctx, int which, float* dst) {
  if (!ctx || !dst) return fail(ctx, LDDMM_ERR_INVALID_ARG, "NULL argument");
  const Level& L = ctx->levels[ctx->cur];
  const int64_t N = L.g.N;
  int rc;
  switch (which) {
    case LDDMM_FIELD_U10:
    case LDDMM_FIELD_U01:
    case LDDMM_FIELD_J0:
      if (!ctx->maps_valid && (rc = refresh_maps(ctx, false))) return rc;
      if (which == LDDMM_FIELD_U10) return copy_out(ctx, dst, ctx->u10, 3 * N * sizeof(float));
      if (which == LDDMM_FIELD_U01) {
        if (is_device_ptr(dst)) {
          launch_quad_to_planar(ctx->u01, dst, N, ctx->stream);
          CK(cudaGetLastError());
          return LDDMM_OK;
        }
        return copy_out(ctx, dst, planar_map(ctx, ctx->u01), 3 * N * sizeof(float));
      }
      return copy_out(ctx, dst, ctx->J0T, N * sizeof(float));
    case LDDMM_FIELD_I0:
    case LDDMM_FIELD_I1:
    case LDDMM_FIELD_M: {
      const void* src = which == LDDMM_FIELD_I0 ? (const void*)L.I0
                        : which == LDDMM_FIELD_I1 ? (const void*)L.I1 : (const void*)L.M;
      launch_from_storage(src, ctx->stage, N, ctx->stream, ctx->st);
      return copy_out(ctx, dst, ctx->stage, N * sizeof(float));
    }
    default: return fail(ctx, LDDMM_ERR_INVALID_ARG, "unknown field");
  }
}

int lddmm_apply_K(lddmm_ctx* ctx, const float* src, float* dst) {
  if (!ctx || !src || !dst) return fail(ctx, LDDMM_ERR_INVALID_ARG, "NULL argument");
  const Level& L = ctx->levels[ctx->cur];
  const int64_t N = L.g.N;
  CK(cudaMemcpyAsync(ctx->stage, src, N * sizeof(float), cudaMemcpyDefault, ctx->stream));
  CK(apply_K(L.kp, ctx->p.k_mode, ctx->stage, ctx->stage, ctx->work, 1, ctx->stream, Hook(),
             nullptr, 0.f, std::min<int64_t>(3 * ctx->Nmax, ctx->kcap)));
  return copy_out(ctx, dst, ctx->stage, N * sizeof(float));
}

int lddmm_energy_eval(lddmm_ctx* ctx, lddmm_energy* out) {
  if (!ctx || !out) return fail(ctx, LDDMM_ERR_INVALID_ARG, "NULL argument");
  int rc = refresh_maps(ctx, true);
  if (rc) return rc;
  return read_energy(ctx, out, false);
}

int lddmm_dice(lddmm_ctx* ctx, const uint16_t* A, const uint16_t* B, int64_t n, double* out) {
  if (!ctx || !A || !B || !out || n < 0) return fail(ctx, LDDMM_ERR_INVALID_ARG, "bad argument");
  const uint16_t* a = A;
  const uint16_t* b = B;
  uint16_t* tmp = nullptr;
  const bool da = is_device_ptr(A), db = is_device_ptr(B);
  if (!da || !db) {
    CK(cudaMalloc((void**)&tmp, (size_t)2 * n * sizeof(uint16_t) + 16));
    if (!da) { CK(cudaMemcpyAsync(tmp, A, n * 2, cudaMemcpyDefault, ctx->stream)); a = tmp; }
    if (!db) { CK(cudaMemcpyAsync(tmp + n, B, n * 2, cudaMemcpyDefault, ctx->stream)); b = tmp + n; }
  }
  CK(cudaMemsetAsync(ctx->hist, 0, 3 * 65536 * sizeof(unsigned long long), ctx->stream));
  launch_dice_hist(a, b, n, ctx->hist, ctx->stream);
  CK(cudaGetLastError());
  std::vector<unsigned long long> h(3 * 65536);
  CK(cudaMemcpyAsync(h.data(), ctx->hist, h.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
  int rc = wait_stream(ctx);
  if (tmp) cudaFree(tmp);
  if (rc) return rc;
  double s = 0.0;
  int cnt = 0;
  for (int l = 1; l < 65536; ++l) {
    const unsigned long long na = h[l], nb = h[65536 + l], ni = h[2 * 65536 + l];
    if (na + nb == 0) continue;
    s += 2.0 * (double)ni / (double)(na + nb);
    ++cnt;
  }
  *out = cnt ? s / cnt : 1.0;
  return LDDMM_OK;
}

int lddmm_surface_distance(lddmm_ctx* ctx, const uint8_t* A, const uint8_t* B, double out[4]) {
  if (!ctx || !A || !B || !out) return fail(ctx, LDDMM_ERR_INVALID_ARG, "NULL argument");
  const Level& L = ctx->levels[ctx->cur];
  const Grid& g = L.g;
  cudaStream_t s = ctx->stream;
  // scratch: host masks, the two counters, then the lists and distances once sized
  uint8_t* mk = nullptr;
  unsigned* cnt = nullptr;
  int4* list = nullptr;
  double* d = nullptr;
  double* st = nullptr;
  auto done = [&](int rc) {
    cudaStreamSynchronize(s);
    cudaFree(mk); cudaFree(cnt); cudaFree(list); cudaFree(d); cudaFree(st);
    cudaGetLastError();
    return rc;
  };
  const uint8_t* ma = A;
  const uint8_t* mb = B;
  const bool da = is_device_ptr(A), db = is_device_ptr(B);
  if (cudaMalloc((void**)&cnt, 2 * sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc((void**)&st, 3 * sizeof(double)) != cudaSuccess)
    return done(fail(ctx, LDDMM_ERR_OOM, "device allocation failed"));
  if (!da || !db) {
    if (cudaMalloc((void**)&mk, 2 * (size_t)g.N) != cudaSuccess)
      return done(fail(ctx, LDDMM_ERR_OOM, "device allocation failed"));
    if (!da) { cudaMemcpyAsync(mk, A, g.N, cudaMemcpyDefault, s); ma = mk; }
    if (!db) { cudaMemcpyAsync(mk + g.N, B, g.N, cudaMemcpyDefault, s); mb = mk + g.N; }
  }
  // count the surface voxels, then list them
  unsigned h[2] = {0, 0};
  cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned), s);
  surface_list(g, ma, nullptr, cnt, 0u, s);
  surface_list(g, mb, nullptr, cnt + 1, 0u, s);
  cudaMemcpyAsync(h, cnt, sizeof(h), cudaMemcpyDeviceToHost, s);
  int rc = wait_stream(ctx);
  if (rc) return done(rc);
  if (cudaGetLastError() != cudaSuccess) return done(fail(ctx, LDDMM_ERR_CUDA, "surface count failed"));
  if (h[0] == 0 || h[1] == 0) return done(fail(ctx, LDDMM_ERR_INVALID_ARG, "a mask has no surface voxel"));
  const unsigned na = h[0], nb = h[1];
  if (cudaMalloc((void**)&list, (size_t)(na + nb) * sizeof(int4)) != cudaSuccess ||
      cudaMalloc((void**)&d, (size_t)(na + nb) * sizeof(double)) != cudaSuccess)
    return done(fail(ctx, LDDMM_ERR_OOM, "device allocation failed"));
  cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned), s);
  surface_list(g, ma, list, cnt, na, s);
  surface_list(g, mb, list + na, cnt + 1, nb, s);
  nearest_distances(list, na, list + na, nb, L.hx, L.hy, L.hz, d, s);
  nearest_distances(list + na, nb, list, na, L.hx, L.hy, L.hz, d + na, s);
  const unsigned n = na + nb;
  order_stats(d, n, (n - 1) / 2, n / 2, st, s);
  double r[3];
  cudaMemcpyAsync(r, st, sizeof(r), cudaMemcpyDeviceToHost, s);
  if (cudaGetLastError() != cudaSuccess) return done(fail(ctx, LDDMM_ERR_CUDA, "surface distance launch failed"));
  rc = wait_stream(ctx);
  if (rc) return done(rc);
  out[0] = r[0];
  out[1] = 0.5 * (r[1] + r[2]);
  out[2] = (double)na;
  out[3] = (double)nb;
  return done(LDDMM_OK);
}

int lddmm_shoot(lddmm_ctx* ctx, const float* v0) {
  if (!ctx || !v0) return fail(ctx, LDDMM_ERR_INVALID_ARG, "NULL argument");
  if (ctx->st != 0) return fail(ctx, LDDMM_ERR_INVALID_ARG, "shooting needs float storage");
  if (rk_of(ctx)) return fail(ctx, LDDMM_ERR_INVALID_ARG, "shooting uses the one-lookup flow");
  const Level& L = ctx->levels[ctx->cur];
  const Grid& g = L.g;
  const int T = ctx->p.T;
  const int64_t N = g.N, F = 3 * N;
  cudaStream_t s = ctx->stream;
  const float dtx = dtv(ctx, L.hx), dty = dtv(ctx, L.hy), dtz = dtv(ctx, L.hz);
  const float ihx2 = 1.0f / (L.hx * L.hx), ihy2 = 1.0f / (L.hy * L.hy), ihz2 = 1.0f / (L.hz * L.hz);
  float* v = reinterpret_cast<float*>(ctx->v);
  CK(cudaMemcpyAsync(v, v0, F * sizeof(float), cudaMemcpyDefault, s));
  int rc;
  if ((rc = check_finite(ctx, v, F, "v0"))) return rc;
  // m_0 = L (L v_0) in stage
  launch_apply_L3(g, v, ctx->work, ctx->p.alpha, ctx->p.gamma, ihx2, ihy2, ihz2, 1.0f, false, s);
  launch_apply_L3(g, ctx->work, ctx->stage, ctx->p.alpha, ctx->p.gamma, ihx2, ihy2, ihz2, 1.0f,
                  false, s);
  const float* uc = nullptr;
  int pf = 0;
  for (int j = 0; j + 1 < T; ++j) {
    float* un = ctx->uF[pf];
    launch_flow_only_fwd(g, v + (int64_t)j * F, uc, un, dtx, dty, dtz, s, 0, 0);
    CK(transport_momentum(g, ctx->stage, un, L.hx, L.hy, L.hz, ctx->b, s));
    CK(apply_K(L.kp, ctx->p.k_mode, ctx->b, ctx->b, ctx->work, 3, s, Hook(), nullptr, 0.f,
               ctx->kcap));
    CK(cudaMemcpyAsync(v + (int64_t)(j + 1) * F, ctx->b, F * sizeof(float),
                       cudaMemcpyDeviceToDevice, s));
    uc = un;
    pf ^= 1;
  }
  CK(cudaGetLastError());
  ctx->maps_valid = false;
  ctx->j0_valid = false;
  ctx->last_E = -1.0;
  return LDDMM_OK;
}

int lddmm_landmark_error(lddmm_ctx* ctx, const float* xk, const float* yk, int n, double* err) {
  if (!ctx || !xk || !yk || !err || n < 0) return fail(ctx, LDDMM_ERR_INVALID_ARG, "bad argument");
  if (n == 0) return LDDMM_OK;
  int rc;
  if (!ctx->maps_valid && (rc = refresh_maps(ctx, false))) return rc;
  const Level& L = ctx->levels[ctx->cur];
  cudaStream_t s = ctx->stream;
  float* pts = nullptr;
  double* e = nullptr;
  const bool dx = is_device_ptr(xk), dy = is_device_ptr(yk), de = is_device_ptr(err);
  if (cudaMalloc((void**)&pts, (size_t)6 * n * sizeof(float)) != cudaSuccess ||
      cudaMalloc((void**)&e, (size_t)n * sizeof(double)) != cudaSuccess) {
    cudaFree(pts);
    cudaGetLastError();
    return fail(ctx, LDDMM_ERR_OOM, "device allocation failed");
  }
  cudaMemcpyAsync(pts, xk, (size_t)3 * n * sizeof(float), dx ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(pts + 3 * n, yk, (size_t)3 * n * sizeof(float), dy ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
  landmark_errors(L.g, planar_map(ctx, ctx->u01), pts, pts + 3 * n, n, L.hx, L.hy, L.hz, e, s);
  cudaMemcpyAsync(err, e, (size_t)n * sizeof(double), de ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
  const cudaError_t le = cudaGetLastError();
  rc = wait_stream(ctx);
  cudaFree(pts);
  cudaFree(e);
  if (le != cudaSuccess) return fail(ctx, LDDMM_ERR_CUDA, cudaGetErrorString(le));
  return rc;
}

namespace {
// Bounded wait for calls without a context.
int wait_plain(cudaStream_t s, double limit = 600.0) {
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaStreamQuery(s);
    if (e == cudaSuccess) return LDDMM_OK;
    if (e != cudaErrorNotReady)
      return fail(nullptr, LDDMM_ERR_CUDA, std::string("stream: ") + cudaGetErrorString(e));
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el > limit) return fail(nullptr, LDDMM_ERR_TIMEOUT, "timed out waiting for the GPU stream");
    std::this_thread::sleep_for(std::chrono::microseconds(el < 0.01 ? 5 : 200));
  }
}
}  // namespace

int lddmm_histogram_match(const float* I0, const float* M0, const float* I1, const float* M1,
                          int64_t n, int bins, int points, float* out, void* stream) {
  if (!I0 || !M0 || !I1 || !M1 || !out || n <= 0 || bins < 1 || bins > 1024 || points < 0 ||
      points > 64)
    return fail(nullptr, LDDMM_ERR_INVALID_ARG, "bad argument");
  const void* ps[5] = {I0, M0, I1, M1, out};
  for (const void* p : ps)
    if (!is_device_ptr(p)) return fail(nullptr, LDDMM_ERR_INVALID_ARG, "device memory expected");
  cudaStream_t s = (cudaStream_t)stream;
  // scratch: two range records (3 ints each, 16-byte slots), two histograms, the nodes
  char* scr = nullptr;
  const size_t hb = (size_t)bins * sizeof(unsigned long long);
  if (cudaMalloc((void**)&scr, 32 + 2 * hb + 2 * 66 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, LDDMM_ERR_OOM, "device allocation failed");
  }
  int* st0 = reinterpret_cast<int*>(scr);
  int* st1 = st0 + 4;
  unsigned long long* c0 = reinterpret_cast<unsigned long long*>(scr + 32);
  unsigned long long* c1 = c0 + bins;
  double* nodes = reinterpret_cast<double*>(scr + 32 + 2 * hb);
  int cnt[8] = {0};
  cudaError_t e = masked_range(I0, M0, n, st0, s);
  if (e == cudaSuccess) e = masked_range(I1, M1, n, st1, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(cnt, scr, 32, cudaMemcpyDeviceToHost, s);
  int rc = e == cudaSuccess ? wait_plain(s) : fail(nullptr, LDDMM_ERR_CUDA, cudaGetErrorString(e));
  if (rc == LDDMM_OK && (cnt[2] == 0 || cnt[6] == 0))
    rc = fail(nullptr, LDDMM_ERR_INVALID_ARG, "a mask is empty");
  if (rc == LDDMM_OK) {
    e = masked_hist(I0, M0, n, st0, bins, c0, s);
    if (e == cudaSuccess) e = masked_hist(I1, M1, n, st1, bins, c1, s);
    if (e == cudaSuccess) e = match_nodes(st0, c0, st1, c1, bins, points, nodes, s);
    if (e == cudaSuccess) e = apply_match(I0, M0, n, nodes, points, out, s);
    rc = e == cudaSuccess ? wait_plain(s) : fail(nullptr, LDDMM_ERR_CUDA, cudaGetErrorString(e));
  }
  cudaFree(scr);
  return rc;
}

int lddmm_mask_morphology(const float* I, int nx, int ny, int nz, float threshold, int r_open,
                          int r_close, uint8_t* out, void* stream) {
  if (!I || !out || nx < 1 || ny < 1 || nz < 1 || r_open < 0 || r_open > 16 || r_close < 0 ||
      r_close > 16)
    return fail(nullptr, LDDMM_ERR_INVALID_ARG, "bad argument");
  if (!is_device_ptr(I) || !is_device_ptr(out))
    return fail(nullptr, LDDMM_ERR_INVALID_ARG, "device memory expected");
  const Grid g{nx, ny, nz, (int64_t)nx * ny * nz};
  cudaStream_t s = (cudaStream_t)stream;
  uint8_t* tmp = nullptr;
  if (cudaMalloc((void**)&tmp, (size_t)g.N) != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, LDDMM_ERR_OOM, "device allocation failed");
  }
  // out -> tmp -> out per pair of operations
  cudaError_t e = threshold_mask(I, g.N, threshold, out, s);
  if (e == cudaSuccess && r_open > 0) {
    e = ball_op(g, out, r_open, true, tmp, s);
    if (e == cudaSuccess) e = ball_op(g, tmp, r_open, false, out, s);
  }
  if (e == cudaSuccess && r_close > 0) {
    e = ball_op(g, out, r_close, false, tmp, s);
    if (e == cudaSuccess) e = ball_op(g, tmp, r_close, true, out, s);
  }
  const int rc = e == cudaSuccess ? wait_plain(s) : fail(nullptr, LDDMM_ERR_CUDA, cudaGetErrorString(e));
  cudaFree(tmp);
  return rc;
}

int lddmm_profile_start(lddmm_ctx* ctx, int max_launches) {
  if (!ctx || max_launches < 1) return fail(ctx, LDDMM_ERR_INVALID_ARG, "bad argument");
  for (cudaEvent_t e : ctx->prof_ev) cudaEventDestroy(e);
  ctx->prof_ev.assign(2 * (size_t)max_launches, nullptr);
  for (auto& e : ctx->prof_ev) CK(cudaEventCreate(&e));
  ctx->prof_kid.assign(max_launches, -1);
  ctx->prof_used = 0;
  ctx->prof_overflow = false;
  ctx->prof_open = -1;
  ctx->prof_on = true;
  return LDDMM_OK;
}

int lddmm_profile_stop(lddmm_ctx* ctx, lddmm_kernel_stat* out, int max_out, int* n_out) {
  if (!ctx) return fail(nullptr, LDDMM_ERR_INVALID_ARG, "ctx is NULL");
  ctx->prof_on = false;
  int rc = wait_stream(ctx);
  if (rc) return rc;
  std::vector<double> tot(KID_COUNT, 0.0);
  std::vector<int> cnt(KID_COUNT, 0);
  for (size_t i = 0; i < ctx->prof_used; ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ctx->prof_ev[2 * i], ctx->prof_ev[2 * i + 1]));
    tot[ctx->prof_kid[i]] += ms;
    cnt[ctx->prof_kid[i]] += 1;
  }
  int n = 0;
  for (int k = 0; k < KID_COUNT; ++k) {
    if (!cnt[k]) continue;
    if (out && n < max_out) {
      std::memset(&out[n], 0, sizeof(lddmm_kernel_stat));
      std::strncpy(out[n].name, kernel_name(k), sizeof(out[n].name) - 1);
      out[n].launches = cnt[k];
      out[n].total_ms = tot[k];
    }
    ++n;
  }
  if (n_out) *n_out = n;
  for (cudaEvent_t e : ctx->prof_ev) cudaEventDestroy(e);
  ctx->prof_ev.clear();
  if (ctx->prof_overflow) return fail(ctx, LDDMM_ERR_STATE, "profile buffer overflowed (raise max_launches)");
  return LDDMM_OK;
}

int lddmm_energy_grad(lddmm_ctx* ctx, const float* v, float* grad, double* E) {
  if (!ctx || !grad) return fail(ctx, LDDMM_ERR_INVALID_ARG, "NULL argument");
  if (ctx->st != 0) return fail(ctx, LDDMM_ERR_INVALID_ARG, "the exact gradient needs float storage");
  if (rk_of(ctx))
    return fail(ctx, LDDMM_ERR_INVALID_ARG, "the exact gradient is built for the one-lookup flow");
  const Level& L = ctx->levels[ctx->cur];
  const Grid& g = L.g;
  const int T = ctx->p.T;
  const int64_t N = g.N, F = 3 * N;
  cudaStream_t s = ctx->stream;
  int rc;
  if (v && (rc = lddmm_set_velocity(ctx, v))) return rc;
  // forward maps: all T+1, or checkpoints every c steps plus a recomputed segment of c
  const bool ckpt = (ctx->p.flags & 2) != 0;
  int c = 1;
  while (c * c < T) ++c;
  const int nslots = ckpt ? (T - 1) / c + 2 : T + 1;   // checkpoints u_0, u_c, ..., and u_T
  if (ctx->uall_slots < nslots) {
    if (ctx->uall) cudaFree(ctx->uall);
    ctx->uall = nullptr;
    ctx->uall_slots = 0;
    CK(cudaMalloc((void**)&ctx->uall, (size_t)nslots * ctx->Nmax * 3 * sizeof(float)));
    ctx->uall_slots = nslots;
  }
  if (ckpt && ctx->seg_slots < c) {
    if (ctx->seg) cudaFree(ctx->seg);
    ctx->seg = nullptr;
    ctx->seg_slots = 0;
    CK(cudaMalloc((void**)&ctx->seg, (size_t)c * ctx->Nmax * 3 * sizeof(float)));
    ctx->seg_slots = c;
  }
  if (!ctx->gA) CK(cudaMalloc((void**)&ctx->gA, (size_t)ctx->Nmax * 3 * sizeof(float)));
  if (!ctx->gB) CK(cudaMalloc((void**)&ctx->gB, (size_t)ctx->Nmax * 3 * sizeof(float)));
  const float dtx = dtv(ctx, L.hx), dty = dtv(ctx, L.hy), dtz = dtv(ctx, L.hz);
  const float ihx2 = 1.0f / (L.hx * L.hx), ihy2 = 1.0f / (L.hy * L.hy), ihz2 = 1.0f / (L.hz * L.hz);
  auto slot_of = [&](int j) -> float* {   // storage of u_j when it is kept
    if (!ckpt) return ctx->uall + (size_t)j * F;
    if (j == T) return ctx->uall + (size_t)(nslots - 1) * F;
    return ctx->uall + (size_t)(j / c) * F;
  };
  // forward sweep (energy, u_j kept or checkpointed)
  if ((rc = reset_acc(ctx))) return rc;
  CK(cudaMemsetAsync(slot_of(0), 0, F * sizeof(float), s));
  launch_ereg(g, ctx->v, T, ctx->p.alpha, ctx->p.gamma, ihx2, ihy2, ihz2, ctx->acc, s, 0);
  const float* uc = nullptr;
  int pf = 0;
  for (int j = 0; j < T; ++j) {
    const bool keep = !ckpt || j + 1 == T || (j + 1) % c == 0;
    float* unx = keep ? slot_of(j + 1) : ctx->uF[pf];
    launch_fwd_flow(g, ctx->v + (int64_t)j * F, uc, unx, dtx, dty, dtz, j == T - 1, L.I0, L.I1,
                    L.M, ctx->J0T, ctx->acc, s, 0);
    uc = unx;
    if (!keep) pf ^= 1;
  }
  CK(cudaGetLastError());
  const bool dev = is_device_ptr(grad);
  float* gout = dev ? grad : ctx->v_tmp;
  // reverse sweep
  const double h3 = (double)L.hx * L.hy * L.hz;
  const double sg = ctx->p.sigma;
  float* gnext = ctx->gA;
  float* gcur = ctx->gB;
  launch_adj_init(g, slot_of(T), L.I0, L.I1, L.M, gnext, (float)(2.0 * h3 / (sg * sg)), s);
  int seg_base = -1;
  for (int j = T - 1; j >= 0; --j) {
    const float* uj;
    if (!ckpt) {
      uj = slot_of(j);
    } else {
      const int k = (j / c) * c;
      if (seg_base != k) {   // recompute u_k .. u_{min(k+c,T)-1} from the checkpoint u_k
        CK(cudaMemcpyAsync(ctx->seg, slot_of(k), F * sizeof(float), cudaMemcpyDeviceToDevice, s));
        for (int i = 1; i < c && k + i < T; ++i)
          launch_flow_only_fwd(g, ctx->v + (int64_t)(k + i - 1) * F, ctx->seg + (size_t)(i - 1) * F,
                               ctx->seg + (size_t)i * F, dtx, dty, dtz, s, 0);
        seg_base = k;
      }
      uj = ctx->seg + (size_t)(j - k) * F;
    }
    float* gradj = gout + (int64_t)j * F;
    if (j > 0) CK(cudaMemsetAsync(gcur, 0, F * sizeof(float), s));
    launch_adj_step(g, ctx->v + (int64_t)j * F, j > 0 ? uj : nullptr, gnext, j > 0 ? gcur : nullptr,
                    gradj, dtx, dty, dtz, s);
    // regulariser: + 2 dt h^3 L(L v_j)
    launch_apply_L3(g, ctx->v + (int64_t)j * F, ctx->work, ctx->p.alpha, ctx->p.gamma, ihx2, ihy2,
                    ihz2, 1.0f, false, s);
    launch_apply_L3(g, ctx->work, gradj, ctx->p.alpha, ctx->p.gamma, ihx2, ihy2, ihz2,
                    (float)(2.0 * h3 / T), true, s);
    std::swap(gnext, gcur);
  }
  CK(cudaGetLastError());
  lddmm_energy e{};
  if ((rc = read_energy(ctx, &e, false))) return rc;
  if (E) *E = e.total;
  if (!dev) {
    CK(cudaMemcpyAsync(grad, gout, (size_t)T * F * sizeof(float), cudaMemcpyDefault, s));
    if ((rc = wait_stream(ctx))) return rc;
  }
  ctx->maps_valid = false;
  ctx->j0_valid = false;
  return LDDMM_OK;
}

int lddmm_set_timeout(lddmm_ctx* ctx, float seconds) {
  if (!ctx) return fail(nullptr, LDDMM_ERR_INVALID_ARG, "ctx is NULL");
  ctx->p.timeout_s = seconds;
  return LDDMM_OK;
}

const char* lddmm_last_error(lddmm_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_global_error.c_str();
}

void lddmm_destroy(lddmm_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (cudaEvent_t e : ctx->prof_ev) cudaEventDestroy(e);
  release(ctx);
  delete ctx;
}

}  // extern "C"
