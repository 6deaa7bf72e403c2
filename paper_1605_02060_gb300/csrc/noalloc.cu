// lddmm_apply_K_noalloc: the smoothing operator K = (gamma - alpha Lap_h)^-2 for callers that
// cannot allocate GPU memory.
//
// Some callers cannot call cudaMalloc: a host callback, a real-time loop that must not stall on
// the allocator, or a process whose GPU memory another framework's pool reserves up front.  This
// entry point therefore allocates nothing.  It runs the same FP32 per-axis real-DFT products as
// lddmm_apply_K with k_mode LDDMM_K_FP32, but its intermediate field and its DFT tables live in
// one file-scope __device__ array of fixed size (kNoAllocFloats floats, about 11.5 MB), which
// every GPU that loads the library keeps until the process exits.
//
// Limits: nx*ny*nz <= 2^21 voxels and every axis <= 512.  All calls share the one array, so
// calls whose work overlaps on the GPU (different streams, or different host threads) race;
// serialise them on one stream.  The tables are written by a kernel on the call's stream when an
// axis's (n, h) differs from what the array holds; the work field is rewritten by every pass
// before it is read, so nothing in the array needs to start at zero.  The first call on a device
// looks up the array's device address (cudaGetSymbolAddress) with that device current; make
// that first call before any stream capture.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/lddmm.h"
#include "kernels.h"

namespace lddmm {
void set_context_free_error(const char* msg);
}

namespace {

constexpr int kNoAllocMaxVoxels = 1 << 21;
constexpr int kNoAllocMaxAxis = 512;
// work field + three R tables (each sized for the largest axis) + three eigenvalue tables
constexpr size_t kNoAllocFloats =
    (size_t)kNoAllocMaxVoxels + 3 * (size_t)kNoAllocMaxAxis * kNoAllocMaxAxis + 3 * kNoAllocMaxAxis;

static __device__ __align__(256) float g_noalloc_scratch[kNoAllocFloats];

constexpr int kMaxDevices = 64;
struct DevState {
  float* base = nullptr;   // device address of g_noalloc_scratch on this device
  int n[3] = {0, 0, 0};    // (n, h) of the tables the array holds per axis (n = 0: none)
  double h[3] = {0, 0, 0};
};
DevState g_dev[kMaxDevices];
std::mutex g_mu;

int nerr(int code, const char* why) {
  lddmm::set_context_free_error(why);
  return code;
}

// R (n x n, row-major) and lambda (n) of one axis: the orthonormal real Fourier basis (constant,
// cos/sin pairs of frequency k = 1.., the Nyquist cosine when n is even) and the eigenvalue of
// the periodic second difference, (2 - 2 cos(2 pi k / n)) / h^2, in double precision with the
// angle k m reduced modulo n, rounded once to float.
__global__ void k_noalloc_tables(float* __restrict__ R, float* __restrict__ lam, int n, double h) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * n) return;
  const int r = i / n, m = i - r * n;
  const int k = (r + 1) / 2;
  const bool is_sin = (r > 0) && (r % 2 == 0);
  const bool nyq = (n % 2 == 0) && (r == n - 1);
  const double two_pi = 6.283185307179586476925286766559;
  const double scale = (r == 0 || nyq) ? sqrt(1.0 / n) : sqrt(2.0 / n);
  const double ang = two_pi * (double)(((long long)k * m) % n) / (double)n;
  R[i] = (float)(scale * (is_sin ? sin(ang) : cos(ang)));
  if (m == 0) lam[r] = (float)((2.0 - 2.0 * cos(two_pi * (double)k / (double)n)) / (h * h));
}

}  // namespace

extern "C" int lddmm_apply_K_noalloc(const float* src, float* dst, int nx, int ny, int nz,
                                     float hx, float hy, float hz, float alpha, float gamma,
                                     void* stream) {
  using namespace lddmm;
  if (!src || !dst) return nerr(LDDMM_ERR_INVALID_ARG, "src and dst are required");
  if (nx < 2 || ny < 2 || nz < 2) return nerr(LDDMM_ERR_INVALID_ARG, "grid sizes must be >= 2");
  if (nx > kNoAllocMaxAxis || ny > kNoAllocMaxAxis || nz > kNoAllocMaxAxis)
    return nerr(LDDMM_ERR_INVALID_ARG, "an axis exceeds 512, the no-alloc limit");
  if ((long long)nx * ny * nz > kNoAllocMaxVoxels)
    return nerr(LDDMM_ERR_INVALID_ARG, "grid exceeds 2^21 voxels, the no-alloc limit");
  if (!(hx > 0 && hy > 0 && hz > 0) || !(gamma > 0) || !(alpha >= 0))
    return nerr(LDDMM_ERR_INVALID_ARG, "need h > 0, gamma > 0, alpha >= 0");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return nerr(LDDMM_ERR_CUDA, "no usable CUDA device");
  }
  // src and dst must be device memory: there is no staging buffer to copy host data through
  for (const void* p : {(const void*)src, (const void*)dst}) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
      cudaGetLastError();
      return nerr(LDDMM_ERR_INVALID_ARG, "src/dst must be device pointers");
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
      return nerr(LDDMM_ERR_INVALID_ARG, "src/dst must be device pointers");
  }
  const int n[3] = {nx, ny, nz};
  const double h[3] = {hx, hy, hz};
  cudaStream_t s = (cudaStream_t)stream;
  float* R[3];
  float* lam[3];
  float* work;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    DevState& ds = g_dev[dev];
    // one-time set-up per device: the device address of the static scratch array (in host code
    // the array's name stands for a host-side shadow, not for device memory)
    if (!ds.base) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return nerr(LDDMM_ERR_CUDA, "cudaGetSymbolAddress of the no-alloc scratch failed");
      }
      ds.base = static_cast<float*>(p);
    }
    work = ds.base;
    float* tab = ds.base + kNoAllocMaxVoxels;
    for (int d = 0; d < 3; ++d) {
      R[d] = tab + (size_t)d * kNoAllocMaxAxis * kNoAllocMaxAxis;
      lam[d] = tab + 3 * (size_t)kNoAllocMaxAxis * kNoAllocMaxAxis + (size_t)d * kNoAllocMaxAxis;
      if (ds.n[d] != n[d] || ds.h[d] != h[d]) {
        const int cnt = n[d] * n[d];
        k_noalloc_tables<<<(cnt + 255) / 256, 256, 0, s>>>(R[d], lam[d], n[d], h[d]);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
          ds.n[d] = 0;
          return nerr(LDDMM_ERR_CUDA, cudaGetErrorString(e));
        }
        ds.n[d] = n[d];
        ds.h[d] = h[d];
      }
    }
  }
  KPlan kp{};
  kp.nx = nx; kp.ny = ny; kp.nz = nz;
  kp.alpha = alpha; kp.gamma = gamma;
  kp.Rx = R[0]; kp.Ry = R[1]; kp.Rz = R[2];
  kp.lx = lam[0]; kp.ly = lam[1]; kp.lz = lam[2];
  cudaError_t e = apply_K(kp, LDDMM_K_FP32, src, dst, work, 1, s);
  if (e != cudaSuccess) return nerr(LDDMM_ERR_CUDA, cudaGetErrorString(e));
  return LDDMM_OK;
}
