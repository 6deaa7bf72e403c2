// lddmm_apply_K_noalloc: the smoothing operator K = (gamma - alpha Lap_h)^-2 for callers that
// cannot allocate GPU memory.
//
// Some callers cannot call cudaMalloc: code running inside a CUDA-graph capture, a host callback,
// a real-time loop that must not stall on the allocator, or a process whose GPU memory is
// reserved up front by another framework's pool.  This entry point therefore allocates nothing.
// It runs the same FP32 per-axis real-DFT products as lddmm_apply_K with k_mode LDDMM_K_FP32,
// but its intermediate field and its DFT tables live in one file-scope __device__ array of fixed
// size (kNoAllocFloats floats, about 11.5 MB), which every GPU that loads the library keeps until
// the process exits.
//
// Limits: nx*ny*nz <= 2^21 voxels and every axis <= 512.  All calls share the one array, so
// calls whose work overlaps on the GPU (different streams, or different host threads) race;
// serialise them on one stream.  Nothing in the array needs to start at zero: each call
// rewrites the tables and every intermediate value it reads.  The first call on a device looks
// up the array's device address (cudaGetSymbolAddress) with that device current; make that first
// call before any stream capture.
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/lddmm.h"
#include "kernels.h"

namespace lddmm {
void host_real_dft_tables(int n, double h, std::vector<float>& R, std::vector<float>& lam);
}

namespace {

constexpr int kNoAllocMaxVoxels = 1 << 21;
constexpr int kNoAllocMaxAxis = 512;
// work field + three R tables + three eigenvalue tables
constexpr size_t kNoAllocFloats =
    (size_t)kNoAllocMaxVoxels + 3 * (size_t)kNoAllocMaxAxis * kNoAllocMaxAxis + 3 * kNoAllocMaxAxis;

static __device__ __align__(256) float g_noalloc_scratch[kNoAllocFloats];

constexpr int kMaxDevices = 64;
float* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Errors are reported by status code only (the message names the cause for readers).
int nerr(int code, const char* /*why*/) { return code; }

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
  // one-time set-up per device: the device address of the static scratch array
  float* base;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) return nerr(LDDMM_ERR_CUDA, "cudaGetSymbolAddress failed");
      g_scratch_addr[dev] = static_cast<float*>(p);
    }
    base = g_scratch_addr[dev];
  }
  const int n[3] = {nx, ny, nz};
  const double h[3] = {hx, hy, hz};
  float* work = base;
  float* R[3];
  float* lam[3];
  float* cursor = base + kNoAllocMaxVoxels;
  for (int d = 0; d < 3; ++d) {
    R[d] = cursor;
    cursor += (size_t)n[d] * n[d];
  }
  for (int d = 0; d < 3; ++d) {
    lam[d] = cursor;
    cursor += n[d];
  }
  cudaStream_t s = (cudaStream_t)stream;
  for (int d = 0; d < 3; ++d) {
    std::vector<float> Rh, lh;
    host_real_dft_tables(n[d], h[d], Rh, lh);
    // pageable source: the runtime stages the bytes before returning, so the vectors may go
    if (cudaMemcpyAsync(R[d], Rh.data(), Rh.size() * sizeof(float), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(lam[d], lh.data(), lh.size() * sizeof(float), cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
      return nerr(LDDMM_ERR_CUDA, "table upload failed");
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
