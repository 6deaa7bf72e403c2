// C ABI of the warm-start network kernels (kernels_net.cu): thin argument checks, then launches.
// All pointers are device pointers; work is enqueued on `stream` (NULL = legacy default stream).
#include "../../include/lddmm.h"
#include "kernels.h"

namespace lddmm {
cudaError_t net_conv_fwd(const float* x, const void* w, const float* bias, float* y, int B, int Ci,
                         int Co, int n, int ks, int relu, int accumulate, cudaStream_t s);
cudaError_t net_conv_dgrad(const float* dy, const void* w, void* wT_scratch, float* dx, int B,
                           int Ci, int Co, int n, int ks, cudaStream_t s);
cudaError_t net_conv_wgrad(const float* x, const float* dy, float* dw, float* db, float* scratch,
                           int B, int Ci, int Co, int n, int ks, cudaStream_t s);
int64_t net_conv_wgrad_scratch(int B, int Ci, int Co, int n, int ks);
cudaError_t net_relu_bwd(float* dy, const float* y, int64_t count, cudaStream_t s);
cudaError_t net_pool_fwd(const float* x, float* y, int64_t BC, int n, cudaStream_t s);
cudaError_t net_pool_bwd(const float* dy, float* dx, int64_t BC, int n, cudaStream_t s);
cudaError_t net_up_fwd(const float* x, float* y, int B, int C, int m, int Cy, int coff,
                       cudaStream_t s);
cudaError_t net_up_bwd(const float* dy, float* dx, int B, int C, int m, int Cy, int coff,
                       cudaStream_t s);
cudaError_t net_copy_ch(const float* src, float* dst, int B, int C, int64_t nv, int Cs, int soff,
                        int Cd, int doff, int accumulate, cudaStream_t s);
cudaError_t net_mse(const float* p, const float* t, float* g, int64_t count, double* loss,
                    cudaStream_t s);
cudaError_t net_adam(float* w, const float* g, float* m, float* v, void* wb, int64_t count,
                     float lr, float b1, float b2, float eps, int step, cudaStream_t s);
cudaError_t net_cast_bf16(const float* a, void* b, int64_t count, cudaStream_t s);
}  // namespace lddmm

using namespace lddmm;

static int ret(cudaError_t e) { return e == cudaSuccess ? LDDMM_OK : LDDMM_ERR_CUDA; }
static bool shape_ok(int B, int Ci, int Co, int n, int ks) {
  return B > 0 && Ci > 0 && Co > 0 && n > 0 && (ks == 1 || ks == 3) &&
         (long long)B * (Ci > Co ? Ci : Co) * n * n * n < (1LL << 40);
}

extern "C" {

int lddmm_net_conv3d_fwd(const float* x, const void* w_bf16, const float* bias, float* y, int B,
                         int Ci, int Co, int n, int ksize, int relu, int accumulate, void* stream) {
  if (!x || !w_bf16 || !y || !shape_ok(B, Ci, Co, n, ksize)) return LDDMM_ERR_INVALID_ARG;
  return ret(net_conv_fwd(x, w_bf16, bias, y, B, Ci, Co, n, ksize, relu, accumulate,
                          (cudaStream_t)stream));
}

int lddmm_net_conv3d_dgrad(const float* dy, const void* w_bf16, void* wT_scratch, float* dx, int B,
                           int Ci, int Co, int n, int ksize, void* stream) {
  if (!dy || !w_bf16 || !wT_scratch || !dx || !shape_ok(B, Ci, Co, n, ksize))
    return LDDMM_ERR_INVALID_ARG;
  return ret(net_conv_dgrad(dy, w_bf16, wT_scratch, dx, B, Ci, Co, n, ksize, (cudaStream_t)stream));
}

int64_t lddmm_net_conv3d_wgrad_scratch(int B, int Ci, int Co, int n, int ksize) {
  if (!shape_ok(B, Ci, Co, n, ksize)) return LDDMM_ERR_INVALID_ARG;
  return net_conv_wgrad_scratch(B, Ci, Co, n, ksize);
}

int lddmm_net_conv3d_wgrad(const float* x, const float* dy, float* dw, float* db, float* scratch,
                           int64_t scratch_floats, int B, int Ci, int Co, int n, int ksize,
                           void* stream) {
  if (!x || !dy || !dw || !scratch || !shape_ok(B, Ci, Co, n, ksize)) return LDDMM_ERR_INVALID_ARG;
  if (scratch_floats < net_conv_wgrad_scratch(B, Ci, Co, n, ksize)) return LDDMM_ERR_INVALID_ARG;
  return ret(net_conv_wgrad(x, dy, dw, db, scratch, B, Ci, Co, n, ksize, (cudaStream_t)stream));
}

int lddmm_net_relu_bwd(float* dy, const float* y, int64_t count, void* stream) {
  if (!dy || !y || count < 0) return LDDMM_ERR_INVALID_ARG;
  return ret(net_relu_bwd(dy, y, count, (cudaStream_t)stream));
}

int lddmm_net_pool2(const float* src, float* dst, int64_t BC, int n, int backward, void* stream) {
  if (!src || !dst || BC <= 0 || n < 2 || n % 2) return LDDMM_ERR_INVALID_ARG;
  return ret(backward ? net_pool_bwd(src, dst, BC, n, (cudaStream_t)stream)
                      : net_pool_fwd(src, dst, BC, n, (cudaStream_t)stream));
}

int lddmm_net_up2(const float* src, float* dst, int B, int C, int m, int Cy, int coff, int backward,
                  void* stream) {
  if (!src || !dst || B <= 0 || C <= 0 || m <= 0 || coff < 0 || coff + C > Cy)
    return LDDMM_ERR_INVALID_ARG;
  return ret(backward ? net_up_bwd(src, dst, B, C, m, Cy, coff, (cudaStream_t)stream)
                      : net_up_fwd(src, dst, B, C, m, Cy, coff, (cudaStream_t)stream));
}

int lddmm_net_copy_channels(const float* src, float* dst, int B, int C, int64_t nv, int Cs,
                            int soff, int Cd, int doff, int accumulate, void* stream) {
  if (!src || !dst || B <= 0 || C <= 0 || nv <= 0 || soff + C > Cs || doff + C > Cd)
    return LDDMM_ERR_INVALID_ARG;
  return ret(net_copy_ch(src, dst, B, C, nv, Cs, soff, Cd, doff, accumulate, (cudaStream_t)stream));
}

int lddmm_net_mse(const float* pred, const float* target, float* grad, int64_t count,
                  double* loss_dev, void* stream) {
  if (!pred || !target || !loss_dev || count <= 0) return LDDMM_ERR_INVALID_ARG;
  return ret(net_mse(pred, target, grad, count, loss_dev, (cudaStream_t)stream));
}

int lddmm_net_adam(float* w, const float* g, float* m, float* v, void* w_bf16, int64_t count,
                   float lr, float beta1, float beta2, float eps, int step, void* stream) {
  if (!w || !g || !m || !v || count <= 0 || step < 1) return LDDMM_ERR_INVALID_ARG;
  return ret(net_adam(w, g, m, v, w_bf16, count, lr, beta1, beta2, eps, step, (cudaStream_t)stream));
}

int lddmm_net_cast_bf16(const float* a, void* b, int64_t count, void* stream) {
  if (!a || !b || count <= 0) return LDDMM_ERR_INVALID_ARG;
  return ret(net_cast_bf16(a, b, count, (cudaStream_t)stream));
}

}  // extern "C"
