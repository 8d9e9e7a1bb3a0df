// C ABI of the denoiser's building blocks: the tensor-core 3x3x3 convolutions.
#include <cstdio>
#include <cstring>

#include "nm_internal.cuh"

using namespace nm;

namespace {

bool dev_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

nm_status err(nm_status st, const char* msg) {
  set_error_message(msg);
  return st;
}

nm_status cuda_err(cudaError_t e, const char* what) {
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  set_error_message(buf);
  return e == cudaErrorMemoryAllocation ? NM_ERR_OOM : NM_ERR_CUDA;
}

// Reads back a device status word, frees it, and maps flags to a status.
nm_status finish(uint32_t* status, cudaStream_t s, const char* what) {
  uint32_t flags = 0;
  cudaError_t e = cudaMemcpyAsync(&flags, status, 4, cudaMemcpyDeviceToHost, s);
  if (!e) e = cudaStreamSynchronize(s);
  cudaFreeAsync(status, s);
  if (e) return cuda_err(e, what);
  if (flags) return err(NM_ERR_DEVICE, "tensor-core wait timed out");
  return NM_OK;
}

}  // namespace

extern "C" {

int32_t nm_conv3d_kpad(int32_t cin) { return conv_kpad(cin); }

nm_status nm_conv3d_fwd(const nm_conv3d_desc* d, const uint16_t* x0, const uint16_t* x1,
                        const uint16_t* w, const float* bias, uint16_t* y, int32_t relu, void* stream) {
  if (!d || !conv_geom_ok(*d)) return err(NM_ERR_ARG, "nm_conv3d_fwd: bad geometry");
  if (!dev_ptr(x0) || !dev_ptr(w) || !dev_ptr(y) || (d->c1 && !dev_ptr(x1)) || (bias && !dev_ptr(bias)))
    return err(NM_ERR_ARG, "nm_conv3d_fwd: operands must be device pointers");
  if (!aligned16(x0) || !aligned16(w) || !aligned16(y) || (d->c1 && !aligned16(x1)))
    return err(NM_ERR_ARG, "nm_conv3d_fwd: operands must be 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t* status = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&status, 4, s);
  if (!e) e = cudaMemsetAsync(status, 0, 4, s);
  if (!e) e = conv3d_fwd(*d, x0, d->c1 ? x1 : nullptr, w, bias, y, relu, status, s);
  if (e) {
    if (status) cudaFreeAsync(status, s);
    return cuda_err(e, "nm_conv3d_fwd");
  }
  return finish(status, s, "nm_conv3d_fwd");
}

nm_status nm_conv3d_dgrad(const nm_conv3d_desc* d, const uint16_t* dy, const uint16_t* w, uint16_t* dx,
                          void* stream) {
  if (!d || !conv_geom_ok(*d)) return err(NM_ERR_ARG, "nm_conv3d_dgrad: bad geometry");
  nm_conv3d_desc b;
  memset(&b, 0, sizeof b);
  b.n = d->n; b.d = d->d; b.h = d->h; b.w = d->w;
  b.c0 = d->cout; b.c1 = 0; b.src0_coarse = 0; b.cout = d->c0 + d->c1;
  if (!conv_geom_ok(b)) return err(NM_ERR_ARG, "nm_conv3d_dgrad: unsupported input channel count");
  if (!dev_ptr(dy) || !dev_ptr(w) || !dev_ptr(dx)) return err(NM_ERR_ARG, "nm_conv3d_dgrad: operands must be device pointers");
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t* status = nullptr;
  void* wb = nullptr;
  const size_t wb_bytes = (size_t)b.cout * conv_kpad(b.c0) * 2;
  cudaError_t e = cudaMallocAsync((void**)&status, 4, s);
  if (!e) e = cudaMallocAsync(&wb, wb_bytes, s);
  if (!e) e = cudaMemsetAsync(status, 0, 4, s);
  if (!e) e = conv3d_flip_weights(*d, w, wb, s);
  if (!e) e = conv3d_fwd(b, dy, nullptr, wb, nullptr, dx, 0, status, s);
  if (wb) cudaFreeAsync(wb, s);
  if (e) {
    if (status) cudaFreeAsync(status, s);
    return cuda_err(e, "nm_conv3d_dgrad");
  }
  return finish(status, s, "nm_conv3d_dgrad");
}

nm_status nm_conv3d_wgrad(const nm_conv3d_desc* d, const uint16_t* x0, const uint16_t* x1,
                          const uint16_t* dy, float* dw, float* db, void* stream) {
  if (!d || !conv_geom_ok(*d) || !(d->cout == 16 || d->cout == 32 || d->cout == 64 || d->cout == 128))
    return err(NM_ERR_ARG, "nm_conv3d_wgrad: bad geometry");
  if (!dev_ptr(x0) || !dev_ptr(dy) || !dev_ptr(dw) || (d->c1 && !dev_ptr(x1)) || (db && !dev_ptr(db)))
    return err(NM_ERR_ARG, "nm_conv3d_wgrad: operands must be device pointers");
  cudaStream_t s = (cudaStream_t)stream;
  uint32_t* status = nullptr;
  void* ws = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&status, 4, s);
  if (!e) e = cudaMallocAsync(&ws, conv_wgrad_workspace(*d), s);
  if (!e) e = cudaMemsetAsync(status, 0, 4, s);
  if (!e) e = conv3d_wgrad(*d, x0, d->c1 ? x1 : nullptr, dy, dw, db, ws, status, s);
  if (ws) cudaFreeAsync(ws, s);
  if (e) {
    if (status) cudaFreeAsync(status, s);
    return cuda_err(e, "nm_conv3d_wgrad");
  }
  return finish(status, s, "nm_conv3d_wgrad");
}

}  // extern "C"
