// Single-pulse candidate classifier: training and inference on the GPU.
//
// The paper plans automatic detection of transients (Sec. 5) without naming a
// method.  The classifier here takes a patch of 32 DM trials x 256 series
// samples around a candidate and runs
//   3 x [Conv1d(32 -> 32, kernel 7, zero padding 3) + ReLU],
//   2:1 max-pool after the first two blocks, global average over time,
//   Linear(32 -> 4) and softmax (classes: dispersed pulse, broadband RFI,
//   narrowband RFI, noise),
// with BF16 weights and activations, FP32 accumulation, FP32 master weights
// and Adam.  Training minimises the mean cross-entropy of a batch.  Training's
// forward and backward passes run on the FP32 pipes (they keep the layers'
// pre-activations for the backward pass); inference (pond_cnn_forward) runs
// the three convolutions as implicit GEMMs on the tensor cores (cnn_tc.cuh).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "../../include/pond.h"
#include "cnn_kernels.cuh"
#include "cnn_tc.cuh"
#include "pond_internal.h"

using namespace pond::cnn;

struct pond_cnn_s {
  int device = 0;
  int max_batch = 0;
  long long step = 0;
  float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
  __nv_bfloat16* wbf = nullptr;
  float *z1 = nullptr, *z2 = nullptr, *z3 = nullptr;
  __nv_bfloat16 *h1 = nullptr, *h2 = nullptr;
  uint8_t *a1 = nullptr, *a2 = nullptr;
  float *gap = nullptr, *prob = nullptr, *loss = nullptr, *dg = nullptr, *lmean = nullptr;
  float *dz3 = nullptr, *dz2 = nullptr, *dz1 = nullptr, *part = nullptr;
  unsigned char* wtc = nullptr;   // the conv weights in the tensor-core operand layout
  int* tc_err = nullptr;          // set when a tensor-core MMA wait gave up
  int sms = 0;
};

namespace {

int cuda_fail(cudaError_t e, const char* what) {
  return pond::set_error(e == cudaErrorMemoryAllocation ? POND_E_OOM : POND_E_CUDA,
                         (std::string(what) + ": " + cudaGetErrorString(e)).c_str());
}

#define CKC(call)                                 \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

template <int T, int MODE>
size_t fwd_smem() { return (size_t)(C * (T + 2 * PAD) + CONV) * sizeof(float); }
template <int T>
size_t wgt_smem() { return (size_t)(C * T + C * (T + 2 * PAD)) * sizeof(float); }

cudaError_t set_attrs() {
  cudaError_t e = cudaFuncSetAttribute(k_conv_fwd<256, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fwd_smem<256, 0>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_conv_bwd_weight<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wgt_smem<256>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_conv_fwd<128, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)fwd_smem<128, 0>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_conv_fwd<64, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem<64, 1>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_conv_bwd_data<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)fwd_smem<128, 0>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_conv_bwd_data<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem<64, 0>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cnn_infer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
  return e;
}

// Refresh the tensor-core copy of the conv weights from the BF16 master copy.
cudaError_t refresh_wtc(pond_cnn_t n, cudaStream_t st) {
  k_cnn_tc_weights<<<(3 * CONV + 255) / 256, 256, 0, st>>>(n->wbf, n->wtc);
  return cudaGetLastError();
}

void free_net(pond_cnn_t n) {
  for (void* p : {(void*)n->theta, (void*)n->m, (void*)n->v, (void*)n->grad, (void*)n->wbf, (void*)n->z1,
                  (void*)n->z2, (void*)n->z3, (void*)n->h1, (void*)n->h2, (void*)n->a1, (void*)n->a2,
                  (void*)n->gap, (void*)n->prob, (void*)n->loss, (void*)n->dg, (void*)n->lmean, (void*)n->dz3,
                  (void*)n->dz2, (void*)n->dz1, (void*)n->part, (void*)n->wtc, (void*)n->tc_err})
    cudaFree(p);
  delete n;
}

// Adam state reset and BF16 copy of the master weights, from host parameters.
int load_params(pond_cnn_t n, const float* params) {
  CKC(cudaMemcpy(n->theta, params, NPARAM * sizeof(float), cudaMemcpyHostToDevice));
  CKC(cudaMemset(n->m, 0, NPARAM * sizeof(float)));
  CKC(cudaMemset(n->v, 0, NPARAM * sizeof(float)));
  CKC(cudaMemset(n->grad, 0, NPARAM * sizeof(float)));
  // lr = 0 makes the update an identity that refreshes the BF16 copy
  k_adam<<<(NPARAM + 255) / 256, 256>>>(n->theta, n->m, n->v, n->grad, n->wbf, 0.f, 1.f, 1.f, 0.9f, 0.999f, 1e-8f);
  CKC(cudaGetLastError());
  CKC(cudaMemset(n->m, 0, NPARAM * sizeof(float)));
  CKC(cudaMemset(n->v, 0, NPARAM * sizeof(float)));
  CKC(refresh_wtc(n, 0));
  CKC(cudaDeviceSynchronize());
  n->step = 0;
  return POND_OK;
}

__global__ void k_mean(const float* __restrict__ x, int n, float* __restrict__ out) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < n; ++i) s += x[i];
    *out = s / (float)n;
  }
}

int forward(pond_cnn_t n, const __nv_bfloat16* x, int B, const int32_t* labels, cudaStream_t st) {
  const __nv_bfloat16* w = n->wbf;
  k_conv_fwd<256, 0><<<B, THREADS, fwd_smem<256, 0>(), st>>>(x, w, n->theta + CONV, n->z1, n->h1, n->a1, nullptr);
  k_conv_fwd<128, 0><<<B, THREADS, fwd_smem<128, 0>(), st>>>(n->h1, w + LAYER, n->theta + LAYER + CONV, n->z2,
                                                             n->h2, n->a2, nullptr);
  k_conv_fwd<64, 1><<<B, THREADS, fwd_smem<64, 1>(), st>>>(n->h2, w + 2 * LAYER, n->theta + 2 * LAYER + CONV,
                                                           n->z3, nullptr, nullptr, n->gap);
  k_head<<<(B + 127) / 128, 128, 0, st>>>(n->gap, w + FC_OFF, n->theta + FC_OFF + NCLS * C, labels, B, n->prob,
                                          n->loss, n->dg, n->part);
  CKC(cudaGetLastError());
  return POND_OK;
}

int backward(pond_cnn_t n, const __nv_bfloat16* x, int B, cudaStream_t st) {
  const __nv_bfloat16* w = n->wbf;
  const long long n3 = (long long)B * C * 64;
  k_gap_bwd<<<(unsigned)((n3 + 255) / 256), 256, 0, st>>>(n->dg, n->z3, B, 64, n->dz3);
  k_conv_bwd_weight<64><<<B, THREADS, wgt_smem<64>(), st>>>(n->dz3, n->h2, n->part, 2 * LAYER);
  k_conv_bwd_data<64><<<B, THREADS, fwd_smem<64, 0>(), st>>>(n->dz3, w + 2 * LAYER, n->a2, n->z2, n->dz2);
  k_conv_bwd_weight<128><<<B, THREADS, wgt_smem<128>(), st>>>(n->dz2, n->h1, n->part, LAYER);
  k_conv_bwd_data<128><<<B, THREADS, fwd_smem<128, 0>(), st>>>(n->dz2, w + LAYER, n->a1, n->z1, n->dz1);
  k_conv_bwd_weight<256><<<B, THREADS, wgt_smem<256>(), st>>>(n->dz1, x, n->part, 0);
  k_reduce<<<(NPARAM + 255) / 256, 256, 0, st>>>(n->part, B, n->grad);
  k_mean<<<1, 32, 0, st>>>(n->loss, B, n->lmean);
  CKC(cudaGetLastError());
  return POND_OK;
}

int check_batch(pond_cnn_t n, const void* x, int B) {
  if (!n || !x || B < 1) return pond::set_error(POND_E_ARG, "cnn: null argument or empty batch");
  if (B > n->max_batch) return pond::set_error(POND_E_ARG, "cnn: batch larger than max_batch");
  return POND_OK;
}

}  // namespace

int pond::cnn_max_batch(pond_cnn_t n) { return n ? n->max_batch : 0; }

extern "C" {

int pond_cnn_create(pond_cnn_t* out, const float* init_params, int32_t max_batch, int32_t device) {
  if (!out || !init_params || max_batch < 1) return pond::set_error(POND_E_ARG, "pond_cnn_create: bad argument");
  *out = nullptr;
  pond_cnn_t n = new pond_cnn_s();
  n->device = device;
  n->max_batch = max_batch;
  const size_t B = (size_t)max_batch;
  cudaError_t e = cudaSetDevice(device);
  auto A = [&](auto** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc((void**)p, bytes);
  };
  A(&n->theta, NPARAM * 4);
  A(&n->m, NPARAM * 4);
  A(&n->v, NPARAM * 4);
  A(&n->grad, NPARAM * 4);
  A(&n->wbf, NPARAM * 2);
  A(&n->z1, B * C * 256 * 4);
  A(&n->z2, B * C * 128 * 4);
  A(&n->z3, B * C * 64 * 4);
  A(&n->h1, B * C * 128 * 2);
  A(&n->h2, B * C * 64 * 2);
  A(&n->a1, B * C * 128);
  A(&n->a2, B * C * 64);
  A(&n->gap, B * C * 4);
  A(&n->prob, B * NCLS * 4);
  A(&n->loss, B * 4);
  A(&n->dg, B * C * 4);
  A(&n->lmean, 4);
  A(&n->dz3, B * C * 64 * 4);
  A(&n->dz2, B * C * 128 * 4);
  A(&n->dz1, B * C * 256 * 4);
  A(&n->part, B * NPARAM * 4);
  A(&n->wtc, WTC_BYTES);
  A(&n->tc_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(n->tc_err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n->sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = set_attrs();
  if (e != cudaSuccess) {
    free_net(n);
    return cuda_fail(e, "pond_cnn_create");
  }
  const int rc = load_params(n, init_params);
  if (rc) {
    free_net(n);
    return rc;
  }
  *out = n;
  return POND_OK;
}

int pond_cnn_set_params(pond_cnn_t n, const float* params) {
  if (!n || !params) return pond::set_error(POND_E_ARG, "pond_cnn_set_params: null argument");
  CKC(cudaSetDevice(n->device));
  return load_params(n, params);
}

int pond_cnn_params(pond_cnn_t n, float* out) {
  if (!n || !out) return pond::set_error(POND_E_ARG, "pond_cnn_params: null argument");
  CKC(cudaSetDevice(n->device));
  CKC(cudaDeviceSynchronize());
  CKC(cudaMemcpy(out, n->theta, NPARAM * sizeof(float), cudaMemcpyDeviceToHost));
  int te = 0;
  CKC(cudaMemcpy(&te, n->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (te) {
    CKC(cudaMemset(n->tc_err, 0, sizeof(int)));
    return pond::set_error(POND_E_TIMEOUT, "a tensor-core MMA wait of the inference kernel expired");
  }
  return POND_OK;
}

int pond_cnn_forward(pond_cnn_t n, const void* d_x, int32_t batch, float* d_prob, void* stream) {
  int rc = check_batch(n, d_x, batch);
  if (rc) return rc;
  if (!d_prob) return pond::set_error(POND_E_ARG, "pond_cnn_forward: null output");
  CKC(cudaSetDevice(n->device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if ((uintptr_t)d_x % 16 == 0) {
    // the tensor-core inference kernel: each CTA runs samples blockIdx.x, + gridDim.x, ...
    const int grid = std::min(batch, 2 * n->sms);
    k_cnn_infer_tc<<<grid, TC_THREADS, TC_SMEM, st>>>(static_cast<const __nv_bfloat16*>(d_x), batch, n->wtc,
                                                      n->theta, n->wbf, d_prob, n->tc_err);
    CKC(cudaGetLastError());
    return POND_OK;
  }
  // patches not 16-byte aligned: the FP32-pipe forward
  rc = forward(n, static_cast<const __nv_bfloat16*>(d_x), batch, nullptr, st);
  if (rc) return rc;
  CKC(cudaMemcpyAsync(d_prob, n->prob, (size_t)batch * NCLS * sizeof(float), cudaMemcpyDeviceToDevice, st));
  return POND_OK;
}

int pond_cnn_gradient(pond_cnn_t n, const void* d_x, const int32_t* d_labels, int32_t batch, float* grad_out,
                      float* loss_out, void* stream) {
  int rc = check_batch(n, d_x, batch);
  if (rc) return rc;
  if (!d_labels) return pond::set_error(POND_E_ARG, "pond_cnn_gradient: null labels");
  CKC(cudaSetDevice(n->device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const __nv_bfloat16* x = static_cast<const __nv_bfloat16*>(d_x);
  if ((rc = forward(n, x, batch, d_labels, st))) return rc;
  if ((rc = backward(n, x, batch, st))) return rc;
  if (grad_out) CKC(cudaMemcpyAsync(grad_out, n->grad, NPARAM * sizeof(float), cudaMemcpyDeviceToHost, st));
  if (loss_out) CKC(cudaMemcpyAsync(loss_out, n->lmean, sizeof(float), cudaMemcpyDeviceToHost, st));
  CKC(cudaStreamSynchronize(st));
  return POND_OK;
}

int pond_cnn_train_step(pond_cnn_t n, const void* d_x, const int32_t* d_labels, int32_t batch, float lr,
                        float* loss_out, void* stream) {
  int rc = check_batch(n, d_x, batch);
  if (rc) return rc;
  if (!d_labels || !(lr >= 0)) return pond::set_error(POND_E_ARG, "pond_cnn_train_step: bad argument");
  CKC(cudaSetDevice(n->device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const __nv_bfloat16* x = static_cast<const __nv_bfloat16*>(d_x);
  if ((rc = forward(n, x, batch, d_labels, st))) return rc;
  if ((rc = backward(n, x, batch, st))) return rc;
  n->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - (float)std::pow((double)b1, (double)n->step);
  const float c2 = 1.f - (float)std::pow((double)b2, (double)n->step);
  k_adam<<<(NPARAM + 255) / 256, 256, 0, st>>>(n->theta, n->m, n->v, n->grad, n->wbf, lr, c1, c2, b1, b2, 1e-8f);
  CKC(cudaGetLastError());
  CKC(refresh_wtc(n, st));
  if (loss_out) {
    CKC(cudaMemcpyAsync(loss_out, n->lmean, sizeof(float), cudaMemcpyDeviceToHost, st));
    CKC(cudaStreamSynchronize(st));
  }
  return POND_OK;
}

int pond_cnn_destroy(pond_cnn_t n) {
  if (!n) return POND_OK;
  cudaSetDevice(n->device);
  cudaDeviceSynchronize();
  free_net(n);
  return POND_OK;
}

int pond_patches(const float* d_series, int32_t ndm, int64_t n, int64_t stride, const int32_t* d_corners,
                 int32_t npatch, void* d_out, void* stream) {
  if (npatch < 0 || ndm < 1 || n < 1 || stride < n || (npatch > 0 && (!d_series || !d_corners || !d_out)))
    return pond::set_error(POND_E_ARG, "pond_patches: bad argument");
  if (npatch == 0) return POND_OK;
  k_patches<<<npatch, THREADS, 0, static_cast<cudaStream_t>(stream)>>>(d_series, ndm, n, stride, d_corners,
                                                                       static_cast<__nv_bfloat16*>(d_out));
  CKC(cudaGetLastError());
  return POND_OK;
}

}  // extern "C"
