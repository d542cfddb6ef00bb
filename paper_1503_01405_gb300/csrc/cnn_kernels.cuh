// Kernels of the single-pulse candidate classifier (see cnn.cu for the network).
//
// Layout: activations [B][C][T] (C = 32 DM-trial channels), BF16 in memory
// between layers, FP32 in registers and shared memory; every sum accumulates
// in FP32.  Weight gradients are formed per sample and reduced over the batch
// in sample order, so a training step is deterministic.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace pond {
namespace cnn {

constexpr int C = 32;          // channels
constexpr int K = 7;           // kernel width
constexpr int PAD = 3;
constexpr int T0 = 256;        // samples per patch
constexpr int NCLS = 4;
constexpr int CONV = C * C * K;                       // 7168 weights per conv layer
constexpr int LAYER = CONV + C;                       // weights + biases
constexpr int FC_OFF = 3 * LAYER;                     // 21,600
constexpr int NPARAM = FC_OFF + NCLS * C + NCLS;      // 21,732
constexpr int THREADS = 256;

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

// Forward conv of one sample per CTA: z = b + w * x (zero padded), a = relu(z).
// MODE 0: 2:1 max-pool of a -> out (BF16) and the argmax of each pair; MODE 1:
// global average of a over time -> gap (FP32).  z is kept for the backward pass.
template <int T, int MODE>
__global__ void __launch_bounds__(THREADS) k_conv_fwd(const __nv_bfloat16* __restrict__ x,
                                                      const __nv_bfloat16* __restrict__ w,
                                                      const float* __restrict__ bias, float* __restrict__ z,
                                                      __nv_bfloat16* __restrict__ out, uint8_t* __restrict__ arg,
                                                      float* __restrict__ gap) {
  extern __shared__ float sm[];
  float* xs = sm;                       // [C][T + 2 PAD]
  float* ws = sm + C * (T + 2 * PAD);   // [C][C][K]
  __shared__ float part[C][THREADS / C];
  const int b = blockIdx.x;
  const __nv_bfloat16* xb = x + (size_t)b * C * T;
  for (int i = threadIdx.x; i < C * (T + 2 * PAD); i += THREADS) {
    const int ci = i / (T + 2 * PAD), t = i % (T + 2 * PAD) - PAD;
    xs[i] = (t >= 0 && t < T) ? bf(xb[ci * T + t]) : 0.f;
  }
  for (int i = threadIdx.x; i < CONV; i += THREADS) ws[i] = bf(w[i]);
  __syncthreads();
  constexpr int PARTS = THREADS / C;    // 8 time ranges per output channel
  constexpr int SPAN = T / PARTS;
  const int co = threadIdx.x / PARTS, tp = threadIdx.x % PARTS;
  const int t0 = tp * SPAN;
  float acc[SPAN];
#pragma unroll
  for (int i = 0; i < SPAN; ++i) acc[i] = bias[co];
  for (int ci = 0; ci < C; ++ci) {
    const float* xr = xs + ci * (T + 2 * PAD) + t0;
    const float* wr = ws + (co * C + ci) * K;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float wv = wr[k];
#pragma unroll
      for (int i = 0; i < SPAN; ++i) acc[i] = fmaf(wv, xr[i + k], acc[i]);
    }
  }
  float* zb = z + ((size_t)b * C + co) * T + t0;
#pragma unroll
  for (int i = 0; i < SPAN; ++i) zb[i] = acc[i];
  if constexpr (MODE == 0) {
#pragma unroll
    for (int i = 0; i < SPAN; i += 2) {
      const float a0 = fmaxf(acc[i], 0.f), a1 = fmaxf(acc[i + 1], 0.f);
      const size_t o = ((size_t)b * C + co) * (T / 2) + (t0 + i) / 2;
      out[o] = __float2bfloat16(a1 > a0 ? a1 : a0);
      arg[o] = a1 > a0 ? 1 : 0;
    }
  } else {
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < SPAN; ++i) s += fmaxf(acc[i], 0.f);
    part[co][tp] = s;
    __syncthreads();
    if (tp == 0) {
      float g = 0.f;
#pragma unroll
      for (int q = 0; q < PARTS; ++q) g += part[co][q];
      gap[(size_t)b * C + co] = g / (float)T;
    }
  }
}

// Head of one sample per thread: logits = fc_w g + fc_b, softmax, per-sample
// cross-entropy, d loss / d logits (scaled by 1/B for the batch mean), dg, and
// the fc gradient partials of this sample.
__global__ void k_head(const float* __restrict__ gap, const __nv_bfloat16* __restrict__ fcw,
                       const float* __restrict__ fcb, const int32_t* __restrict__ labels, int B,
                       float* __restrict__ prob, float* __restrict__ loss, float* __restrict__ dg,
                       float* __restrict__ part) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float* g = gap + (size_t)b * C;
  float lg[NCLS], mx = -INFINITY;
#pragma unroll
  for (int j = 0; j < NCLS; ++j) {
    float s = fcb[j];
    for (int c = 0; c < C; ++c) s = fmaf(bf(fcw[j * C + c]), g[c], s);
    lg[j] = s;
    mx = fmaxf(mx, s);
  }
  float den = 0.f;
#pragma unroll
  for (int j = 0; j < NCLS; ++j) {
    lg[j] = expf(lg[j] - mx);
    den += lg[j];
  }
#pragma unroll
  for (int j = 0; j < NCLS; ++j) {
    lg[j] /= den;
    prob[(size_t)b * NCLS + j] = lg[j];
  }
  if (!labels) return;
  const int y = labels[b];
  loss[b] = -logf(fmaxf(lg[y], 1e-30f));
  float dl[NCLS];
#pragma unroll
  for (int j = 0; j < NCLS; ++j) dl[j] = (lg[j] - (j == y ? 1.f : 0.f)) / (float)B;
  float* pb = part + (size_t)b * NPARAM + FC_OFF;
  for (int c = 0; c < C; ++c) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < NCLS; ++j) {
      pb[j * C + c] = dl[j] * g[c];
      s = fmaf(dl[j], bf(fcw[j * C + c]), s);
    }
    dg[(size_t)b * C + c] = s;
  }
#pragma unroll
  for (int j = 0; j < NCLS; ++j) pb[NCLS * C + j] = dl[j];
}

// Backward of the global average: dz3[b][c][t] = (z3 > 0) dg[b][c] / T.
__global__ void k_gap_bwd(const float* __restrict__ dg, const float* __restrict__ z, int B, int T,
                          float* __restrict__ dz) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)B * C * T) return;
  dz[i] = z[i] > 0.f ? dg[i / T] / (float)T : 0.f;
}

// Backward data pass of one sample per CTA for a conv layer of length T:
// dh[ci][t] = sum_{co,k} w[co][ci][k] dz[co][t + PAD - k], then the previous
// layer's max-pool and ReLU are undone: dz_prev[ci][2t + arg] = dh (z_prev > 0).
template <int T>
__global__ void __launch_bounds__(THREADS) k_conv_bwd_data(const float* __restrict__ dz,
                                                           const __nv_bfloat16* __restrict__ w,
                                                           const uint8_t* __restrict__ arg_prev,
                                                           const float* __restrict__ z_prev,
                                                           float* __restrict__ dz_prev) {
  extern __shared__ float sm[];
  float* ds = sm;                        // [C][T + 2 PAD]
  float* ws = sm + C * (T + 2 * PAD);    // [C][C][K]
  const int b = blockIdx.x;
  const float* db = dz + (size_t)b * C * T;
  for (int i = threadIdx.x; i < C * (T + 2 * PAD); i += THREADS) {
    const int co = i / (T + 2 * PAD), t = i % (T + 2 * PAD) - PAD;
    ds[i] = (t >= 0 && t < T) ? db[co * T + t] : 0.f;
  }
  for (int i = threadIdx.x; i < CONV; i += THREADS) ws[i] = bf(w[i]);
  __syncthreads();
  constexpr int PARTS = THREADS / C;
  constexpr int SPAN = T / PARTS;
  const int ci = threadIdx.x / PARTS, tp = threadIdx.x % PARTS;
  const int t0 = tp * SPAN;
  float acc[SPAN];
#pragma unroll
  for (int i = 0; i < SPAN; ++i) acc[i] = 0.f;
  for (int co = 0; co < C; ++co) {
    const float* dr = ds + co * (T + 2 * PAD) + t0;     // dr[i + 2 PAD - k] = dz[co][t0 + i + PAD - k]
    const float* wr = ws + (co * C + ci) * K;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float wv = wr[k];
#pragma unroll
      for (int i = 0; i < SPAN; ++i) acc[i] = fmaf(wv, dr[i + 2 * PAD - k], acc[i]);
    }
  }
  const size_t row = ((size_t)b * C + ci);
#pragma unroll
  for (int i = 0; i < SPAN; ++i) {
    const int t = t0 + i;
    const int a = arg_prev[row * T + t];
    const size_t p = row * (2 * T) + 2 * t;
    dz_prev[p + a] = z_prev[p + a] > 0.f ? acc[i] : 0.f;
    dz_prev[p + 1 - a] = 0.f;
  }
}

// Per-sample weight and bias gradients of a conv layer of length T:
// dW[co][ci][k] = sum_t dz[co][t] x[ci][t + k - PAD], db[co] = sum_t dz[co][t],
// written to this sample's row of the partials at offset `off`.
template <int T>
__global__ void __launch_bounds__(THREADS) k_conv_bwd_weight(const float* __restrict__ dz,
                                                             const __nv_bfloat16* __restrict__ x,
                                                             float* __restrict__ part, int off) {
  extern __shared__ float sm[];
  float* ds = sm;                        // [C][T]
  float* xs = sm + C * T;                // [C][T + 2 PAD]
  const int b = blockIdx.x;
  for (int i = threadIdx.x; i < C * T; i += THREADS) ds[i] = dz[(size_t)b * C * T + i];
  for (int i = threadIdx.x; i < C * (T + 2 * PAD); i += THREADS) {
    const int ci = i / (T + 2 * PAD), t = i % (T + 2 * PAD) - PAD;
    xs[i] = (t >= 0 && t < T) ? bf(x[((size_t)b * C + ci) * T + t]) : 0.f;
  }
  __syncthreads();
  float* pb = part + (size_t)b * NPARAM + off;
  for (int pair = threadIdx.x; pair < C * C; pair += THREADS) {
    const int co = pair / C, ci = pair % C;
    const float* dr = ds + co * T;
    const float* xr = xs + ci * (T + 2 * PAD);
    float acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.f;
    for (int t = 0; t < T; ++t) {
      const float d = dr[t];
#pragma unroll
      for (int k = 0; k < K; ++k) acc[k] = fmaf(d, xr[t + k], acc[k]);
    }
#pragma unroll
    for (int k = 0; k < K; ++k) pb[(co * C + ci) * K + k] = acc[k];
  }
  for (int co = threadIdx.x; co < C; co += THREADS) {
    float s = 0.f;
    for (int t = 0; t < T; ++t) s += ds[co * T + t];
    pb[CONV + co] = s;
  }
}

// grad[p] = sum over samples b (in order) of part[b][p].
__global__ void k_reduce(const float* __restrict__ part, int B, float* __restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NPARAM) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += part[(size_t)b * NPARAM + p];
  grad[p] = s;
}

// Adam (Kingma & Ba 2015) on the FP32 master weights; refreshes the BF16 copy.
__global__ void k_adam(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ grad, __nv_bfloat16* __restrict__ wbf, float lr, float c1,
                       float c2, float beta1, float beta2, float eps) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NPARAM) return;
  const float g = grad[p];
  const float mm = beta1 * m[p] + (1.f - beta1) * g;
  const float vv = beta2 * v[p] + (1.f - beta2) * g * g;
  m[p] = mm;
  v[p] = vv;
  const float th = theta[p] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
  theta[p] = th;
  wbf[p] = __float2bfloat16(th);
}

// Patch p: trials d0..d0+C-1, samples t0..t0+T0-1 of a series block
// [ndm][stride] (samples outside [0, n) repeat the nearest edge sample), less
// its mean and over its standard deviation (1 when that is zero), as BF16.
__global__ void __launch_bounds__(THREADS) k_patches(const float* __restrict__ series, int ndm, long long n,
                                                     long long stride, const int32_t* __restrict__ corner,
                                                     __nv_bfloat16* __restrict__ out) {
  __shared__ float red[THREADS];
  __shared__ float stat[2];
  const int p = blockIdx.x;
  const int d0 = corner[2 * p];
  const long long t0 = corner[2 * p + 1];
  constexpr int NV = C * T0 / THREADS;
  float v[NV];
  float s = 0.f;
#pragma unroll
  for (int u = 0; u < NV; ++u) {
    const int i = threadIdx.x + u * THREADS;
    const int d = min(max(d0 + i / T0, 0), ndm - 1);
    const long long t = min(max(t0 + i % T0, 0ll), n - 1);
    v[u] = series[(size_t)d * stride + t];
    s += v[u];
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = THREADS / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) stat[0] = red[0] / (float)(C * T0);
  __syncthreads();
  const float mean = stat[0];
  s = 0.f;
#pragma unroll
  for (int u = 0; u < NV; ++u) s += (v[u] - mean) * (v[u] - mean);
  __syncthreads();
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = THREADS / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const float sd = sqrtf(red[0] / (float)(C * T0));
    stat[1] = sd > 0.f ? sd : 1.f;
  }
  __syncthreads();
  const float inv = 1.f / stat[1];
#pragma unroll
  for (int u = 0; u < NV; ++u)
    out[(size_t)p * C * T0 + threadIdx.x + u * THREADS] = __float2bfloat16((v[u] - mean) * inv);
}

}  // namespace cnn
}  // namespace pond
