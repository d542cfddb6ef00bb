// Inference of the candidate classifier on the tensor cores (tcgen05, BF16
// operands, FP32 accumulators in tensor memory).
//
// A conv layer z[t][co] = b[co] + sum_{k, ci} w[co][ci][k] x[ci][t + k - 3] is
// a sum over the seven taps k of dense products A_k B_k^T with
// A_k[t][ci] = x[ci][t + k - 3] (M = 128 time samples, K = 32 channels) and
// B_k[co][ci] = w[co][ci][k] (N = 32).  The activations sit in shared memory
// channels-last in the K-major no-swizzle operand layout with rows at a
// uniform 16-byte stride inside each 8-channel chunk (row t of chunk j at
// j * XLBO + (t + 3) * 16; 8-row groups 128 bytes apart), so A_k is the same
// buffer with its start moved by k rows: no im2col copy.  Per 128-sample
// block a layer is 7 taps x 2 K-steps = 14 MMAs into 32 TMEM columns.  The
// epilogue (bias, ReLU, 2:1 max-pool or the global average) reads each time
// sample's 32 outputs from its own TMEM lane and writes the next layer's
// activations (BF16, as the FP32-pipe path rounds them) into the other
// buffer; the head (Linear 32 -> 4, softmax) follows the FP32 path's order.
// One CTA of 128 threads takes samples blockIdx.x, blockIdx.x + gridDim.x, ...
// with the three layers' weights copied once into shared memory.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "cnn_kernels.cuh"
#include "tc_dft.cuh"

namespace pond {
namespace cnn {

constexpr int TC_THREADS = 128;
constexpr int XR = 264;                         // rows per activation chunk: 3 + 256 + 3, rounded up
constexpr int XLBO = XR * 16;                   // bytes between 8-channel chunks
constexpr int XBYTES = 4 * XLBO;                // one activation buffer (32 channels)
constexpr int WTAP = 32 * 32 * 2;               // B_k of one tap: 2 KiB
constexpr int WLAYER = 7 * WTAP;                // 14 KiB per layer
constexpr int WTC_BYTES = 3 * WLAYER;           // device copy of the three layers' operands
constexpr int SM_W = 0, SM_X0 = WTC_BYTES, SM_X1 = SM_X0 + XBYTES, SM_BIAS = SM_X1 + XBYTES;
constexpr int SM_RED = SM_BIAS + 3 * 32 * 4;    // [64][33] FP32 for the global average
constexpr int SM_TAIL = SM_RED + 64 * 33 * 4;
constexpr int TC_SMEM = 128 + SM_TAIL + 64;     // about 86 KiB: two CTAs per SM
constexpr uint32_t TC_TMEM_COLS = 64;           // D of two 128-sample blocks
static_assert(SM_X0 % 128 == 0 && SM_X1 % 128 == 0, "operand buffers on core-matrix boundaries");

// Byte offset of w[co][ci][k] of one layer in the tensor-core operand block:
// tap k's B_k in the K-major layout (core matrix (co/8, ci/8) at co/8 * 512 + ci/8 * 128).
__host__ __device__ constexpr int wtc_offset(int k, int co, int ci) {
  return k * WTAP + (co >> 3) * 512 + (ci >> 3) * 128 + (co & 7) * 16 + (ci & 7) * 2;
}

// BF16 master copy (flat parameter layout) -> the tensor-core operand block.
__global__ void k_cnn_tc_weights(const __nv_bfloat16* __restrict__ wbf, unsigned char* __restrict__ wtc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 3 * CONV) return;
  const int l = i / CONV, r = i % CONV;
  const int co = r / (C * K), ci = (r / K) % C, k = r % K;
  *reinterpret_cast<__nv_bfloat16*>(wtc + l * WLAYER + wtc_offset(k, co, ci)) = wbf[l * LAYER + r];
}

__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// M = 128, N = 32, BF16 A and B (K-major), FP32 accumulator.
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(32 >> 3) << 17) |
                              ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(TC_IDESC), "r"(acc));
}

// D (TMEM columns 32 g) = sum over taps and K-steps of A_k (block g of the
// activations in x) B_k^T (layer l's operands).
__device__ __forceinline__ void tc_layer_mmas(uint32_t tmem, uint32_t x, uint32_t w, int nblk) {
  for (int g = 0; g < nblk; ++g) {
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const uint64_t a = tc_desc(x + 2 * s * XLBO + (uint32_t)(128 * g + k) * 16, XLBO, 128);
        const uint64_t b = tc_desc(w + k * WTAP + s * 256, 128, 512);
        tc_mma(tmem + 32 * g, a, b, acc);
        acc = 1;
      }
    }
  }
}

// Wait for the layer's MMAs (bounded); false when the wait gave up.
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t& phase, int* fail, int* err) {
  bool ok = true;
  if (!*fail && !tc::mbar_wait(bar, phase)) {
    *fail = 1;
    if (err) atomicExch(err, 1);
    ok = false;
  }
  phase ^= 1u;
  tc::fence_after_sync();
  return ok;
}

__device__ __forceinline__ void tc_load32(uint32_t taddr, float* v) { tc::tmem_load32(taddr, v); }

// Row t (0 .. T/2 - 1 after pooling) of an activation buffer: 32 BF16 values in four 16-byte chunks.
__device__ __forceinline__ void store_row(unsigned char* xb, int row, const float* v) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    uint32_t p[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(v[8 * j + 2 * q], v[8 * j + 2 * q + 1]);
      p[q] = *reinterpret_cast<const uint32_t*>(&h);
    }
    *reinterpret_cast<uint4*>(xb + j * XLBO + (row + PAD) * 16) = make_uint4(p[0], p[1], p[2], p[3]);
  }
}

__global__ void __launch_bounds__(TC_THREADS) k_cnn_infer_tc(const __nv_bfloat16* __restrict__ x, int B,
                                                             const unsigned char* __restrict__ wtc,
                                                             const float* __restrict__ theta,
                                                             const __nv_bfloat16* __restrict__ wbf,
                                                             float* __restrict__ prob, int* __restrict__ err) {
  extern __shared__ unsigned char dsm[];
  unsigned char* sm = tc::align128(dsm);
  unsigned char* x0 = sm + SM_X0;
  unsigned char* x1 = sm + SM_X1;
  float* bias = reinterpret_cast<float*>(sm + SM_BIAS);
  float* red = reinterpret_cast<float*>(sm + SM_RED);
  unsigned char* tail = sm + SM_TAIL;
  const uint32_t bar = tc::smem_addr(tail);
  uint32_t* slot = reinterpret_cast<uint32_t*>(tail + 8);
  int* fail = reinterpret_cast<int*>(tail + 16);
  __shared__ float gsm[C];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < WTC_BYTES / 16; i += TC_THREADS)
    reinterpret_cast<uint4*>(sm + SM_W)[i] = __ldg(reinterpret_cast<const uint4*>(wtc) + i);
  for (int i = tid; i < 2 * XBYTES / 16; i += TC_THREADS) reinterpret_cast<uint4*>(x0)[i] = make_uint4(0, 0, 0, 0);
  for (int i = tid; i < 3 * C; i += TC_THREADS) bias[i] = theta[(i / C) * LAYER + CONV + i % C];
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(slot), TC_TMEM_COLS);
  if (tid == 0) {
    tc::mbar_init(bar, 1);
    *fail = 0;
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *slot;
  const uint32_t lane_addr = tmem + ((uint32_t)(32 * warp) << 16);
  const uint32_t w_s = tc::smem_addr(sm + SM_W), x0_s = tc::smem_addr(x0), x1_s = tc::smem_addr(x1);
  uint32_t phase = 0;
  for (int b = blockIdx.x; b < B; b += gridDim.x) {
    {  // the patch [32 ch][256 t] -> channels-last rows of buffer 0: thread = (8-sample run o, chunk j)
      const int o = tid & 31, j = tid >> 5;
      const uint4* src = reinterpret_cast<const uint4*>(x + (size_t)b * C * T0);
      uint32_t r[8][4];   // r[c][i]: samples 2i, 2i + 1 of channel 8 j + c
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const uint4 u = __ldg(src + (8 * j + c) * (T0 / 8) + o);
        r[c][0] = u.x;
        r[c][1] = u.y;
        r[c][2] = u.z;
        r[c][3] = u.w;
      }
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        // channels 2q, 2q + 1 of sample t: the low (t even) or high halves of word t / 2
        const uint32_t sel = (t & 1) ? 0x7632u : 0x5410u;
        uint32_t p[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) p[q] = __byte_perm(r[2 * q][t >> 1], r[2 * q + 1][t >> 1], sel);
        *reinterpret_cast<uint4*>(x0 + j * XLBO + (8 * o + t + PAD) * 16) = make_uint4(p[0], p[1], p[2], p[3]);
      }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    // layer 1: 256 samples (two blocks), pooled into buffer 1
    if (tid == 0 && !*fail) {
      tc::fence_after_sync();
      tc_layer_mmas(tmem, x0_s, w_s, 2);
      tc::mma_commit(bar);
    }
    tc_wait(bar, phase, fail, err);
#pragma unroll 1
    for (int g = 0; g < 2; ++g) {
      float v[32];
      tc_load32(lane_addr + 32 * g, v);
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const float a = fmaxf(v[c] + bias[c], 0.f);
        v[c] = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, 1));
      }
      if ((lane & 1) == 0) store_row(x1, (128 * g + 32 * warp + lane) >> 1, v);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    // layer 2: 128 samples, pooled into buffer 0 (rows 64 .. 66 cleared: the input's rows are still there)
    if (tid == 0 && !*fail) {
      tc::fence_after_sync();
      tc_layer_mmas(tmem, x1_s, w_s + WLAYER, 1);
      tc::mma_commit(bar);
    }
    tc_wait(bar, phase, fail, err);
    {
      float v[32];
      tc_load32(lane_addr, v);
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const float a = fmaxf(v[c] + bias[C + c], 0.f);
        v[c] = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, 1));
      }
      if ((lane & 1) == 0) store_row(x0, (32 * warp + lane) >> 1, v);
      if (tid < 12)   // chunk tid % 4, row 64 + PAD + tid / 4
        *reinterpret_cast<uint4*>(x0 + (tid & 3) * XLBO + (64 + PAD + tid / 4) * 16) = make_uint4(0, 0, 0, 0);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    // layer 3: 64 samples (rows 64 .. 127 of the block are not used), global average
    if (tid == 0 && !*fail) {
      tc::fence_after_sync();
      tc_layer_mmas(tmem, x0_s, w_s + 2 * WLAYER, 1);
      tc::mma_commit(bar);
    }
    tc_wait(bar, phase, fail, err);
    {
      float v[32];
      tc_load32(lane_addr, v);
      if (warp < 2) {
        const int t = 32 * warp + lane;
#pragma unroll
        for (int c = 0; c < 32; ++c) red[t * 33 + c] = fmaxf(v[c] + bias[2 * C + c], 0.f);
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (tid < C) {
      float s = 0.f;
      for (int t = 0; t < 64; ++t) s += red[t * 33 + tid];
      gsm[tid] = s / 64.f;
    }
    __syncthreads();
    if (tid < NCLS) {
      // logits and softmax in the FP32-pipe head's order
      float lg[NCLS], mx = -INFINITY;
#pragma unroll
      for (int j = 0; j < NCLS; ++j) {
        float s = theta[FC_OFF + NCLS * C + j];
        for (int c = 0; c < C; ++c) s = fmaf(bf(wbf[FC_OFF + j * C + c]), gsm[c], s);
        lg[j] = s;
        mx = fmaxf(mx, s);
      }
      float den = 0.f;
#pragma unroll
      for (int j = 0; j < NCLS; ++j) {
        lg[j] = expf(lg[j] - mx);
        den += lg[j];
      }
      const float pj = *fail ? __int_as_float(0x7fc00000) : lg[tid] / den;
      prob[(size_t)b * NCLS + tid] = pj;
    }
    __syncthreads();   // gsm and red are rewritten by the next sample
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, TC_TMEM_COLS);
  }
}

}  // namespace cnn
}  // namespace pond
