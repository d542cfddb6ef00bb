// pond_probe_fp32_fma: the FP32 arithmetic ceiling of the GPU the engine runs
// on.  The forward and inverse FFT butterflies are FP32 multiply-adds, so at
// the method's algorithmic minimum of DRAM traffic the path is bound by the
// FP32 pipes, not by HBM; this kernel measures that bound on the same device,
// under the same clocks, for the roofline the benchmark reports.
#include <cuda_runtime.h>

#include <cstdio>
#include <string>

#include "../../include/pond.h"
#include "pond_internal.h"

namespace {

constexpr int kThreads = 512;
constexpr int kChains = 8;     // independent FMA chains per thread (covers the FMA latency)
constexpr int kUnroll = 16;    // FMA steps per chain per loop trip

// Each thread runs kChains independent chains a <- a * m + c for
// iters * kUnroll steps and writes the chains' sum, so no step can be dropped.
__global__ void __launch_bounds__(kThreads) k_fma_probe(float* __restrict__ out, int iters, float m, float c) {
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (float)(threadIdx.x + i) * 1e-3f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int i = 0; i < kChains; ++i) a[i] = fmaf(a[i], m, c);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  out[(size_t)blockIdx.x * kThreads + threadIdx.x] = s;
}

}  // namespace

extern "C" int pond_probe_fp32_fma(float* d_out, int32_t blocks, int32_t iters, void* cuda_stream,
                                   double* flops) {
  if (!d_out || !flops || blocks < 1 || iters < 1)
    return pond::set_error(POND_E_ARG, "pond_probe_fp32_fma: need d_out, flops, blocks >= 1, iters >= 1");
  // m slightly below 1 and c small keep every chain finite and normal
  k_fma_probe<<<blocks, kThreads, 0, static_cast<cudaStream_t>(cuda_stream)>>>(d_out, iters, 0.999999f, 1e-6f);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return pond::set_error(POND_E_CUDA, (std::string("pond_probe_fp32_fma: ") + cudaGetErrorString(e)).c_str());
  *flops = 2.0 * blocks * (double)kThreads * iters * kUnroll * kChains;
  return POND_OK;
}
