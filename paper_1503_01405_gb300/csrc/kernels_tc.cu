// Tensor-core instantiations of the four FFT passes (split-BF16 radix-16
// stages, tc_dft.cuh) and the host-built W16 operand parts.
#include <cmath>
#include <cstring>

#include "passes.cuh"

namespace pond {

cudaError_t set_kernel_attributes_tc() { return set_attributes_t<true>(); }

cudaError_t launch_fwd_cols_tc(const Geom& g, SegIn in, float2* out, const float2* tw, cudaStream_t st) {
  return launch_fwd_cols_t<true>(g, in, out, tw, st);
}

cudaError_t launch_fwd_rows_tc(const Geom& g, const float2* in, float2* out, const float2* tw3L, Tw2 tw2L, const float2* tw,
                               cudaStream_t st) {
  return launch_fwd_rows_t<true>(g, in, out, tw3L, tw2L, tw, st);
}

cudaError_t launch_inv_cols_tc(const Geom& g, const float2* in, float2* out, const ChirpAnchor* anc,
                               int clog, const float2* tw, cudaStream_t st) {
  return launch_inv_cols_t<true>(g, in, out, anc, clog, tw, st);
}

cudaError_t launch_inv_rows_tc(const Geom& g, const float2* buf, float* P, float2* vout, long long vstride,
                               long long vofs, int m_lo, int m_hi, const float2* tw3M, const float2* tw,
                               cudaStream_t st) {
  return launch_inv_rows_t<true>(g, buf, P, vout, vstride, vofs, m_lo, m_hi, tw3M, tw, st);
}

// One CTA waits, with the tensor-core stages' bounded wait, on a barrier that
// no thread or MMA ever arrives on: the wait must give up after limit_ns.
__global__ void k_wait_probe(unsigned long long limit_ns, int* status, unsigned long long* waited) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) tc::mbar_init(tc::smem_addr(&bar), 1);
  __syncthreads();
  const unsigned long long t0 = tc::globaltimer_ns();
  const bool done = tc::mbar_wait(tc::smem_addr(&bar), 0, limit_ns);
  const unsigned long long t1 = tc::globaltimer_ns();
  if (threadIdx.x == 0) {
    *status = done ? 0 : 1;
    *waited = t1 - t0;
  }
}

cudaError_t launch_wait_probe(unsigned long long limit_ns, int* status, unsigned long long* waited) {
  k_wait_probe<<<1, 32>>>(limit_ns, status, waited);
  return cudaGetLastError();
}

namespace {

// Round to the nearest BF16 (ties to even) through FP32.
uint16_t bf16_bits(double x) {
  const float f = (float)x;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

double bf16_value(uint16_t h) {
  const uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return (double)f;
}

}  // namespace

// Real block form of the 16-point DFT with w = exp(sigma 2 pi i / 16):
// X_c = sum_j x_j w^{jc}; with theta = 2 pi (jc mod 16) / 16,
// Re X_c = sum_j (Re x_j cos theta - sigma Im x_j sin theta) and
// Im X_c = sum_j (sigma Re x_j sin theta + Im x_j cos theta).  B[n][k] (row n =
// output real index, k = input real index) is split into hi + mid + lo BF16
// parts, each stored in the K-major operand layout of tc_dft.cuh.
void build_w16_parts(uint16_t* out) {
  const double two_pi = 6.283185307179586476925286766559;
  for (int dir = 0; dir < 2; ++dir) {
    const double sigma = dir == 0 ? -1.0 : 1.0;
    uint16_t* base = out + dir * 3 * 1024;
    for (int n = 0; n < 32; ++n)
      for (int k = 0; k < 32; ++k) {
        const int c = n & 15, j = k & 15;
        const double th = two_pi * (double)((j * c) & 15) / 16.0;
        double b;
        if (n < 16) b = k < 16 ? std::cos(th) : -sigma * std::sin(th);
        else b = k < 16 ? sigma * std::sin(th) : std::cos(th);
        const int off = ((n >> 3) * 512 + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2) / 2;
        double r = b;
        for (int p = 0; p < 3; ++p) {
          const uint16_t h = bf16_bits(r);
          base[p * 1024 + off] = h;
          r -= bf16_value(h);
        }
      }
  }
}

}  // namespace pond
