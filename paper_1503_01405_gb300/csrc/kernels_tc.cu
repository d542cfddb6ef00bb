// Tensor-core instantiations of the four FFT passes (split-BF16 radix-16
// stages, tc_dft.cuh) and the host-built W16 operand parts.
#include <cmath>
#include <cstring>

#include "passes.cuh"
#include "tc_cols.cuh"

namespace pond {

cudaError_t set_kernel_attributes_tc() {
  cudaError_t e = set_attributes_t<true>();
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_inv_cols_det_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, tcc::SMEM_BYTES);
  return e;
}

bool ic_tc_geometry(const Geom& g) { return fused_geometry(g) && g.logR2 == 11 && g.nchan >= 4; }

cudaError_t launch_inv_cols_det_tc(const Geom& g, const float2* in, float* P, float* part, int* cnt, float2* vout,
                                   long long vstride, long long vofs, int m_lo, int m_hi, const uint4* ops, int* err,
                                   cudaStream_t st, int ntr) {
  if (!ic_tc_geometry(g)) return cudaErrorInvalidValue;
  const int nl = 4;
  const dim3 grid((unsigned)((1 << g.logR1) / nl), (unsigned)ntr);
  const float scale = 1.0f / (float)(1u << g.logM);
  const int lognch = g.logR1 - (g.logM - g.logR2);
  const TrialStride ts = ntr > 1 ? TrialStride{g.L, g.M, (long long)fused_groups(g) * g.M, FUSED_J}
                                 : TrialStride{0, 0, 0, 0};
  k_inv_cols_det_tc<<<grid, NT, tcc::SMEM_BYTES, st>>>(in, P, part, cnt, vout, vstride, vofs, lognch, m_lo, m_hi,
                                                       scale, ops, err, ts);
  return cudaGetLastError();
}

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

// Operand block of the tensor-core column pass (tc_cols.cuh): the cosine and
// sine matrices of the 64- and 32-point inverse factors, e^{+2 pi i b p / 64}
// and e^{+2 pi i a q / 32}, rows = output index, K = input index, each split
// into BF16 hi + mid parts in the K-major operand layout, then the twiddle
// tables T0[i] = e^{2 pi i i / 2048} (i < 64) and T1[j] = e^{2 pi i 64 j / 2048}
// (j < 32) as FP32 pairs.  Built in FP64.
void build_ic_tc_ops(unsigned char* out) {
  const double two_pi = 6.283185307179586476925286766559;
  std::memset(out, 0, tcc::OPS_BYTES);
  auto put = [&](int off_part, int off_elem, double v, int part) {
    uint16_t h = bf16_bits(v);
    if (part == 1) h = bf16_bits(v - bf16_value(h));
    std::memcpy(out + off_part + off_elem, &h, 2);
  };
  for (int n = 0; n < 64; ++n)
    for (int k = 0; k < 64; ++k) {
      const double th = two_pi * (double)((n * k) & 63) / 64.0;
      const int o = tcc::off_k64(n, k);
      put(tcc::OFF_C64_HI, o, std::cos(th), 0);
      put(tcc::OFF_C64_MID, o, std::cos(th), 1);
      put(tcc::OFF_S64_HI, o, std::sin(th), 0);
      put(tcc::OFF_S64_MID, o, std::sin(th), 1);
    }
  for (int n = 0; n < 32; ++n)
    for (int k = 0; k < 32; ++k) {
      const double th = two_pi * (double)((n * k) & 31) / 32.0;
      const int o = tcc::off_k32(n, k);
      put(tcc::OFF_C32_HI, o, std::cos(th), 0);
      put(tcc::OFF_C32_MID, o, std::cos(th), 1);
      put(tcc::OFF_S32_HI, o, std::sin(th), 0);
      put(tcc::OFF_S32_MID, o, std::sin(th), 1);
    }
  for (int i = 0; i < 64; ++i) {
    const float v[2] = {(float)std::cos(two_pi * i / 2048.0), (float)std::sin(two_pi * i / 2048.0)};
    std::memcpy(out + tcc::OFF_T0 + 8 * i, v, 8);
  }
  for (int j = 0; j < 32; ++j) {
    const float v[2] = {(float)std::cos(two_pi * 64 * j / 2048.0), (float)std::sin(two_pi * 64 * j / 2048.0)};
    std::memcpy(out + tcc::OFF_T1 + 8 * j, v, 8);
  }
}

int ic_tc_ops_bytes() { return tcc::OPS_BYTES; }

}  // namespace pond
