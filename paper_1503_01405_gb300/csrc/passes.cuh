// The four FFT passes of a segment (PONDER Sec. 3.7), templated on the line
// length and on the arithmetic of their radix-16 stages: FP32 butterflies
// (TC = false) or split-BF16 16-point DFT-matrix products on the tensor cores
// (TC = true, tc_dft.cuh).  kernels.cu instantiates the FP32 form and
// kernels_tc.cu the tensor-core form; both share everything else.
//
//  F1 k_fwd_cols   : unpack z[n] = x[2n] + i x[2n+1]; length-R2 FFTs down the
//                    R1 columns n1 of z viewed as [R2][R1]; multiply by
//                    exp(-2 pi i n1 k2 / L); store in place of the column.
//  F2 k_fwd_rows   : length-R1 FFTs along the rows k2 (Z[k2 + R2 k1]); rows k2
//                    and R2-k2 share a CTA so the real-input split
//                    X[k] = (Z[k] + Z*[L-k])/2 - i e^{-i pi k/L} (Z[k] - Z*[L-k])/2
//                    is local; multiply by the inverse ISM response (Eq. 4);
//                    store Y[k] in natural order.
//  I1 k_inv_cols   : per sub-channel c (bins cM..cM+M-1), inverse length-Q2
//                    FFTs down the Q1 columns j1, multiply by exp(+2 pi i j1 m2 / M).
//  I2 k_inv_rows   : inverse length-Q1 FFTs along rows m2 for all sub-channels
//                    of the same m2 in one CTA: v_c[m2 + Q2 m1] / M, keep the
//                    valid span n_past <= m < M - n_fut, detect |v|^2 and sum
//                    over sub-channels into P (and optionally store v).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "fft_block.cuh"
#include "pond_internal.h"
#include "tc_dft.cuh"

namespace pond {

// exp(-2 pi i phi(k)) from the anchor table (phase error < 1e-7 cycles).
__device__ __forceinline__ float2 chirp_factor(const ChirpAnchor* __restrict__ anc, int clog, unsigned k) {
  const ChirpAnchor a = anc[k >> clog];
  const int d = (int)(k & ((1u << clog) - 1)) - (int)((1u << clog) >> 1);
  const unsigned u = a.p0 + a.p1 * (unsigned)d;           // mod 2^32: phase mod 1 cycle
  const float df = (float)d;
  float r = (float)(int)u * 2.3283064365386963e-10f;      // 2^-32
  r += fmaf(a.p3, df, a.p2) * (df * df);
  float s, c;
  sincospif(2.0f * r, &s, &c);
  return make_float2(c, -s);
}


__device__ __forceinline__ float2 tw2(const Tw2& t, unsigned e) {
  return cmul(__ldg(t.hi + (e >> TW2_LOG)), __ldg(t.lo + (e & (TW2_LO - 1))));
}

constexpr int EPT = TILE / NT;   // tile elements per thread


// Tile entries (float2) a pass allocates for nl lines of length R.  The
// tensor-core form pads its tile so that the CTA's shared memory (tables +
// tile + extras) is at least tc::MIN_SMEM_BYTES: then at most two CTAs share
// an SM and their 2 x 256 TMEM columns always fit.
template <int R, bool TC>
__host__ __device__ constexpr int tile_f2(int nl) {
  return TC ? (nl * line_stride(R) > tc::MIN_TILE_F2 - stage_table_size(R)
                   ? nl * line_stride(R)
                   : tc::MIN_TILE_F2 - stage_table_size(R))
            : nl * line_stride(R);
}

// ---------------------------------------------------------------------------
// F1: unpack + column FFTs of the forward transform
// ---------------------------------------------------------------------------

__device__ __forceinline__ float sample_at(const SegIn& in, long long r) {
  if (r < in.a_len) return (float)in.a[r];
  r -= in.a_len;
  if (r < in.b_len) return (float)in.b[r];
  return 0.f;
}

// z viewed as [R2][R1] (z[n1 + R1 n2]); a CTA transforms nl adjacent columns n1
// and stores them in place, scaled by exp(-2 pi i n1 k2 / L).
template <int R2, bool TC>
__global__ void __launch_bounds__(NT) k_fwd_cols(SegIn in, float2* __restrict__ out, int logR1, Tw2 twL,
                                                    const float2* __restrict__ tw, TcArgs tca) {
  extern __shared__ float2 smem[];
  float2* stw = smem;
  float2* sm = smem + stage_table_size(R2);
  constexpr int LSTR = line_stride(R2);
  const int R1 = 1 << logR1;
  const int nl = min(TILE / R2, R1);
  const int lognl = __ffs(nl) - 1;
  const int tot = nl * R2;
  load_twiddles<R2>(stw, tw);
  tc::Ctx tcc;
  if constexpr (TC) tc::setup(tcc, sm, tile_f2<R2, TC>(nl), tca);
  const int tile = blockIdx.x;
  const int n1_0 = tile * nl;
  if (in.vec8) {
    // 8-byte loads: 4 consecutive columns of one row per load (runs 8-aligned)
    constexpr int CPT = EPT / 4;
    const int logq = lognl - 2;            // chunks per row = nl / 4
    uint2 w[CPT];
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
      const int c = threadIdx.x + u * NT;
      if (c < tot / 4) {
        const int n2 = c >> logq, b0 = (c & ((nl >> 2) - 1)) << 2;
        const long long r = 2 * ((long long)(n1_0 + b0) + ((long long)n2 << logR1));
        if (r < in.a_len) w[u] = __ldg(reinterpret_cast<const uint2*>(in.a + r));
        else if (r - in.a_len < in.b_len) w[u] = __ldg(reinterpret_cast<const uint2*>(in.b + (r - in.a_len)));
        else w[u] = make_uint2(0u, 0u);
      }
    }
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
      const int c = threadIdx.x + u * NT;
      if (c < tot / 4) {
        const int n2 = c >> logq, b0 = (c & ((nl >> 2) - 1)) << 2;
        const unsigned lo = w[u].x, hi = w[u].y;
        sm[pidx(b0 + 0, n2, LSTR)] = make_float2((float)(signed char)(lo & 0xff), (float)(signed char)((lo >> 8) & 0xff));
        sm[pidx(b0 + 1, n2, LSTR)] = make_float2((float)(signed char)((lo >> 16) & 0xff), (float)(signed char)(lo >> 24));
        sm[pidx(b0 + 2, n2, LSTR)] = make_float2((float)(signed char)(hi & 0xff), (float)(signed char)((hi >> 8) & 0xff));
        sm[pidx(b0 + 3, n2, LSTR)] = make_float2((float)(signed char)((hi >> 16) & 0xff), (float)(signed char)(hi >> 24));
      }
    }
  } else {
    float2 r[EPT];
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      const int idx = threadIdx.x + u * NT;
      if (idx < tot) {
        const int n2 = idx >> lognl, b = idx & (nl - 1);
        const long long q = (long long)(n1_0 + b) + ((long long)n2 << logR1);
        r[u] = make_float2(sample_at(in, 2 * q), sample_at(in, 2 * q + 1));
      }
    }
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      const int idx = threadIdx.x + u * NT;
      if (idx < tot) sm[pidx(idx & (nl - 1), idx >> lognl, LSTR)] = r[u];
    }
  }
  __syncthreads();
  fft_lines<R2, false, TC>(sm, nl, stw, &tcc);
  if constexpr (TC) tc::teardown(tcc);
#pragma unroll 4
  for (int idx = threadIdx.x; idx < tot; idx += NT) {
    const int k2 = idx >> lognl, b = idx & (nl - 1);
    const unsigned n1 = (unsigned)(n1_0 + b);
    out[(size_t)n1 + ((size_t)k2 << logR1)] = cmul(sm[pidx(b, k2, LSTR)], tw2(twL, n1 * (unsigned)k2));
  }
}

// ---------------------------------------------------------------------------
// F2: row FFTs + real-input split + dedispersion chirp
// ---------------------------------------------------------------------------

// Row k2 of the column-transformed z holds, after a length-R1 FFT, Z[k2 + R2 k1].
// Rows k2 and R2-k2 share a CTA (row 0 and row R2/2 pair with themselves) so that
// X[k] can be formed from Z[k] and Z[L-k]; the chirped spectrum Y[k2 + R2 k1] is
// stored at row k2, column k1 of the output (the same place the row was read).
template <int R1, bool TC>
__global__ void __launch_bounds__(NT) k_fwd_rows(const float2* __restrict__ in, float2* __restrict__ out,
                                                    int logR2, int logL, Tw2 tw2L,
                                                    const ChirpAnchor* __restrict__ anc, int clog, int apply_chirp,
                                                    const float2* __restrict__ tw, TcArgs tca) {
  extern __shared__ float2 smem[];
  float2* stw = smem;
  float2* sm = smem + stage_table_size(R1);
  constexpr int LSTR = line_stride(R1);
  constexpr int LOGR1 = ilog2c(R1);
  const int R2 = 1 << logR2;
  const int nl = min(TILE / R1, R2);   // 2 * pairs
  const int np = nl >> 1;
  const int tot = nl * R1;
  load_twiddles<R1>(stw, tw);
  tc::Ctx tcc;
  if constexpr (TC) tc::setup(tcc, sm, tile_f2<R1, TC>(nl), tca);
  const int tile = blockIdx.x;
  const int q0 = tile * np;
  auto line_of = [&](int slot) -> int {
    if (slot < np) return q0 + slot;
    const int t = slot - np;
    if (q0 + t == 0) return R2 >> 1;          // row R2/2 pairs with itself
    return R2 - (q0 + t);
  };
  float2 r[EPT];
#pragma unroll
  for (int u = 0; u < EPT; ++u) {
    const int idx = threadIdx.x + u * NT;
    if (idx < tot) r[u] = in[((size_t)line_of(idx >> LOGR1) << LOGR1) + (idx & (R1 - 1))];
  }
#pragma unroll
  for (int u = 0; u < EPT; ++u) {
    const int idx = threadIdx.x + u * NT;
    if (idx < tot) sm[pidx(idx >> LOGR1, idx & (R1 - 1), LSTR)] = r[u];
  }
  __syncthreads();
  fft_lines<R1, false, TC>(sm, nl, stw, &tcc);
  if constexpr (TC) tc::teardown(tcc);
  const unsigned lmask = (1u << logL) - 1;
#pragma unroll 4
  for (int idx = threadIdx.x; idx < tot; idx += NT) {
    const int slot = idx >> LOGR1, k1 = idx & (R1 - 1);
    const int line = line_of(slot);
    const unsigned k = (unsigned)line + ((unsigned)k1 << logR2);
    const unsigned kp = (0u - k) & lmask;
    const int linep = (int)(kp & (unsigned)(R2 - 1));
    const int k1p = (int)(kp >> logR2);
    const int slotp = (linep == line) ? slot : (slot < np ? slot + np : slot - np);
    const float2 A = sm[pidx(slot, k1, LSTR)];
    const float2 B = cconj(sm[pidx(slotp, k1p, LSTR)]);
    const float2 E = cscale(cadd(A, B), 0.5f);
    const float2 O = cscale(csub(A, B), 0.5f);
    float2 X = cadd(E, rot90<false>(cmul(tw2(tw2L, k), O)));   // E - i exp(-i pi k/L) O
    if (apply_chirp) X = cmul(X, chirp_factor(anc, clog, k));
    out[((size_t)line << LOGR1) + k1] = X;
  }
}

// ---------------------------------------------------------------------------
// I1: per-sub-channel inverse column FFTs
// ---------------------------------------------------------------------------

// Line (c, j1) holds Y[c M + j1 + Q1 j2], j2 < Q2, read from the row layout
// written by F2 (bin k at (k >> logR2) + (k mod R2) R1; with Q1 <= R2 the
// values j2 = j2lo + 2^s j2hi, s = logR2 - logQ1, lie in runs of M/R2
// consecutive addresses in j2hi).  The inverse column transform, scaled by
// exp(+2 pi i j1 m2 / M), is stored in natural order c M + j1 + Q1 m2.
template <int Q2, bool TC>
__global__ void __launch_bounds__(NT) k_inv_cols(const float2* __restrict__ in, float2* __restrict__ out,
                                                    int logQ1, int logM, int logR1, int logR2, int nchan, Tw2 twM,
                                                    const ChirpAnchor* __restrict__ anc, int clog,
                                                    const float2* __restrict__ tw, TcArgs tca) {
  extern __shared__ float2 smem[];
  float2* stw = smem;
  float2* sm = smem + stage_table_size(Q2);
  constexpr int LSTR = line_stride(Q2);
  constexpr int LOGQ2 = ilog2c(Q2);
  const int Q1 = 1 << logQ1;
  const int nl = min(TILE / Q2, nchan * Q1);
  const int lognl = __ffs(nl) - 1;
  const int tot = nl * Q2;
  load_twiddles<Q2>(stw, tw);
  tc::Ctx tcc;
  if constexpr (TC) tc::setup(tcc, sm, tile_f2<Q2, TC>(nl), tca);
  const int tile = blockIdx.x;
  const int l0 = tile * nl;
  const int s = logR2 - logQ1;                 // j2 = j2lo + 2^s j2hi
  const int logrun = LOGQ2 - s;                // run length M / R2 (>= 1)
  float2 r[EPT];
#pragma unroll
  for (int u = 0; u < EPT; ++u) {
    const int idx = threadIdx.x + u * NT;
    if (idx < tot) {
      const int j2hi = idx & ((1 << logrun) - 1);
      const int rest = idx >> logrun;
      const int j2lo = rest & ((1 << s) - 1);
      const int l = l0 + (rest >> s);
      const int c = l >> logQ1, j1 = l & (Q1 - 1);
      const size_t k1 = ((size_t)c << (logM - logR2)) + j2hi;
      const size_t k2 = (size_t)j1 + ((size_t)j2lo << logQ1);
      r[u] = in[k1 + (k2 << logR1)];
      if (anc) r[u] = cmul(r[u], chirp_factor(anc, clog, (unsigned)(k2 + (k1 << logR2))));
    }
  }
#pragma unroll
  for (int u = 0; u < EPT; ++u) {
    const int idx = threadIdx.x + u * NT;
    if (idx < tot) {
      const int j2hi = idx & ((1 << logrun) - 1);
      const int rest = idx >> logrun;
      const int j2lo = rest & ((1 << s) - 1);
      sm[pidx(rest >> s, j2lo + (j2hi << s), LSTR)] = r[u];
    }
  }
  __syncthreads();
  fft_lines<Q2, true, TC>(sm, nl, stw, &tcc);
  if constexpr (TC) tc::teardown(tcc);
#pragma unroll 4
  for (int idx = threadIdx.x; idx < tot; idx += NT) {
    const int m2 = idx >> lognl, b = idx & (nl - 1);
    const int l = l0 + b;
    const unsigned j1 = (unsigned)(l & (Q1 - 1));
    const size_t addr = ((size_t)(l >> logQ1) << logM) + j1 + ((size_t)m2 << logQ1);
    out[addr] = cmul(sm[pidx(b, m2, LSTR)], tw2(twM, j1 * (unsigned)m2));
  }
}

// ---------------------------------------------------------------------------
// I2: inverse row FFTs, discard, detect, sum over sub-channels
// ---------------------------------------------------------------------------

template <int Q1, bool TC>
__global__ void __launch_bounds__(NT) k_inv_rows(const float2* __restrict__ buf, float* __restrict__ P,
                                                    float2* __restrict__ vout, long long vstride,
                                                    long long vofs, int logQ2, int logM, int nchan,
                                                    int m_lo, int m_hi, float scale,
                                                    const float2* __restrict__ tw, TcArgs tca) {
  extern __shared__ float2 smem[];
  float2* stw = smem;
  float2* sm = smem + stage_table_size(Q1);
  constexpr int LSTR = line_stride(Q1);
  constexpr int LOGQ1 = ilog2c(Q1);
  const int Q2 = 1 << logQ2;
  const int b2 = min(TILE / (Q1 * nchan), Q2);
  const int logb2 = __ffs(b2) - 1;
  const int nl = nchan * b2;
  const int tot = nl * Q1;
  load_twiddles<Q1>(stw, tw);
  tc::Ctx tcc;
  if constexpr (TC) tc::setup(tcc, sm, tile_f2<Q1, TC>(nl), tca);
  const int tile = blockIdx.x;
  const int m2_0 = tile * b2;
  float2 r[EPT];
#pragma unroll
  for (int u = 0; u < EPT; ++u) {
    const int idx = threadIdx.x + u * NT;
    if (idx < tot) {
      const int slot = idx >> LOGQ1, e = idx & (Q1 - 1);
      const int c = slot >> logb2, bb = slot & (b2 - 1);
      r[u] = buf[((size_t)c << logM) + ((size_t)(m2_0 + bb) << LOGQ1) + e];
    }
  }
#pragma unroll
  for (int u = 0; u < EPT; ++u) {
    const int idx = threadIdx.x + u * NT;
    if (idx < tot) sm[pidx(idx >> LOGQ1, idx & (Q1 - 1), LSTR)] = r[u];
  }
  __syncthreads();
  fft_lines<Q1, true, TC>(sm, nl, stw, &tcc);
  if constexpr (TC) tc::teardown(tcc);
  for (int idx = threadIdx.x; idx < b2 * Q1; idx += NT) {
    const int m1 = idx >> logb2, bb = idx & (b2 - 1);
    const int m = m2_0 + bb + (m1 << logQ2);
    if (m < m_lo || m >= m_hi) continue;
    float p = 0.f;
    for (int c = 0; c < nchan; ++c) {
      const float2 v = cscale(sm[pidx((c << logb2) + bb, m1, LSTR)], scale);
      p = fmaf(v.x, v.x, p);
      p = fmaf(v.y, v.y, p);
      if (vout) vout[(size_t)c * vstride + vofs + (m - m_lo)] = v;
    }
    P[m - m_lo] = p;
  }
}


// ---------------------------------------------------------------------------
// Host launchers (one CTA per tile)
// ---------------------------------------------------------------------------

// Stage twiddle tables + padded tile (+ the tensor-core extras).
template <int R, bool TC>
size_t smem_bytes(int nl) {
  return ((size_t)stage_table_size(R) + (size_t)tile_f2<R, TC>(nl)) * sizeof(float2) +
         (TC ? (size_t)tc::EXTRA_BYTES : 0);
}

#define POND_FOR_R(X) X(4) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096)

// Largest dynamic shared memory over the line lengths 4..4096.
template <bool TC>
size_t max_smem_t() {
  size_t m = 0;
#define MAXS(R) m = std::max(m, smem_bytes<R, TC>(TILE / R));
  POND_FOR_R(MAXS)
#undef MAXS
  return m;
}

template <bool TC>
cudaError_t set_attributes_t() {
  const int max_smem = (int)max_smem_t<TC>();
  cudaError_t e = cudaSuccess;
#define SET_ATTR(R)                                                                                   \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fwd_cols<R, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem); \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fwd_rows<R, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem); \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_inv_cols<R, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem); \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_inv_rows<R, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  POND_FOR_R(SET_ATTR)
#undef SET_ATTR
  return e;
}

template <bool TC>
cudaError_t launch_fwd_cols_t(const Geom& g, SegIn in, float2* out, Tw2 twL, const float2* tw, cudaStream_t st) {
  const int R2 = 1 << g.logR2, R1 = 1 << g.logR1;
  const int nl = std::min(TILE / R2, R1);
  const unsigned grid = (unsigned)(R1 / nl);
  switch (R2) {
#define CASE(R) case R: k_fwd_cols<R, TC><<<grid, NT, smem_bytes<R, TC>(nl), st>>>(in, out, g.logR1, twL, tw, g.tc_fwd); break;
    POND_FOR_R(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <bool TC>
cudaError_t launch_fwd_rows_t(const Geom& g, const float2* in, float2* out, Tw2 tw2L, const ChirpAnchor* anc,
                              int clog, int apply_chirp, const float2* tw, cudaStream_t st) {
  const int R2 = 1 << g.logR2, R1 = 1 << g.logR1;
  const int nl = std::min(TILE / R1, R2);
  const unsigned grid = (unsigned)(R2 / nl);
  switch (R1) {
#define CASE(R) case R: k_fwd_rows<R, TC><<<grid, NT, smem_bytes<R, TC>(nl), st>>>(in, out, g.logR2, g.logL, tw2L, anc, clog, apply_chirp, tw, g.tc_fwd); break;
    POND_FOR_R(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <bool TC>
cudaError_t launch_inv_cols_t(const Geom& g, const float2* in, float2* out, Tw2 twM, const ChirpAnchor* anc,
                              int clog, const float2* tw, cudaStream_t st) {
  const int Q2 = 1 << g.logQ2, Q1 = 1 << g.logQ1;
  const int lines = g.nchan * Q1;
  const int nl = std::min(TILE / Q2, lines);
  const unsigned grid = (unsigned)(lines / nl);
  switch (Q2) {
#define CASE(R) case R: k_inv_cols<R, TC><<<grid, NT, smem_bytes<R, TC>(nl), st>>>(in, out, g.logQ1, g.logM, g.logR1, g.logR2, g.nchan, twM, anc, clog, tw, g.tc_inv); break;
    POND_FOR_R(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <bool TC>
cudaError_t launch_inv_rows_t(const Geom& g, const float2* buf, float* P, float2* vout, long long vstride,
                              long long vofs, int m_lo, int m_hi, const float2* tw, cudaStream_t st) {
  const int Q2 = 1 << g.logQ2, Q1 = 1 << g.logQ1;
  const int b2 = std::min(TILE / (Q1 * g.nchan), Q2);
  const int nl = g.nchan * b2;
  const unsigned grid = (unsigned)(Q2 / b2);
  const float scale = 1.0f / (float)(1u << g.logM);
  switch (Q1) {
#define CASE(R) case R: k_inv_rows<R, TC><<<grid, NT, smem_bytes<R, TC>(nl), st>>>(buf, P, vout, vstride, vofs, g.logQ2, g.logM, g.nchan, m_lo, m_hi, scale, tw, g.tc_inv); break;
    POND_FOR_R(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Tensor-core instantiations (kernels_tc.cu).
cudaError_t launch_fwd_cols_tc(const Geom& g, SegIn in, float2* out, Tw2 twL, const float2* tw, cudaStream_t st);
cudaError_t launch_fwd_rows_tc(const Geom& g, const float2* in, float2* out, Tw2 tw2L, const ChirpAnchor* anc,
                               int clog, int apply_chirp, const float2* tw, cudaStream_t st);
cudaError_t launch_inv_cols_tc(const Geom& g, const float2* in, float2* out, Tw2 twM, const ChirpAnchor* anc,
                               int clog, const float2* tw, cudaStream_t st);
cudaError_t launch_inv_rows_tc(const Geom& g, const float2* buf, float* P, float2* vout, long long vstride,
                               long long vofs, int m_lo, int m_hi, const float2* tw, cudaStream_t st);

}  // namespace pond
