// Segment kernels of the coherent-dedispersion path (PONDER Sec. 3.7).
//
// One overlap-save segment of N real int8 samples goes through four FFT passes
// over a spectrum of L = N/2 complex bins, then fold and decimation:
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
//  k_fold_partial / k_fold_merge : deterministic fold of P (FP64 phase).
//  k_decimate      : deterministic decimation of P into the time series.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_block.cuh"
#include "pond_internal.h"

namespace pond {

// ---------------------------------------------------------------------------
// Tables (built once per plan, FP64 on the device)
// ---------------------------------------------------------------------------

// Concatenated stage twiddle tables of a length-R line FFT (see fft_block.cuh):
// entry (j-1) LS + k of the stage after sub-transforms of length LS holds
// exp(-2 pi i j k / (LS RAD)).
__global__ void k_make_stage_tw(float2* out, int R) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  int off = 0;
  for (int ls = 1; ls < R; ls *= stage_radix(R, ls)) {
    const int rad = stage_radix(R, ls);
    if (ls == 1) continue;
    const int n = (rad - 1) * ls;
    if (m >= off && m < off + n) {
      const int j = (m - off) / ls + 1, k = (m - off) % ls;
      double sn, cs;
      sincospi(-2.0 * (double)(j * k) / (double)(ls * rad), &sn, &cs);
      out[m] = make_float2((float)cs, (float)sn);
    }
    off += n;
  }
}

// Anchor a covers the 2^clog bins k = 2^clog a + d (d < 2^clog); it holds the
// Taylor coefficients of the dedispersion phase phi(k) = sgn * c(f_k) (cycles)
// about k_a = 2^clog a + 2^(clog-1): phi(k_a) and phi'(k_a) reduced mod 1 in
// Q0.32 fixed point, phi''/2 and phi'''/6 in FP32.  c(f) = alpha f^2 / (f0 + f)
// with alpha = K 1e6 DM / f0^2 (Eq. 4), f = k du - |bw|/2 (upper sideband) or
// |bw|/2 - k du (inverted).  The planner picks clog so that the dropped quartic
// term stays below 1e-9 cycles.
__global__ void k_make_chirp_anchors(ChirpAnchor* anc, long long nanc, int clog, double du, double half,
                                     double f0, double alpha, int sgn) {
  const long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nanc) return;
  const long long span = 1ll << clog;
  const double ka = (double)(a * span + span / 2);
  const double f = sgn > 0 ? __dsub_rn(__dmul_rn(ka, du), half) : __dsub_rn(half, __dmul_rn(ka, du));
  const double g = f0 + f;
  const double q = f0 * f0 / (g * g);
  const double c = alpha * f * f / g;
  const double d1 = alpha * (1.0 - q);
  const double d2 = 2.0 * alpha * q / g;
  const double d3 = -6.0 * alpha * q / (g * g);
  const double phi0 = sgn * c;
  const double phi1 = du * d1;
  const double phi2 = sgn * du * du * d2 * 0.5;
  const double phi3 = du * du * du * d3 / 6.0;
  const double fr0 = phi0 - floor(phi0);
  const double fr1 = phi1 - floor(phi1);
  ChirpAnchor r;
  r.p0 = (unsigned)((unsigned long long)llrint(fr0 * 4294967296.0) & 0xffffffffull);
  r.p1 = (unsigned)((unsigned long long)llrint(fr1 * 4294967296.0) & 0xffffffffull);
  r.p2 = (float)phi2;
  r.p3 = (float)phi3;
  anc[a] = r;
}

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

// ---------------------------------------------------------------------------
// Two-level twiddle tables: w^e = hi[e >> 12] * lo[e & 4095], w = exp(+-2 pi i / n)
// ---------------------------------------------------------------------------

__global__ void k_make_tw2(float2* lo, float2* hi, int logn, int sign) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const double inv = 2.0 * sign / (double)(1ll << logn);
  double s, c;
  if (i < TW2_LO) {
    sincospi(inv * (double)i, &s, &c);
    lo[i] = make_float2((float)c, (float)s);
  }
  const long long nhi = logn > TW2_LOG ? (1ll << (logn - TW2_LOG)) : 1;
  if (i < nhi) {
    sincospi(inv * (double)((long long)i << TW2_LOG), &s, &c);
    hi[i] = make_float2((float)c, (float)s);
  }
}

__device__ __forceinline__ float2 tw2(const Tw2& t, unsigned e) {
  return cmul(__ldg(t.hi + (e >> TW2_LOG)), __ldg(t.lo + (e & (TW2_LO - 1))));
}

constexpr int EPT = TILE / NT;   // tile elements per thread

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
template <int R2>
__global__ void __launch_bounds__(NT) k_fwd_cols(SegIn in, float2* __restrict__ out, int logR1, Tw2 twL,
                                                    const float2* __restrict__ tw) {
  extern __shared__ float2 smem[];
  float2* stw = smem;
  float2* sm = smem + stage_table_size(R2);
  constexpr int LSTR = line_stride(R2);
  const int R1 = 1 << logR1;
  const int nl = min(TILE / R2, R1);
  const int lognl = __ffs(nl) - 1;
  const int tot = nl * R2;
  load_twiddles<R2>(stw, tw);
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
  block_fft<R2, false>(sm, nl, stw);
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
template <int R1>
__global__ void __launch_bounds__(NT) k_fwd_rows(const float2* __restrict__ in, float2* __restrict__ out,
                                                    int logR2, int logL, Tw2 tw2L,
                                                    const ChirpAnchor* __restrict__ anc, int clog, int apply_chirp,
                                                    const float2* __restrict__ tw) {
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
  block_fft<R1, false>(sm, nl, stw);
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
template <int Q2>
__global__ void __launch_bounds__(NT) k_inv_cols(const float2* __restrict__ in, float2* __restrict__ out,
                                                    int logQ1, int logM, int logR1, int logR2, int nchan, Tw2 twM,
                                                    const ChirpAnchor* __restrict__ anc, int clog,
                                                    const float2* __restrict__ tw) {
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
  block_fft<Q2, true>(sm, nl, stw);
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

template <int Q1>
__global__ void __launch_bounds__(NT) k_inv_rows(const float2* __restrict__ buf, float* __restrict__ P,
                                                    float2* __restrict__ vout, long long vstride,
                                                    long long vofs, int logQ2, int logM, int nchan,
                                                    int m_lo, int m_hi, float scale,
                                                    const float2* __restrict__ tw) {
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
  block_fft<Q1, true>(sm, nl, stw);
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
// Fold (Sec. 3.4 fold thread): deterministic per-warp histograms
// ---------------------------------------------------------------------------

constexpr int FOLD_WARPS = 4;

// bin(g) = min(floor(frac(g * inc) * nbins), nbins - 1), FP64, correctly rounded.
__device__ __forceinline__ int fold_bin(long long g, double inc, int nbins) {
  const double x = __dmul_rn((double)g, inc);
  const double ph = __dsub_rn(x, floor(x));
  const int b = (int)__dmul_rn(ph, (double)nbins);
  return b < nbins - 1 ? b : nbins - 1;
}

__global__ void __launch_bounds__(FOLD_WARPS * 32) k_fold_partial(const float* __restrict__ P, long long n,
                                                                  long long g0, double inc, int nbins,
                                                                  long long chunk, double* __restrict__ psum,
                                                                  int* __restrict__ phits) {
  extern __shared__ unsigned char fsm[];
  double* hsum = reinterpret_cast<double*>(fsm);                  // [FOLD_WARPS][nbins]
  int* hcnt = reinterpret_cast<int*>(hsum + FOLD_WARPS * nbins);  // [FOLD_WARPS][nbins]
  float* pbuf = reinterpret_cast<float*>(hcnt + FOLD_WARPS * nbins);  // [FOLD_WARPS][32]
  for (int i = threadIdx.x; i < FOLD_WARPS * nbins; i += blockDim.x) {
    hsum[i] = 0.0;
    hcnt[i] = 0;
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long c0 = (long long)blockIdx.x * chunk;
  const long long c1 = min(n, c0 + chunk);
  double* myh = hsum + w * nbins;
  int* myc = hcnt + w * nbins;
  float* mybuf = pbuf + w * 32;
  for (long long base = c0 + w * 32; base < c1; base += FOLD_WARPS * 32) {
    const long long i = base + lane;
    const bool ok = i < c1;
    int b = -1;
    float p = 0.f;
    if (ok) {
      b = fold_bin(g0 + i, inc, nbins);
      p = P[i];
    }
    const unsigned peers = __match_any_sync(0xffffffffu, b);
    const int first = __ffs(peers) - 1;
    const int last = 31 - __clz(peers);
    const unsigned span = (last == 31 ? 0xffffffffu : ((1u << (last + 1)) - 1u)) & ~((1u << first) - 1u);
    if (__all_sync(0xffffffffu, peers == span)) {
      // every bin's lanes are contiguous: segmented scan in a fixed tree order
      float x = p;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const float y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane - d >= first) x += y;
      }
      if (ok && lane == last) {
        myh[b] += (double)x;
        myc[b] += last - first + 1;
      }
    } else {
      // a period shorter than a warp: the group leader sums its lanes in order
      mybuf[lane] = p;
      __syncwarp();
      if (ok && lane == first) {
        float sum = 0.f;
        unsigned m = peers;
        while (m) {
          sum += mybuf[__ffs(m) - 1];
          m &= m - 1;
        }
        myh[b] += (double)sum;
        myc[b] += __popc(peers);
      }
    }
    __syncwarp();
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
    double s = 0.0;
    int h = 0;
#pragma unroll
    for (int k = 0; k < FOLD_WARPS; ++k) {
      s += hsum[k * nbins + b];
      h += hcnt[k * nbins + b];
    }
    psum[(size_t)blockIdx.x * nbins + b] = s;
    phits[(size_t)blockIdx.x * nbins + b] = h;
  }
}

// One warp per bin: lanes take every 32nd part, then a fixed xor-tree sum.
__global__ void k_fold_merge(const double* __restrict__ psum, const int* __restrict__ phits, int nparts,
                             int nbins, double* __restrict__ prof_sum, long long* __restrict__ prof_hits) {
  const int b = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= nbins) return;
  double s = 0.0;
  long long h = 0;
#pragma unroll 4
  for (int k = lane; k < nparts; k += 32) {
    s += psum[(size_t)k * nbins + b];
    h += phits[(size_t)k * nbins + b];
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, off);
    h += __shfl_xor_sync(0xffffffffu, h, off);
  }
  if (lane == 0) {
    prof_sum[b] += s;
    prof_hits[b] += h;
  }
}

// ---------------------------------------------------------------------------
// Decimation: T[j] += sum of P[g], floor(g den / num) = j; one warp per j
// ---------------------------------------------------------------------------

__device__ __forceinline__ long long ceil_div_ll(long long a, long long b) { return (a + b - 1) / b; }

__global__ void k_decimate(const float* __restrict__ P, long long n, long long g0, long long num,
                           long long den, long long j_lo, long long nj, float* __restrict__ T,
                           int* __restrict__ C, long long ring) {
  const long long jj = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (jj >= nj) return;
  const long long j = j_lo + jj;
  long long ga = ceil_div_ll(j * num, den), gb = ceil_div_ll((j + 1) * num, den);
  ga = max(ga, g0);
  gb = min(gb, g0 + n);
  float s = 0.f;
  for (long long g = ga + lane; g < gb; g += 32) s += P[g - g0];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) {
    const long long slot = j % ring;
    T[slot] += s;
    C[slot] += (int)(gb - ga);
  }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------

// Stage twiddle tables + padded tile (nl lines of line_stride(R)).
template <int R>
static size_t smem_bytes(int nl) {
  return ((size_t)stage_table_size(R) + (size_t)nl * line_stride(R)) * sizeof(float2);
}

// Largest stage tables + padded tile over the line lengths 4..4096.
static size_t max_tile_smem_bytes() {
  size_t m = 0;
  for (int R = 4; R <= 4096; R *= 2)
    m = std::max(m, ((size_t)stage_table_size(R) + (size_t)(TILE / R) * (R + R / 16 + 1)) * sizeof(float2));
  return m;
}

cudaError_t launch_stage_tw(float2* out, int R, cudaStream_t st) {
  const int n = stage_table_size(R);
  if (n > 0) k_make_stage_tw<<<(n + 255) / 256, 256, 0, st>>>(out, R);
  return cudaGetLastError();
}

int stage_tw_entries(int R) { return stage_table_size(R); }

// One CTA per tile.
static unsigned grid_for(int tiles, int) { return (unsigned)tiles; }

#define POND_FOR_R(X) X(4) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096)

cudaError_t set_kernel_attributes() {
  const int max_smem = (int)max_tile_smem_bytes();
  cudaError_t e = cudaSuccess;
#define SET_ATTR(R)                                                                                   \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fwd_cols<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem); \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fwd_rows<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem); \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_inv_cols<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem); \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_inv_rows<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
  POND_FOR_R(SET_ATTR)
#undef SET_ATTR
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fold_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, fold_smem_bytes(MAX_NBINS));
  return e;
}

cudaError_t launch_tw2(float2* lo, float2* hi, int logn, int sign, cudaStream_t st) {
  const long long nhi = logn > TW2_LOG ? (1ll << (logn - TW2_LOG)) : 1;
  const long long n = std::max<long long>(TW2_LO, nhi);
  k_make_tw2<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(lo, hi, logn, sign);
  return cudaGetLastError();
}

cudaError_t launch_tables(ChirpAnchor* anc, long long nanc, int clog, double du, double half,
                          double f0, double alpha, int sgn, cudaStream_t st) {
  k_make_chirp_anchors<<<(unsigned)((nanc + 127) / 128), 128, 0, st>>>(anc, nanc, clog, du, half, f0, alpha, sgn);
  return cudaGetLastError();
}

cudaError_t launch_fwd_cols(const Geom& g, SegIn in, float2* out, Tw2 twL, const float2* tw, cudaStream_t st) {
  const int R2 = 1 << g.logR2, R1 = 1 << g.logR1;
  const int nl = std::min(TILE / R2, R1);
  const unsigned grid = grid_for(R1 / nl, g.sms);
  switch (R2) {
#define CASE(R) case R: k_fwd_cols<R><<<grid, NT, smem_bytes<R>(nl), st>>>(in, out, g.logR1, twL, tw); break;
    POND_FOR_R(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_fwd_rows(const Geom& g, const float2* in, float2* out, Tw2 tw2L, const ChirpAnchor* anc, int clog,
                            int apply_chirp, const float2* tw, cudaStream_t st) {
  const int R2 = 1 << g.logR2, R1 = 1 << g.logR1;
  const int nl = std::min(TILE / R1, R2);
  const unsigned grid = grid_for(R2 / nl, g.sms);
  switch (R1) {
#define CASE(R) case R: k_fwd_rows<R><<<grid, NT, smem_bytes<R>(nl), st>>>(in, out, g.logR2, g.logL, tw2L, anc, clog, apply_chirp, tw); break;
    POND_FOR_R(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_inv_cols(const Geom& g, const float2* in, float2* out, Tw2 twM, const ChirpAnchor* anc,
                            int clog, const float2* tw, cudaStream_t st) {
  const int Q2 = 1 << g.logQ2, Q1 = 1 << g.logQ1;
  const int lines = g.nchan * Q1;
  const int nl = std::min(TILE / Q2, lines);
  const unsigned grid = grid_for(lines / nl, g.sms);
  switch (Q2) {
#define CASE(R) case R: k_inv_cols<R><<<grid, NT, smem_bytes<R>(nl), st>>>(in, out, g.logQ1, g.logM, g.logR1, g.logR2, g.nchan, twM, anc, clog, tw); break;
    POND_FOR_R(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_inv_rows(const Geom& g, const float2* buf, float* P, float2* vout, long long vstride,
                            long long vofs, int m_lo, int m_hi, const float2* tw, cudaStream_t st) {
  const int Q2 = 1 << g.logQ2, Q1 = 1 << g.logQ1;
  const int b2 = std::min(TILE / (Q1 * g.nchan), Q2);
  const int nl = g.nchan * b2;
  const unsigned grid = grid_for(Q2 / b2, g.sms);
  const float scale = 1.0f / (float)(1u << g.logM);
  switch (Q1) {
#define CASE(R) case R: k_inv_rows<R><<<grid, NT, smem_bytes<R>(nl), st>>>(buf, P, vout, vstride, vofs, g.logQ2, g.logM, g.nchan, m_lo, m_hi, scale, tw); break;
    POND_FOR_R(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

size_t fold_smem_bytes(int nbins) {
  return (size_t)FOLD_WARPS * nbins * (sizeof(double) + sizeof(int)) + FOLD_WARPS * 32 * sizeof(float);
}

int fold_parts(long long n, long long* chunk) {
  long long c = std::max<long long>(1024, (n + MAX_FOLD_PARTS - 1) / MAX_FOLD_PARTS);
  c = (c + 127) / 128 * 128;
  *chunk = c;
  return (int)((n + c - 1) / c);
}

cudaError_t launch_fold(const float* P, long long n, long long g0, double inc, int nbins, double* psum,
                        int* phits, double* prof_sum, long long* prof_hits, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  long long chunk;
  const int parts = fold_parts(n, &chunk);
  k_fold_partial<<<parts, FOLD_WARPS * 32, fold_smem_bytes(nbins), st>>>(P, n, g0, inc, nbins, chunk, psum, phits);
  k_fold_merge<<<(nbins * 32 + 255) / 256, 256, 0, st>>>(psum, phits, parts, nbins, prof_sum, prof_hits);
  return cudaGetLastError();
}

cudaError_t launch_decimate(const float* P, long long n, long long g0, long long num, long long den,
                            long long j_lo, long long nj, float* T, int* C, long long ring, cudaStream_t st) {
  if (n <= 0 || nj <= 0) return cudaSuccess;
  const long long threads = nj * 32;
  k_decimate<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(P, n, g0, num, den, j_lo, nj, T, C, ring);
  return cudaGetLastError();
}

}  // namespace pond
