// Segment kernels of the coherent-dedispersion path (PONDER Sec. 3.7).
//
// One overlap-save segment of N real int8 samples goes through four FFT passes
// over a spectrum of L = N/2 complex bins (passes.cuh; FP32 instantiations
// here), then fold and decimation:
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

#include "passes.cuh"

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
// about k_a = 2^clog a + 2^(clog-1): phi(k_a) mod 1 in Q0.32, phi'(k_a) and
// phi''(k_a)/2 mod 1 in Q0.64 (so the polynomial up to d^2 is exact mod 1 in
// integer arithmetic), phi'''(k_a)/6 in FP32.  c(f) = alpha f^2 / (f0 + f)
// with alpha = K 1e6 DM / f0^2 (Eq. 4), f = k du - |bw|/2 (upper sideband) or
// |bw|/2 - k du (inverted).  The planner picks clog so that the dropped
// quartic term stays below 1e-9 cycles.
__device__ __forceinline__ unsigned long long frac_q064(double x) {
  const double fr = x - floor(x);                 // in [0, 1), exact in FP64
  const double t = fr * 4294967296.0;             // exact scaling
  const double h = floor(t);
  const long long l = llrint((t - h) * 4294967296.0);
  return ((unsigned long long)h << 32) + (unsigned long long)l;   // a carry from l = 2^32 wraps mod 2^64
}

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
  ChirpAnchor r;
  r.p0 = (unsigned)((unsigned long long)llrint(fr0 * 4294967296.0) & 0xffffffffull);
  r.p1 = frac_q064(phi1);
  r.p2 = frac_q064(phi2);
  r.p3 = (float)phi3;
  r.pad[0] = r.pad[1] = 0u;
  anc[a] = r;
}

// Three-level table for exponents e < 2^24: entry 256 l + j holds
// w^(j 2^(8 l)), w = exp(sign 2 pi i / 2^logn) (FP64 sincospi).
__global__ void k_make_tw3(float2* out, int logn, int sign) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 768) return;
  const long long e = (long long)(i & 255) << (8 * (i >> 8));
  double s, c;
  sincospi(2.0 * sign * (double)e / (double)(1ll << logn), &s, &c);
  out[i] = make_float2((float)c, (float)s);
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

// ---------------------------------------------------------------------------
// Fold (Sec. 3.4 fold thread): deterministic per-warp histograms
// ---------------------------------------------------------------------------

constexpr int FOLD_WARPS = 4;
constexpr int FOLD_U = 4;        // 32-sample groups in flight per warp

// bin(g) = min(floor(frac(g * inc) * nbins), nbins - 1), FP64, correctly rounded.
__device__ __forceinline__ int fold_bin(long long g, double inc, int nbins) {
  const double x = __dmul_rn((double)g, inc);
  const double ph = __dsub_rn(x, floor(x));
  const int b = (int)__dmul_rn(ph, (double)nbins);
  return b < nbins - 1 ? b : nbins - 1;
}

// The bin of g under the fold's phase rule: the constant period, or the
// polynomial phase model (Horner's rule, each FP64 multiply and add rounded
// on its own; bin = min(floor((phi - floor(phi)) nbins), nbins - 1)).
__device__ __forceinline__ int fold_bin(long long g, const FoldPhase& r, int nbins) {
  if (r.nc == 0) return fold_bin(g, r.inc, nbins);
  const double tau = __dsub_rn(__dmul_rn((double)g, r.dt), r.t_ref);
  double x = r.c[r.nc - 1];
  for (int k = r.nc - 2; k >= 0; --k) x = __dadd_rn(__dmul_rn(x, tau), r.c[k]);
  const int b = (int)__dmul_rn(__dsub_rn(x, floor(x)), (double)nbins);
  return b < nbins - 1 ? b : nbins - 1;
}

// Fold channel samples [c0, c1) of P (global index g0 + c) into this warp's
// histogram (FOLD_WARPS warps share the chunk: warp w takes groups of
// 32 * FOLD_U samples w, w + FOLD_WARPS, ...).  Bin b is kept at entry
// (b - b0) mod nbins, so a chunk that spans a short cyclic run of bins starting
// at b0 needs only that run's entries.
template <class Rule>
__device__ __forceinline__ void fold_chunk(const float* __restrict__ P, long long c0, long long c1, long long g0,
                                           const Rule& rule, int nbins, int b0, double* myh, int* myc, float* mybuf) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // FOLD_U groups of 32 samples per warp and iteration: their loads and FP64
  // bin computations are all in flight before the groups are scanned in order
  for (long long base = c0 + (long long)w * 32 * FOLD_U; base < c1; base += FOLD_WARPS * 32 * FOLD_U) {
    float pv[FOLD_U];
    int bv[FOLD_U];
#pragma unroll
    for (int u = 0; u < FOLD_U; ++u) {
      const long long i = base + u * 32 + lane;
      pv[u] = 0.f;
      bv[u] = -1;
      if (i < c1) {
        pv[u] = __ldg(P + i);
        bv[u] = fold_bin(g0 + i, rule, nbins);
      }
    }
#pragma unroll
    for (int u = 0; u < FOLD_U; ++u) {
      const int b = bv[u];
      const bool ok = b >= 0;
      const float p = pv[u];
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
          const int e = b >= b0 ? b - b0 : b - b0 + nbins;
          myh[e] += (double)x;
          myc[e] += last - first + 1;
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
          const int e = b >= b0 ? b - b0 : b - b0 + nbins;
          myh[e] += (double)sum;
          myc[e] += __popc(peers);
        }
      }
      __syncwarp();
    }
  }
}

// Shared-memory layout of the fold kernels: [FOLD_WARPS][nbins] FP64 sums,
// [FOLD_WARPS][nbins] int32 hits, [FOLD_WARPS][32] FP32 staging.
struct FoldSmem {
  double* hsum;
  int* hcnt;
  float* pbuf;
};

__device__ __forceinline__ FoldSmem fold_smem_init(unsigned char* fsm, int nbins, int used) {
  FoldSmem f;
  f.hsum = reinterpret_cast<double*>(fsm);
  f.hcnt = reinterpret_cast<int*>(f.hsum + FOLD_WARPS * nbins);
  f.pbuf = reinterpret_cast<float*>(f.hcnt + FOLD_WARPS * nbins);
  for (int i = threadIdx.x; i < FOLD_WARPS * used; i += blockDim.x) {
    const int k = (i / used) * nbins + i % used;
    f.hsum[k] = 0.0;
    f.hcnt[k] = 0;
  }
  __syncthreads();
  return f;
}

// One CTA per chunk of channel samples: the CTA's histogram (warps added in
// order) is written to row blockIdx.x of the partials.
__global__ void __launch_bounds__(FOLD_WARPS * 32) k_fold_partial(const float* __restrict__ P, long long n,
                                                                  long long g0, double inc, int nbins,
                                                                  long long chunk, double* __restrict__ psum,
                                                                  int* __restrict__ phits) {
  extern __shared__ unsigned char fsm[];
  const FoldSmem f = fold_smem_init(fsm, nbins, nbins);
  const int w = threadIdx.x >> 5;
  const long long c0 = (long long)blockIdx.x * chunk;
  fold_chunk(P, c0, min(n, c0 + chunk), g0, inc, nbins, 0, f.hsum + w * nbins, f.hcnt + w * nbins,
             f.pbuf + w * 32);
  __syncthreads();
  for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
    double s = 0.0;
    int h = 0;
#pragma unroll
    for (int k = 0; k < FOLD_WARPS; ++k) {
      s += f.hsum[k * nbins + b];
      h += f.hcnt[k * nbins + b];
    }
    psum[(size_t)blockIdx.x * nbins + b] = s;
    phits[(size_t)blockIdx.x * nbins + b] = h;
  }
}

__device__ __forceinline__ long long ceil_div_ll(long long a, long long b) { return (a + b - 1) / b; }

// Series samples spanning at most DEC_SPAN channel samples load them together.
constexpr int DEC_SPAN = 16;

// Fold + decimation of one segment's valid span [g0, g0 + n) in one launch.
// CTA b owns the series samples j in [j_lo + b jpc, j_lo + (b+1) jpc) and the
// channel samples they cover: it folds them (its histogram is added to
// partial row b, which accumulates over the segments of the stream and is
// merged when the profile is read) and then sums each of its series samples
// (one thread per j for spans under 64 channel samples, else one warp per j
// with four partial sums).  Every j belongs to one CTA, so no atomics.
template <bool MODEL>
__global__ void __launch_bounds__(FOLD_WARPS * 32) k_fold_dec(const float* __restrict__ P, long long n,
                                                              long long g0, FoldPhase rule, int nbins,
                                                              long long num, long long den, long long j_lo,
                                                              long long nj, long long jpc,
                                                              float* __restrict__ T, int* __restrict__ C,
                                                              long long ring, double* __restrict__ psum,
                                                              long long* __restrict__ phits) {
  extern __shared__ unsigned char fsm[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long ja = j_lo + (long long)blockIdx.x * jpc;
  const long long jb = min(j_lo + nj, ja + jpc);
  const long long ga = max(ceil_div_ll(ja * num, den), g0);
  const long long gb = min(ceil_div_ll(jb * num, den), g0 + n);
  // at the constant period the phase grows with g, so a chunk shorter than one
  // period (with a margin of two bins) covers the cyclic run of bins
  // fold_bin(ga) .. fold_bin(gb - 1); a phase model keeps every bin
  int b0 = 0, used = nbins;
  if (!MODEL && gb > ga && (double)(gb - 1 - ga) * rule.inc < 1.0 - 2.0 / nbins) {
    b0 = fold_bin(ga, rule.inc, nbins);
    const int b1 = fold_bin(gb - 1, rule.inc, nbins);
    used = (b1 >= b0 ? b1 - b0 : b1 - b0 + nbins) + 1;
  }
  const FoldSmem f = fold_smem_init(fsm, nbins, used);
  if constexpr (MODEL)
    fold_chunk(P, ga - g0, gb - g0, g0, rule, nbins, b0, f.hsum + w * nbins, f.hcnt + w * nbins, f.pbuf + w * 32);
  else
    fold_chunk(P, ga - g0, gb - g0, g0, rule.inc, nbins, b0, f.hsum + w * nbins, f.hcnt + w * nbins,
               f.pbuf + w * 32);
  __syncthreads();
  for (int e = threadIdx.x; e < used; e += blockDim.x) {
    double s = 0.0;
    int h = 0;
#pragma unroll
    for (int k = 0; k < FOLD_WARPS; ++k) {
      s += f.hsum[k * nbins + e];
      h += f.hcnt[k * nbins + e];
    }
    const int b = b0 + e < nbins ? b0 + e : b0 + e - nbins;
    psum[(size_t)blockIdx.x * nbins + b] += s;
    phits[(size_t)blockIdx.x * nbins + b] += h;
  }
  if (num < 64 * den) {
    for (long long j = ja + threadIdx.x; j < jb; j += blockDim.x) {
      const long long a = max(ceil_div_ll(j * num, den), g0), e = min(ceil_div_ll((j + 1) * num, den), g0 + n);
      float s = 0.f;
      if (e - a <= DEC_SPAN) {
        // loads issued together, added in sample order
        float v[DEC_SPAN];
#pragma unroll
        for (int i = 0; i < DEC_SPAN; ++i) v[i] = a + i < e ? __ldg(P + (a + i - g0)) : 0.f;
#pragma unroll
        for (int i = 0; i < DEC_SPAN; ++i)
          if (a + i < e) s += v[i];
      } else {
        for (long long g = a; g < e; ++g) s += __ldg(P + (g - g0));
      }
      const long long slot = j % ring;
      T[slot] += s;
      C[slot] += (int)max(e - a, 0ll);
    }
  } else {
    for (long long j = ja + w; j < jb; j += FOLD_WARPS) {
      const long long a = max(ceil_div_ll(j * num, den), g0), e = min(ceil_div_ll((j + 1) * num, den), g0 + n);
      float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
      long long g = a + lane;
      for (; g + 96 < e; g += 128) {
        s0 += __ldg(P + (g - g0));
        s1 += __ldg(P + (g + 32 - g0));
        s2 += __ldg(P + (g + 64 - g0));
        s3 += __ldg(P + (g + 96 - g0));
      }
      if (g < e) s0 += __ldg(P + (g - g0));
      if (g + 32 < e) s1 += __ldg(P + (g + 32 - g0));
      if (g + 64 < e) s2 += __ldg(P + (g + 64 - g0));
      float s = (s0 + s1) + (s2 + s3);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      if (lane == 0) {
        const long long slot = j % ring;
        T[slot] += s;
        C[slot] += (int)max(e - a, 0ll);
      }
    }
  }
}

// A CTA merges 32 consecutive bins: warp y sums parts y, y + 8, y + 16, ... in
// order (lanes read 32 consecutive bins of a part: coalesced), then lane x of
// warp 0 adds the eight warp sums of bin x in a fixed order.  ACC adds the
// result to the profile, otherwise it replaces it.
constexpr int MERGE_WARPS = 8;

template <typename H, bool ACC>
__global__ void __launch_bounds__(MERGE_WARPS * 32) k_fold_merge(const double* __restrict__ psum,
                                                                 const H* __restrict__ phits, int nparts,
                                                                 int nbins, double* __restrict__ prof_sum,
                                                                 long long* __restrict__ prof_hits) {
  __shared__ double ss[MERGE_WARPS][32];
  __shared__ long long sh[MERGE_WARPS][32];
  const int x = threadIdx.x & 31, y = threadIdx.x >> 5;
  const int b = blockIdx.x * 32 + x;
  double s = 0.0;
  long long h = 0;
  if (b < nbins) {
#pragma unroll 4
    for (int k = y; k < nparts; k += MERGE_WARPS) {
      s += __ldg(psum + (size_t)k * nbins + b);
      h += (long long)__ldg(phits + (size_t)k * nbins + b);
    }
  }
  ss[y][x] = s;
  sh[y][x] = h;
  __syncthreads();
  if (y == 0 && b < nbins) {
    double t = 0.0;
    long long c = 0;
#pragma unroll
    for (int k = 0; k < MERGE_WARPS; ++k) {
      t += ss[k][x];
      c += sh[k][x];
    }
    if (ACC) {
      prof_sum[b] += t;
      prof_hits[b] += c;
    } else {
      prof_sum[b] = t;
      prof_hits[b] = c;
    }
  }
}

// ---------------------------------------------------------------------------
// Decimation: T[j] += sum of P[g], floor(g den / num) = j; one warp per j
// ---------------------------------------------------------------------------

// One warp per series sample j (spans of 64 or more channel samples): four
// independent partial sums keep four loads in flight per lane, combined in a
// fixed order, then a fixed xor-tree over the lanes.
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
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
  long long g = ga + lane;
  for (; g + 96 < gb; g += 128) {
    s0 += __ldg(P + (g - g0));
    s1 += __ldg(P + (g + 32 - g0));
    s2 += __ldg(P + (g + 64 - g0));
    s3 += __ldg(P + (g + 96 - g0));
  }
  if (g < gb) s0 += __ldg(P + (g - g0));
  if (g + 32 < gb) s1 += __ldg(P + (g + 32 - g0));
  if (g + 64 < gb) s2 += __ldg(P + (g + 64 - g0));
  float s = (s0 + s1) + (s2 + s3);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) {
    const long long slot = j % ring;
    T[slot] += s;
    C[slot] += (int)max(gb - ga, 0ll);
  }
}

// One thread per series sample j (spans shorter than 64 channel samples): the
// span is summed in index order; neighbouring threads read neighbouring spans.
__global__ void k_decimate_short(const float* __restrict__ P, long long n, long long g0, long long num,
                                 long long den, long long j_lo, long long nj, float* __restrict__ T,
                                 int* __restrict__ C, long long ring) {
  const long long jj = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (jj >= nj) return;
  const long long j = j_lo + jj;
  long long ga = ceil_div_ll(j * num, den), gb = ceil_div_ll((j + 1) * num, den);
  ga = max(ga, g0);
  gb = min(gb, g0 + n);
  float s = 0.f;
  for (long long g = ga; g < gb; ++g) s += __ldg(P + (g - g0));
  const long long slot = j % ring;
  T[slot] += s;
  C[slot] += (int)max(gb - ga, 0ll);
}

// k_decimate_short for the trials of one batched launch: blockIdx.y = trial t,
// reading P + t pstride and adding to series row rows[t].
__global__ void k_decimate_short_multi(const float* __restrict__ P, long long pstride, long long n, long long g0,
                                       long long num, long long den, long long j_lo, long long nj,
                                       float* __restrict__ T, int* __restrict__ C, long long ring,
                                       const int* __restrict__ rows) {
  const long long jj = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (jj >= nj) return;
  const int row = __ldg(rows + blockIdx.y);
  P += blockIdx.y * pstride;
  const long long j = j_lo + jj;
  long long ga = ceil_div_ll(j * num, den), gb = ceil_div_ll((j + 1) * num, den);
  ga = max(ga, g0);
  gb = min(gb, g0 + n);
  float s = 0.f;
  for (long long g = ga; g < gb; ++g) s += __ldg(P + (g - g0));
  const long long slot = (size_t)row * ring + j % ring;
  T[slot] += s;
  C[slot] += (int)max(gb - ga, 0ll);
}

// Chirp table of a batched lane whose DMs are whole multiples of dDM: entry
// k2 R1 + k1 (the spectrum's row layout, bin k = k2 + R2 k1) holds the phase of
// Eq. 4's inverse at bin k for one DM step, sgn dDM c(f_k) mod 1, as a Q0.32
// word (FP64, the same formula as the anchors' phase term).
__global__ void k_make_chirp_table(unsigned* tab, int logR1, int logR2, double du, double half, double f0,
                                   double alpha, int sgn) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (1ll << (logR1 + logR2))) return;
  const long long k2 = i >> logR1, k1 = i & ((1ll << logR1) - 1);
  const double k = (double)(k2 + (k1 << logR2));
  const double f = sgn > 0 ? __dsub_rn(__dmul_rn(k, du), half) : __dsub_rn(half, __dmul_rn(k, du));
  const double g = f0 + f;
  const double phi = sgn * (alpha * f * f / g);
  const double fr = phi - floor(phi);
  tab[i] = (unsigned)((unsigned long long)llrint(fr * 4294967296.0) & 0xffffffffull);
}

// The inverse filter of Eq. 4 per bin as FP32 (cos, -sin) of 2 pi phi(k), in
// the spectrum's row layout (bin k2 + R2 k1 at k2 R1 + k1): phi in FP64 with the
// anchors' formula, reduced mod 1, then FP64 sincospi, rounded once to FP32.
__global__ void k_make_chirp_c64(float2* tab, int logR1, int logR2, double du, double half, double f0, double alpha,
                                 int sgn) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (1ll << (logR1 + logR2))) return;
  const long long k2 = i >> logR1, k1 = i & ((1ll << logR1) - 1);
  const double k = (double)(k2 + (k1 << logR2));
  const double f = sgn > 0 ? __dsub_rn(__dmul_rn(k, du), half) : __dsub_rn(half, __dmul_rn(k, du));
  const double g = f0 + f;
  const double phi = sgn * (alpha * f * f / g);
  double r = phi - floor(phi);
  if (r > 0.5) r -= 1.0;
  double sn, cs;
  sincospi(2.0 * r, &sn, &cs);
  tab[i] = make_float2((float)cs, (float)-sn);
}

// Byte copy between device buffers (any alignment): 16-byte words where both
// sides allow, single bytes otherwise.
__global__ void k_copy_bytes(int8_t* __restrict__ dst, const int8_t* __restrict__ src, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if ((((uintptr_t)dst | (uintptr_t)src) & 15) == 0) {
    const long long n16 = n >> 4;
    for (long long i = i0; i < n16; i += stride)
      reinterpret_cast<uint4*>(dst)[i] = __ldg(reinterpret_cast<const uint4*>(src) + i);
    for (long long i = (n16 << 4) + i0; i < n; i += stride) dst[i] = src[i];
  } else {
    for (long long i = i0; i < n; i += stride) dst[i] = src[i];
  }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------

// Host (mapped, pinned) -> device copy by a few CTAs: each thread keeps four
// 16-byte loads in flight, so 8 CTAs stream host memory (191 GB/s alone, the
// link's 211 GB/s from 16 CTAs on) faster than the passes consume it while
// leaving the other SMs to them.  Both pointers 16-byte aligned.
__global__ void __launch_bounds__(512) k_copy_host(uint4* __restrict__ dst, const uint4* __restrict__ src,
                                                    long long n16) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n16; i += 4 * stride) {
    const uint4 a = __ldcs(src + i), b = __ldcs(src + i + stride), c = __ldcs(src + i + 2 * stride),
                d = __ldcs(src + i + 3 * stride);
    dst[i] = a;
    dst[i + stride] = b;
    dst[i + 2 * stride] = c;
    dst[i + 3 * stride] = d;
  }
  for (; i < n16; i += stride) dst[i] = __ldcs(src + i);
}

cudaError_t launch_copy_host(int8_t* dst, const int8_t* src, long long n, int blocks, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (((((uintptr_t)dst | (uintptr_t)src) & 15) != 0) || (n & 15)) return launch_copy_bytes(dst, src, n, st);
  k_copy_host<<<blocks, 512, 0, st>>>(reinterpret_cast<uint4*>(dst), reinterpret_cast<const uint4*>(src), n >> 4);
  return cudaGetLastError();
}

cudaError_t launch_copy_bytes(int8_t* dst, const int8_t* src, long long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  // at most two CTAs per SM: the copy runs beside segment passes, whose CTAs
  // cannot share an SM with a third resident CTA
  const long long words = std::max(1ll, n >> 4);
  const unsigned blocks = (unsigned)std::min<long long>((words + 255) / 256, 304);
  k_copy_bytes<<<blocks, 256, 0, st>>>(dst, src, n);
  return cudaGetLastError();
}

cudaError_t launch_chirp_c64(float2* tab, const Geom& g, double du, double half, double f0, double alpha, int sgn,
                             cudaStream_t st) {
  const long long n = g.L;
  k_make_chirp_c64<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(tab, g.logR1, g.logR2, du, half, f0, alpha, sgn);
  return cudaGetLastError();
}

cudaError_t launch_chirp_table(unsigned* tab, const Geom& g, double du, double half, double f0, double alpha, int sgn,
                               cudaStream_t st) {
  const long long n = g.L;
  k_make_chirp_table<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(tab, g.logR1, g.logR2, du, half, f0, alpha, sgn);
  return cudaGetLastError();
}

cudaError_t launch_decimate_multi(const float* P, long long pstride, long long n, long long g0, long long num,
                                  long long den, long long j_lo, long long nj, float* T, int* C, long long ring,
                                  const int* rows, int ntr, cudaStream_t st) {
  if (n <= 0 || nj <= 0) return cudaSuccess;
  if (num >= 64 * den) return cudaErrorInvalidValue;   // short spans only (batched plans decimate by a few)
  const dim3 grid((unsigned)((nj + 255) / 256), (unsigned)ntr);
  k_decimate_short_multi<<<grid, 256, 0, st>>>(P, pstride, n, g0, num, den, j_lo, nj, T, C, ring, rows);
  return cudaGetLastError();
}

cudaError_t launch_stage_tw(float2* out, int R, cudaStream_t st) {
  const int n = stage_table_size(R);
  if (n > 0) k_make_stage_tw<<<(n + 255) / 256, 256, 0, st>>>(out, R);
  return cudaGetLastError();
}

int stage_tw_entries(int R) { return stage_table_size(R); }

cudaError_t launch_tw2(float2* lo, float2* hi, int logn, int sign, cudaStream_t st) {
  const long long nhi = logn > TW2_LOG ? (1ll << (logn - TW2_LOG)) : 1;
  const long long n = std::max<long long>(TW2_LO, nhi);
  k_make_tw2<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(lo, hi, logn, sign);
  return cudaGetLastError();
}

cudaError_t launch_tw3(float2* out, int logn, int sign, cudaStream_t st) {
  k_make_tw3<<<3, 256, 0, st>>>(out, logn, sign);
  return cudaGetLastError();
}

cudaError_t launch_tables(ChirpAnchor* anc, long long nanc, int clog, double du, double half,
                          double f0, double alpha, int sgn, cudaStream_t st) {
  k_make_chirp_anchors<<<(unsigned)((nanc + 127) / 128), 128, 0, st>>>(anc, nanc, clog, du, half, f0, alpha, sgn);
  return cudaGetLastError();
}

// Fused schedule: F2f for R1 = 512..4096 with J = 64, Ic for R2 = 16..2048.
#define POND_FUSED_R1(X) X(512) X(1024) X(2048) X(4096)
#define POND_FUSED_R2(X) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048)

bool fused_geometry(const Geom& g) {
  return g.logM - g.logR2 == 6 && g.logR1 >= 9 && g.logR1 <= 12 && g.logR2 >= 4 && g.logR2 <= 11;
}

namespace {
size_t smem_fwd_rows_inv(int R1, int nl) {
  return ((size_t)TW3_SN + stage_table_size(R1) + stage_table_size(FUSED_J) + (size_t)nl * FUSED_J +
          (size_t)nl * (R1 + R1 / 16)) * sizeof(float2);
}
template <int R2>
size_t smem_inv_cols_det(int nl) {
  return ((size_t)stage_table_size(R2) + (size_t)nl * col_stride<R2>()) * sizeof(float2);
}
}  // namespace

cudaError_t launch_fwd_rows_inv(const Geom& g, const float2* in, float2* out, const float2* tw3L, Tw2 tw2L,
                                const float2* tw, const float2* twJ, const ChirpAnchor* anc, int clog,
                                const float2* ctab, cudaStream_t st) {
  const int R2 = 1 << g.logR2, R1 = 1 << g.logR1;
  const int nl = std::min(TILE / R1, R2);
  const unsigned grid = (unsigned)(R2 / nl);
  switch (R1) {
#define CASE(R)                                                                                             \
  case R:                                                                                                   \
    if (ctab)                                                                                               \
      k_fwd_rows_inv<R, FUSED_J, true><<<grid, NT, smem_fwd_rows_inv(R, nl), st>>>(                        \
          in, out, g.logR2, g.logL, tw3L, tw2L, tw, twJ, anc, clog, ctab);                                  \
    else                                                                                                    \
      k_fwd_rows_inv<R, FUSED_J, false><<<grid, NT, smem_fwd_rows_inv(R, nl), st>>>(                       \
          in, out, g.logR2, g.logL, tw3L, tw2L, tw, twJ, anc, clog, ctab);                                  \
    break;
    POND_FUSED_R1(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

namespace {
size_t smem_inv_rows_chirp(int R1, int nl) {
  return ((size_t)TW3_SN + stage_table_size(FUSED_J) + (size_t)nl * FUSED_J + (size_t)nl * (R1 + R1 / 16)) *
         sizeof(float2);
}
// k_inv_rows_chirp_res: the row pass's tables and tile plus the resident rows
// (8 bytes per bin) and their table words (4 bytes per bin), in the tile's layout
size_t smem_inv_rows_res(int R1, int nl) {
  return smem_inv_rows_chirp(R1, nl) + (size_t)nl * (R1 + R1 / 16) * (sizeof(float2) + sizeof(unsigned));
}
}  // namespace

cudaError_t launch_inv_rows_chirp(const Geom& g, const float2* in, float2* out, const float2* tw3L, const float2* twJ,
                                  const ChirpAnchor* anc, int clog, cudaStream_t st) {
  const int R2 = 1 << g.logR2, R1 = 1 << g.logR1;
  const int nl = std::min(TILE / R1, R2);
  const unsigned grid = (unsigned)(R2 / nl);
  switch (R1) {
#define CASE(R) case R: k_inv_rows_chirp<R, FUSED_J><<<grid, NT, smem_inv_rows_chirp(R, nl), st>>>(in, out, g.logR2, tw3L, twJ, anc, clog); break;
    POND_FUSED_R1(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_inv_rows_chirp_multi(const Geom& g, const float2* in, float2* out, int ntr, const float2* tw3L,
                                        const float2* twJ, MultiChirp mc, bool table, cudaStream_t st) {
  const int R2 = 1 << g.logR2, R1 = 1 << g.logR1;
  const int nl = std::min(TILE / R1, R2);
  if (ntr < 1) return cudaErrorInvalidValue;
  // table form: one CTA per row tile runs every trial; anchor form: one CTA
  // per (trial, row tile)
  const unsigned tiles = (unsigned)(R2 / nl);
  switch (R1) {
#define CASE(R)                                                                                             \
  case R:                                                                                                   \
    if (table)                                                                                              \
      k_inv_rows_chirp_res<R, FUSED_J><<<tiles, NT, smem_inv_rows_res(R, nl), st>>>(in, out, g.L, g.logR2,  \
                                                                                    tw3L, twJ, mc, ntr);    \
    else                                                                                                    \
      k_inv_rows_chirp_multi<R, FUSED_J><<<dim3((unsigned)ntr, tiles), NT, smem_inv_rows_chirp(R, nl), st>>>( \
          in, out, g.L, g.logR2, tw3L, twJ, mc);                                                            \
    break;
    POND_FUSED_R1(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

int fused_groups(const Geom& g) {
  const int nl = std::min(TILE >> g.logR2, g.nchan);
  return g.nchan / nl;
}

cudaError_t launch_inv_cols_det(const Geom& g, const float2* in, float* P, float* part, int* cnt, float2* vout,
                                long long vstride, long long vofs, int m_lo, int m_hi, const float2* tw,
                                cudaStream_t st, int ntr) {
  const int R2 = 1 << g.logR2, R1 = 1 << g.logR1;
  const int nl = std::min(TILE / R2, g.nchan);
  const dim3 grid((unsigned)(R1 / nl), (unsigned)ntr);
  const float scale = 1.0f / (float)(1u << g.logM);
  const int lognch = g.logR1 - (g.logM - g.logR2);
  // several trials: each has its own L-element input, M-element P, partials and tickets
  const TrialStride ts = ntr > 1 ? TrialStride{g.L, g.M, (long long)fused_groups(g) * g.M, FUSED_J}
                                 : TrialStride{0, 0, 0, 0};
  switch (R2) {
#define CASE(R) case R: k_inv_cols_det<R><<<grid, NT, smem_inv_cols_det<R>(nl), st>>>(in, P, part, cnt, vout, vstride, vofs, g.logR1, lognch, g.logM - g.logR2, m_lo, m_hi, scale, tw, ts); break;
    POND_FUSED_R2(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t set_kernel_attributes() {
  cudaError_t e = set_attributes_t<false>();
#define SET_F(R) \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fwd_rows_inv<R, FUSED_J, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_fwd_rows_inv(R, TILE / R)); \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fwd_rows_inv<R, FUSED_J, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_fwd_rows_inv(R, TILE / R));
  POND_FUSED_R1(SET_F)
#undef SET_F
#define SET_I(R) \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_inv_rows_chirp<R, FUSED_J>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_inv_rows_chirp(R, TILE / R));
  POND_FUSED_R1(SET_I)
#undef SET_I
#define SET_M(R)                                                                                       \
  if (e == cudaSuccess)                                                                                \
    e = cudaFuncSetAttribute(k_inv_rows_chirp_res<R, FUSED_J>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)smem_inv_rows_res(R, TILE / R));                                        \
  if (e == cudaSuccess)                                                                                \
    e = cudaFuncSetAttribute(k_inv_rows_chirp_multi<R, FUSED_J>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)smem_inv_rows_chirp(R, TILE / R));
  POND_FUSED_R1(SET_M)
#undef SET_M
#define SET_C(R) \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_inv_cols_det<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_inv_cols_det<R>(TILE / R));
  POND_FUSED_R2(SET_C)
#undef SET_C
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fold_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, fold_smem_bytes(MAX_NBINS));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fold_dec<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, fold_smem_bytes(MAX_NBINS));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_fold_dec<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, fold_smem_bytes(MAX_NBINS));
  return e;
}

// The pass launchers pick the FP32 or the tensor-core instantiation.
cudaError_t launch_fwd_cols(const Geom& g, SegIn in, float2* out, const float2* tw, cudaStream_t st) {
  return g.tc_terms ? launch_fwd_cols_tc(g, in, out, tw, st) : launch_fwd_cols_t<false>(g, in, out, tw, st);
}

cudaError_t launch_fwd_rows(const Geom& g, const float2* in, float2* out, const float2* tw3L, Tw2 tw2L, const float2* tw,
                            cudaStream_t st) {
  return g.tc_terms ? launch_fwd_rows_tc(g, in, out, tw3L, tw2L, tw, st)
                    : launch_fwd_rows_t<false>(g, in, out, tw3L, tw2L, tw, st);
}

cudaError_t launch_inv_cols(const Geom& g, const float2* in, float2* out, const ChirpAnchor* anc,
                            int clog, const float2* tw, cudaStream_t st) {
  return g.tc_terms ? launch_inv_cols_tc(g, in, out, anc, clog, tw, st)
                    : launch_inv_cols_t<false>(g, in, out, anc, clog, tw, st);
}

cudaError_t launch_inv_rows(const Geom& g, const float2* buf, float* P, float2* vout, long long vstride,
                            long long vofs, int m_lo, int m_hi, const float2* tw3M, const float2* tw,
                               cudaStream_t st) {
  return g.tc_terms ? launch_inv_rows_tc(g, buf, P, vout, vstride, vofs, m_lo, m_hi, tw3M, tw, st)
                    : launch_inv_rows_t<false>(g, buf, P, vout, vstride, vofs, m_lo, m_hi, tw3M, tw, st);
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
  k_fold_merge<int, true><<<(nbins + 31) / 32, MERGE_WARPS * 32, 0, st>>>(psum, phits, parts, nbins, prof_sum,
                                                                          prof_hits);
  return cudaGetLastError();
}

cudaError_t launch_fold_dec(const float* P, long long n, long long g0, const FoldPhase& ph, int nbins, long long num,
                            long long den, long long j_lo, long long nj, float* T, int* C, long long ring,
                            double* psum, long long* phits, cudaStream_t st) {
  if (n <= 0 || nj <= 0) return cudaSuccess;
  // whole series samples per CTA: at least FOLD_MIN_SAMPLES channel samples
  // each, at most MAX_FOLD_PARTS CTAs.  The fold runs beside the passes of the
  // next segments, and each resident fold CTA holds registers a pass CTA would
  // use: a few long-lived CTAs displace less than many short ones (full rate,
  // 105k samples per segment, CTAs: 304: 112.5k, 152: 113.9k, 76: 114.8k,
  // 38: 114.8k, 19: 114.0k Msamples/s), while segments of a million samples
  // (one sub-channel) still spread over every SM.
  constexpr long long FOLD_MIN_SAMPLES = 1400;
  const long long per_j = std::max(1ll, num / den);
  long long jpc = std::max((nj + MAX_FOLD_PARTS - 1) / MAX_FOLD_PARTS, (FOLD_MIN_SAMPLES + per_j - 1) / per_j);
  jpc = std::min(jpc, nj);
  const unsigned parts = (unsigned)((nj + jpc - 1) / jpc);
  if (ph.nc > 0)
    k_fold_dec<true><<<parts, FOLD_WARPS * 32, fold_smem_bytes(nbins), st>>>(P, n, g0, ph, nbins, num, den, j_lo, nj,
                                                                           jpc, T, C, ring, psum, phits);
  else
    k_fold_dec<false><<<parts, FOLD_WARPS * 32, fold_smem_bytes(nbins), st>>>(P, n, g0, ph, nbins, num, den, j_lo, nj,
                                                                            jpc, T, C, ring, psum, phits);
  return cudaGetLastError();
}

cudaError_t launch_fold_snapshot(const double* psum, const long long* phits, int nbins, double* prof_sum,
                                 long long* prof_hits, cudaStream_t st) {
  k_fold_merge<long long, false><<<(nbins + 31) / 32, MERGE_WARPS * 32, 0, st>>>(psum, phits, MAX_FOLD_PARTS, nbins,
                                                                                prof_sum, prof_hits);
  return cudaGetLastError();
}

cudaError_t launch_decimate(const float* P, long long n, long long g0, long long num, long long den,
                            long long j_lo, long long nj, float* T, int* C, long long ring, cudaStream_t st) {
  if (n <= 0 || nj <= 0) return cudaSuccess;
  if (num < 64 * den) {   // fewer than 64 channel samples per series sample
    k_decimate_short<<<(unsigned)((nj + 255) / 256), 256, 0, st>>>(P, n, g0, num, den, j_lo, nj, T, C, ring);
  } else {
    const long long threads = nj * 32;
    k_decimate<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(P, n, g0, num, den, j_lo, nj, T, C, ring);
  }
  return cudaGetLastError();
}

}  // namespace pond
