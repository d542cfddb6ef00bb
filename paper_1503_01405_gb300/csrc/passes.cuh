// The four FFT passes of a segment (PONDER Sec. 3.7), templated on the line
// length and on the arithmetic of their radix-16 stages: FP32 butterflies
// (TC = false) or split-BF16 16-point DFT-matrix products on the tensor cores
// (TC = true, tc_dft.cuh).  kernels.cu instantiates the FP32 form and
// kernels_tc.cu the tensor-core form; both share everything else.
//
//  F1 k_fwd_cols   : unpack z[n] = x[2n] + i x[2n+1]; length-R2 FFTs down the
//                    R1 columns n1 of z viewed as [R2][R1]; store in place.
//  F2 k_fwd_rows   : multiply row k2 by exp(-2 pi i n1 k2 / L) as it is loaded,
//                    length-R1 FFTs along the rows (Z[k2 + R2 k1]); rows k2
//                    and R2-k2 share a CTA so the real-input split
//                    X[k] = (Z[k] + Z*[L-k])/2 - i e^{-i pi k/L} (Z[k] - Z*[L-k])/2
//                    is local; store X[k] at row k2, column k1.
//  I1 k_inv_cols   : per sub-channel c (bins cM..cM+M-1): multiply each bin by
//                    the inverse ISM response (Eq. 4) as it is loaded, inverse
//                    length-Q2 FFTs down the Q1 columns j1; store in natural order.
//  I2 k_inv_rows   : multiply row m2 by exp(+2 pi i j1 m2 / M) as it is loaded,
//                    inverse length-Q1 FFTs along rows m2 for all sub-channels
//                    of the same m2 in one CTA: v_c[m2 + Q2 m1] / M, keep the
//                    valid span n_past <= m < M - n_fut, detect |v|^2 and sum
//                    over sub-channels into P (and optionally store v).
//
//  Single-trial FP32 plans with J = M / R2 = 64 run three passes instead
//  (F1, F2f, Ic): F2f k_fwd_rows_inv is F2 followed, in the same tile, by the
//  chirp and the length-J first factor of every sub-channel's inverse; Ic
//  k_inv_cols_det takes the remaining length-R2 factor down the columns, then
//  discards, detects and sums over sub-channels.  F1 is shared.
//  Table lookups (twiddles, chirp anchors) sit in the load phases, where their
//  latency overlaps the tile's own loads; I1 stages its CTA's chirp anchors in
//  shared memory when they are few (one anchor covers up to 2^15 bins).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "fft_block.cuh"
#include "pond_internal.h"
#include "tc_dft.cuh"

namespace pond {

// exp(-2 pi i phi(k)) from the anchor table: the phase mod 1 is exact to
// < 1e-7 cycles (FP64-built fixed point, see k_make_chirp_anchors); the final
// sine and cosine of 2 pi r, |r| <= 1/2 + 1e-3, use the hardware approximation
// (absolute error about 4e-7 on [-pi, pi]).
__device__ __forceinline__ float2 chirp_from(const ChirpAnchor& a, int clog, unsigned k) {
  const int d = (int)(k & ((1u << clog) - 1)) - (int)((1u << clog) >> 1);   // |d| <= 2^14
  const unsigned dd = (unsigned)(d * d);
  // top 32 bits of phi0 + phi1 d + phi2 d^2 mod 1 in Q0.64: the high words
  // multiply mod 2^32, the low words contribute their products' high words
  // (each truncation loses < 2^-32 cycles)
  const unsigned p1h = (unsigned)(a.p1 >> 32), p1l = (unsigned)a.p1;
  const unsigned p2h = (unsigned)(a.p2 >> 32), p2l = (unsigned)a.p2;
  const unsigned u = a.p0 + p1h * (unsigned)d + (unsigned)(((long long)p1l * d) >> 32) + p2h * dd +
                     __umulhi(p2l, dd);
  const float df = (float)d;
  float r = (float)(int)u * 2.3283064365386963e-10f;   // 2^-32
  r = fmaf(a.p3 * df, df * df, r);
  float s, c;
  __sincosf(6.2831853071795865f * r, &s, &c);
  return make_float2(c, -s);
}

// Chirp anchors an I1 CTA stages in shared memory (16 KiB) before its lookups.
constexpr int ANC_STAGE = 512;
constexpr int ANC_BYTES = ANC_STAGE * (int)sizeof(ChirpAnchor);


__device__ __forceinline__ float2 tw2(const Tw2& t, unsigned e) {
  return cmul(__ldg(t.hi + (e >> TW2_LOG)), __ldg(t.lo + (e & (TW2_LO - 1))));
}

constexpr int EPT = TILE / NT;   // tile elements per thread

// Element maps of the load and store phases.  A thread visits
// idx = threadIdx.x + u NT (u < NU, NT a power of two), and each map f used
// there (global offset, bin number, shared-memory slot) is a sum of terms
// that each depend on one bit field of idx, with disjoint fields placed at
// disjoint bits or (the padded slot) scaled linearly; so f is additive over
// disjoint bits: f(a | b) = f(a) + f(b) - f(0).  Lin keeps f(threadIdx.x) and
// the warp-uniform weights f(NT 2^b) - f(0) of the bits b of u: f at an
// unrolled u is then one add of a uniform sum.
template <int NU>
struct Lin {
  static constexpr int NB = ilog2c(NU);
  unsigned base;
  unsigned w[NB > 0 ? NB : 1];
  template <class F>
  __device__ __forceinline__ explicit Lin(F f) {
    const unsigned f0 = f(0u);
    base = f((unsigned)threadIdx.x);
#pragma unroll
    for (int b = 0; b < NB; ++b) w[b] = f((unsigned)NT << b) - f0;
  }
  __device__ __forceinline__ unsigned operator()(int u) const {
    unsigned o = 0;
#pragma unroll
    for (int b = 0; b < NB; ++b)
      if ((u >> b) & 1) o += w[b];
    return base + o;
  }
};

// Per-trial strides (elements) of a column pass launched over several trials
// (blockIdx.y = trial); all zero for a single trial.
struct TrialStride {
  long long in, P, part;
  int cnt;
};

// Three-level table of w^e, e < 2^24, held in shared memory by F2 and I2:
// w^e = t0[e0] t1[e1] t2[e2], e = e0 + 2^8 e1 + 2^16 e2 (each level built in
// FP64 on the device; two FP32 products).  In shared memory level 0 is padded
// by one entry every 16 (entry e0 at e0 + e0/16) so that lanes whose
// exponents step by a multiple of 16 still fall in different banks.
constexpr int TW3_N = 768;                 // global table: three levels of 256
constexpr int TW3_SN = 784;                // shared copy: padded level 0 (272) + 512
constexpr int TW3_BYTES = TW3_SN * (int)sizeof(float2);
__device__ __forceinline__ void load_tw3(float2* st, const float2* __restrict__ g) {
  for (int i = threadIdx.x; i < TW3_N; i += blockDim.x) st[i < 256 ? i + (i >> 4) : i + 16] = __ldg(g + i);
}
__device__ __forceinline__ float2 tw3(const float2* t, unsigned e) {
  const unsigned e0 = e & 255u;
  return cmul(cmul(t[e0 + (e0 >> 4)], t[272 + ((e >> 8) & 255u)]), t[528 + (e >> 16)]);
}


// Offsets into the segment buffers are 32-bit: every buffer holds L <= 2^24
// elements (nfft <= 2^25).

// Tile entries (float2) a pass allocates for nl lines of length R.  The
// tensor-core form pads its tile so that the CTA's shared memory (tables +
// tile + extras) is at least tc::MIN_SMEM_BYTES: then at most two CTAs share
// an SM and their 2 x 256 TMEM columns always fit.
template <int R, bool TC, int LS = line_stride(R)>
__host__ __device__ constexpr int tile_f2(int nl) {
  return TC ? (nl * LS > tc::MIN_TILE_F2 - stage_table_size(R) ? nl * LS : tc::MIN_TILE_F2 - stage_table_size(R))
            : nl * LS;
}

// Line stride of the column passes (F1, I1): their epilogues read TILE/R lines x
// (16 R / TILE) consecutive elements per half-warp, which fall in distinct
// banks when the stride is 16 R / TILE (mod 16) in 8-byte words.
template <int R>
__host__ __device__ constexpr int col_stride() {
  return R + R / 16 + (TILE / R >= 16 ? 1 : 16 / (TILE / R));
}

// ---------------------------------------------------------------------------
// F1: unpack + column FFTs of the forward transform
// ---------------------------------------------------------------------------

// Real sample m of the segment (one byte, or the sum of an N / S pair).
__device__ __forceinline__ float sample_at(const SegIn& in, long long m) {
  long long r = m * in.ch;
  float x = 0.f;
  for (int c = 0; c < in.ch; ++c, ++r) {
    if (r < in.a_len) x += (float)in.a[r];
    else if (r - in.a_len < in.b_len) x += (float)in.b[r - in.a_len];
  }
  return x;
}

// Unaligned runs or N / S pairs: element (b, n2) of the tile sample by sample
// (rare; out of line so that the aligned load paths keep their registers).
template <int LSTR>
__device__ __noinline__ void f1_load_any(const SegIn in, float2* sm, int n1_0, int nl, int lognl, int logR1,
                                         int tot) {
  for (int idx = threadIdx.x; idx < tot; idx += NT) {
    const int n2 = idx >> lognl, b = idx & (nl - 1);
    const long long q = (long long)(n1_0 + b) + ((long long)n2 << logR1);
    sm[pidx(b, n2, LSTR)] = make_float2(sample_at(in, 2 * q), sample_at(in, 2 * q + 1));
  }
}

// Complex sample q = n1 + R1 n2 of z straight from global memory: one int8 pair
// x[2q], x[2q + 1] (CH 1, 2-byte load), or the two halves' pairs of both real
// samples added in phase (CH 2, 4-byte load N S N S).  Offsets are multiples of
// 2 CH and both runs' lengths multiples of 2 CH, so no load straddles a run or
// passes its end; past both runs the sample is zero.
template <int CH>
__device__ __forceinline__ float2 f1_pair(const SegIn& in, long long q) {
  const long long r = 2ll * CH * q;
  if constexpr (CH == 1) {
    unsigned short w = 0;
    if (r < in.a_len) w = __ldg(reinterpret_cast<const unsigned short*>(in.a + r));
    else if (r - in.a_len < in.b_len) w = __ldg(reinterpret_cast<const unsigned short*>(in.b + (r - in.a_len)));
    return make_float2((float)(signed char)(w & 0xff), (float)(signed char)(w >> 8));
  } else {
    unsigned w = 0;
    if (r < in.a_len) w = __ldg(reinterpret_cast<const unsigned*>(in.a + r));
    else if (r - in.a_len < in.b_len) w = __ldg(reinterpret_cast<const unsigned*>(in.b + (r - in.a_len)));
    return make_float2((float)((int)(signed char)(w & 0xff) + (int)(signed char)((w >> 8) & 0xff)),
                       (float)((int)(signed char)((w >> 16) & 0xff) + (int)(signed char)(w >> 24)));
  }
}

// z viewed as [R2][R1] (z[n1 + R1 n2]); a CTA transforms nl adjacent columns n1
// and stores them in place (the twiddle exp(-2 pi i n1 k2 / L) is F2's).
template <int R2, bool TC>
__global__ void __launch_bounds__(NT, 2) k_fwd_cols(SegIn in, float2* __restrict__ out, int logR1,
                                                    const float2* __restrict__ tw, TcArgs tca) {
  extern __shared__ float2 smem[];
  float2* stw = smem;
  float2* sm = smem + stage_table_size(R2);
  constexpr int LSTR = col_stride<R2>();
  const int R1 = 1 << logR1;
  const int nl = min(TILE / R2, R1);
  const int lognl = __ffs(nl) - 1;
  const int tot = nl * R2;
  load_twiddles<R2>(stw, tw);
  tc::Ctx tcc;
  if constexpr (TC) tc::setup(tcc, sm, tile_f2<R2, TC, LSTR>(nl), tca);
  const int tile = blockIdx.x;
  const int n1_0 = tile * nl;
  // every CTA reads a column slice of every row, so the first F1PF_CTAS CTAs
  // ask L2 for the whole segment (its carried and new runs), a 1/F1PF_CTAS
  // share each, before the strided loads of the first wave arrive (full rate:
  // 111.2k -> 112.8k Msamples/s)
  constexpr int F1PF_CTAS = 64;
  if (threadIdx.x == 0 && tile < F1PF_CTAS && gridDim.x >= F1PF_CTAS) {
    const long long pa = (in.a_len + F1PF_CTAS - 1) / F1PF_CTAS, pb = (in.b_len + F1PF_CTAS - 1) / F1PF_CTAS;
    if (in.a_len > 0) prefetch_range(in.a, min(in.a_len, tile * pa), min(in.a_len, (tile + 1) * pa));
    if (in.b_len > 0) prefetch_range(in.b, min(in.b_len, tile * pb), min(in.b_len, (tile + 1) * pb));
  }
  // FP32 form, R2 >= 512, aligned runs: the first radix-16 stage takes its inputs
  // straight from global memory (butterfly t of column b, columns fastest: a warp
  // reads the nl columns of 8 rows per load) and the stages after it start from
  // LS = 16; the unpack's shared-memory round trip and a barrier go away
  const bool direct1 = !TC && R2 >= 512 && (in.vec8 || in.pair4);
  if (direct1) {
    constexpr int NB = R2 / 16;
    const int b = (int)threadIdx.x & (nl - 1), t = (int)threadIdx.x >> lognl;
    if (t < NB) {
      float2 v[16];
      const long long q0 = (long long)(n1_0 + b) + ((long long)t << logR1);
      if (in.ch == 1) {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = f1_pair<1>(in, q0 + ((long long)(NB * j) << logR1));
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = f1_pair<2>(in, q0 + ((long long)(NB * j) << logR1));
      }
      Dft<16, false>::run(v);
      float2* dst = sm + b * LSTR + pidx(0, 16 * t, 0);    // element 16 t + j
#pragma unroll
      for (int j = 0; j < 16; ++j) dst[j] = v[j];
    }
  } else if (in.vec8) {
    // 8-byte loads: 4 consecutive columns of one row per load (runs 8-aligned)
    constexpr int CPT = EPT / 4;
    const int logq = lognl - 2;            // chunks per row = nl / 4
    const unsigned qm = (unsigned)(nl >> 2) - 1;
    // chunk c: row n2 = c / (nl/4), columns b0..b0+3 with b0 = 4 (c mod nl/4);
    // int8 offset 2 (n1_0 + b0 + n2 R1), shared slot of (b0, n2)
    const Lin<CPT> xofs([&](unsigned c) { return 2u * ((unsigned)n1_0 + ((c & qm) << 2) + ((c >> logq) << logR1)); });
    const Lin<CPT> slot([&](unsigned c) { return (unsigned)pidx((int)((c & qm) << 2), (int)(c >> logq), LSTR); });
    uint2 w[CPT];
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
      if ((int)threadIdx.x + u * NT < tot / 4) {
        const long long r = xofs(u);
        if (r < in.a_len) w[u] = __ldg(reinterpret_cast<const uint2*>(in.a + r));
        else if (r - in.a_len < in.b_len) w[u] = __ldg(reinterpret_cast<const uint2*>(in.b + (r - in.a_len)));
        else w[u] = make_uint2(0u, 0u);
      }
    }
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
      if ((int)threadIdx.x + u * NT < tot / 4) {
        const unsigned lo = w[u].x, hi = w[u].y;
        float2* p = sm + slot(u);
        p[0] = make_float2((float)(signed char)(lo & 0xff), (float)(signed char)((lo >> 8) & 0xff));
        p[LSTR] = make_float2((float)(signed char)((lo >> 16) & 0xff), (float)(signed char)(lo >> 24));
        p[2 * LSTR] = make_float2((float)(signed char)(hi & 0xff), (float)(signed char)((hi >> 8) & 0xff));
        p[3 * LSTR] = make_float2((float)(signed char)((hi >> 16) & 0xff), (float)(signed char)(hi >> 24));
      }
    }
  } else {
    f1_load_any<LSTR>(in, sm, n1_0, nl, lognl, logR1, tot);
  }
  __syncthreads();
  if constexpr (!TC && R2 >= 512) {
    // the last stage (LS 256, radix RL) stores its outputs X[t + 256 j] straight
    // to global memory: butterflies go lines first, so a warp's stores are the
    // nl columns of consecutive rows (32-byte runs) and its loads fall in
    // distinct banks (line stride 16 R2 / TILE mod 16)
    constexpr int RL = R2 / 256, BPTL = 16 / RL;
    if (direct1) StagesUntil<R2, 16, false, LSTR, 256>::run(sm, nl, stw);
    else StagesUntil<R2, 1, false, LSTR, 256>::run(sm, nl, stw);
    const float2* tws = stw + stage_table_offset(R2, 256);
#pragma unroll
    for (int q = 0; q < BPTL; ++q) {
      const int bf = (int)threadIdx.x + q * NT;
      if (bf < nl * 256) {
        const int b = bf & (nl - 1), t = bf >> lognl;
        const float2* src = sm + b * LSTR + t + (t >> 4);
        float2 u[RL];
#pragma unroll
        for (int j = 0; j < RL; ++j) u[j] = src[j * (256 + 16)];   // element t + 256 j
#pragma unroll
        for (int j = 1; j < RL; ++j) u[j] = cmul(u[j], tws[(j - 1) * 256 + t]);
        Dft<RL, false>::run(u);
#pragma unroll
        for (int j = 0; j < RL; ++j) out[(unsigned)(n1_0 + b) + ((unsigned)(t + 256 * j) << logR1)] = u[j];
      }
    }
    return;
  }
  fft_lines<R2, false, TC, LSTR>(sm, nl, stw, &tcc);
  if constexpr (TC) tc::teardown(tcc);
  // neighbouring threads take the nl columns of one row, then the next rows:
  // each warp store fills whole 32-byte sectors
  const Lin<EPT> oofs([&](unsigned idx) { return (unsigned)n1_0 + (idx & (nl - 1)) + ((idx >> lognl) << logR1); });
  const Lin<EPT> oslot([&](unsigned idx) { return (unsigned)pidx((int)(idx & (nl - 1)), (int)(idx >> lognl), LSTR); });
#pragma unroll
  for (int u = 0; u < EPT; ++u)
    if ((int)threadIdx.x + u * NT < tot) out[oofs(u)] = sm[oslot(u)];
}

// ---------------------------------------------------------------------------
// F2: row FFTs + real-input split
// ---------------------------------------------------------------------------

// Row k2 of the column-transformed z holds, after a length-R1 FFT, Z[k2 + R2 k1].
// Rows k2 and R2-k2 share a CTA (row 0 and row R2/2 pair with themselves) so that
// X[k] can be formed from Z[k] and Z[L-k].  Slot s < np of tile q0 np is row
// q0 + s, slot np + t its partner.
__device__ __forceinline__ int f2_line(int slot, int q0, int np, int R2) {
  if (slot < np) return q0 + slot;
  const int t = slot - np;
  if (q0 + t == 0) return R2 >> 1;          // row R2/2 pairs with itself
  return R2 - (q0 + t);
}

// Load the tile's rows (tot = 2 np R1 elements) into sm (line stride LSTR),
// each element scaled by w^{n1 k2}, w = exp(-2 pi i / L), once st3 (being
// filled by the caller) is in: 16-byte loads of columns n1, n1 + 1.
template <int R1, int LSTR>
__device__ __forceinline__ void f2_load(const float2* __restrict__ in, float2* sm, const float2* st3, int q0, int np,
                                        int R2, int tot) {
  constexpr int LOGR1 = ilog2c(R1);
  const float4* in4 = reinterpret_cast<const float4*>(in);
  constexpr int H = EPT / 2;
  float4 r[H];
  // with R1 >= 2 NT the slot of a load is fixed by u: (2 u NT) / R1
  auto slot_of = [&](int u, int idx) { return R1 >= 2 * NT ? (2 * u * NT) >> LOGR1 : idx >> LOGR1; };
  int rows[H];
#pragma unroll
  for (int u = 0; u < H; ++u) {
    const int idx = 2 * (threadIdx.x + u * NT);
    if (R1 >= 2 * NT && u > 0 && slot_of(u, idx) == slot_of(u - 1, idx)) rows[u] = rows[u - 1];
    else rows[u] = f2_line(slot_of(u, idx), q0, np, R2);
    if (idx < tot) {
      const unsigned k2 = (unsigned)rows[u], n1 = (unsigned)(idx & (R1 - 1));
      r[u] = __ldg(in4 + (((k2 << LOGR1) + n1) >> 1));
    }
  }
  __syncthreads();   // st3 filled
  // UPS consecutive loads of a thread fall in one row, n1 apart by 2 NT: there
  // w^{n1 k2} advances by one product with w^{2 NT k2} (at most UPS - 1 steps)
  // and w^{(n1+1) k2} = w^{n1 k2} w^{k2}
  constexpr int UPS = R1 / (2 * NT) > 1 ? R1 / (2 * NT) : 1;
  float2 wa = make_float2(1.f, 0.f), wk = wa, ws = wa;
#pragma unroll
  for (int u = 0; u < H; ++u) {
    const int idx = 2 * (threadIdx.x + u * NT);
    if (idx < tot) {
      const int slot = slot_of(u, idx);
      const unsigned k2 = (unsigned)rows[u], n1 = (unsigned)(idx & (R1 - 1));
      float2 wb;
      if constexpr (UPS > 1) {
        if (u % UPS == 0) {
          wk = tw3(st3, k2);
          ws = tw3(st3, (unsigned)(2 * NT) * k2);
          wa = tw3(st3, n1 * k2);
        } else {
          wa = cmul(wa, ws);
        }
        wb = cmul(wa, wk);
      } else {
        wa = tw3(st3, n1 * k2);
        wb = tw3(st3, (n1 + 1) * k2);
      }
      float2* p = sm + pidx(slot, (int)n1, LSTR);   // n1 even: no pad between the two
      p[0] = cmul(make_float2(r[u].x, r[u].y), wa);
      p[1] = cmul(make_float2(r[u].z, r[u].w), wb);
    }
  }
}

// F2's first radix-16 stage straight from global memory: butterfly t of line
// `slot` (one per thread: nl R1 / 16 <= NT) reads x[t + NB j], j < 16, which
// consecutive lanes load contiguously, scales element n1 = t + NB j of row k2 by
// w^{n1 k2} (direct every fourth j, else one step by w^{NB k2}), and writes its
// outputs to 16 t + j as the Stockham stage would.  Waits for st3 (being filled
// by the caller); R1 >= 256.
template <int R1, int LSTR>
__device__ __forceinline__ void f2_stage1(const float2* __restrict__ in, float2* sm, const float2* st3, int q0,
                                          int np, int R2, int nl) {
  static_assert(R1 >= 256, "radix-16 first stage with at least 16 butterflies per line");
  constexpr int NB = R1 / 16, LOGNB = ilog2c(NB), LOGR1 = ilog2c(R1);
  const int slot = (int)threadIdx.x >> LOGNB, t = (int)threadIdx.x & (NB - 1);
  const bool on = slot < nl;
  const unsigned k2 = on ? (unsigned)f2_line(slot, q0, np, R2) : 0u;
  const float2* src = in + ((size_t)k2 << LOGR1) + t;
  float2 v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = on ? __ldg(src + j * NB) : make_float2(0.f, 0.f);
  __syncthreads();   // st3 filled
  if (on) {
    const float2 ws = tw3(st3, (unsigned)NB * k2);
    float2 w = make_float2(1.f, 0.f);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      w = (j % 4 == 0) ? tw3(st3, (unsigned)(t + NB * j) * k2) : cmul(w, ws);
      v[j] = cmul(v[j], w);
    }
    Dft<16, false>::run(v);
    float2* dst = sm + slot * LSTR + 16 * t + t;    // element 16 t + j
#pragma unroll
    for (int j = 0; j < 16; ++j) dst[j] = v[j];
  }
}

// Real-input split by conjugate pairs after the row FFTs: with A = Z[k],
// B = conj(Z[L-k]), E = (A + B)/2, O = (A - B)/2 and W = exp(-i pi k / L),
//   X[k] = E - i W O   and   X[L-k] = conj(E) - i conj(W O),
// so one item produces both bins of a pair (slot t < np, column k1) and
// (slot t + np, column R1-1-k1), handed to emit(slot, row, k1, X).  In tile 0 lines
// 0 and R2/2 pair with themselves: line 0 pairs columns k1 and R1-k1 (k1 = 0
// and R1/2 alone), line R2/2 columns k1 and R1-1-k1.  Both bins of a pair are
// read before either is emitted, so emit may overwrite them in sm.
template <int R1, int LSTR, class Emit>
__device__ __forceinline__ void f2_split(float2* sm, int q0, int np, int R2, int logR2, int logL, Tw2 tw2L,
                                         Emit emit) {
  constexpr int LOGR1 = ilog2c(R1);
  const unsigned lmask = (1u << logL) - 1;
  int ra = 0, rb = 0;   // rows of the current slot pair
  auto split_w = [&](int sa, int ra, int ka, int sb, int rb, int kb, bool both, float2 W) {
    const float2 A = sm[pidx(sa, ka, LSTR)];
    const float2 B = cconj(sm[pidx(sb, kb, LSTR)]);
    const float2 E = cscale(cadd(A, B), 0.5f);
    const float2 O = cscale(csub(A, B), 0.5f);
    const float2 WO = cmul(W, O);
    emit(sa, ra, ka, cadd(E, rot90<false>(WO)));
    if (both) emit(sb, rb, kb, cadd(cconj(E), rot90<false>(cconj(WO))));
  };
  auto split = [&](int sa, int ka, int sb, int kb, bool both) {
    const int ra = f2_line(sa, q0, np, R2), rb = f2_line(sb, q0, np, R2);
    const unsigned k = (unsigned)ra + ((unsigned)ka << logR2);
    split_w(sa, ra, ka, sb, rb, kb, both, tw2(tw2L, k & lmask));
  };
  // a thread's items of one row are NT columns apart, so W advances by
  // exp(-i pi NT R2 / L) (refreshed from the table every fourth item)
  constexpr int UPI = R1 / NT > 1 ? R1 / NT : 1;
  const float2 wstep = tw2(tw2L, ((unsigned)NT << logR2) & lmask);
  float2 W = make_float2(1.f, 0.f);
  const int items = np * R1;
  if constexpr (R1 >= NT) {
    if (q0 != 0) {
      // every tile but tile 0: fully unrolled, a thread's items u are columns
      // threadIdx.x + u NT of slot (u NT) / R1 (at most EPT/2 of them)
#pragma unroll
      for (int u = 0; u < EPT / 2; ++u) {
        if (u * NT < items) {
          const int t = (u * NT) >> LOGR1, k1 = (int)threadIdx.x + ((u * NT) & (R1 - 1));
          if ((u * NT) % R1 == 0) {
            ra = f2_line(t, q0, np, R2);
            rb = f2_line(t + np, q0, np, R2);
          }
          if ((u * NT) % R1 != 0 && (u & 3) != 0) W = cmul(W, wstep);
          else W = tw2(tw2L, ((unsigned)ra + ((unsigned)k1 << logR2)) & lmask);
          split_w(t, ra, k1, t + np, rb, R1 - 1 - k1, true, W);
        }
      }
      return;
    }
  }
  int u = 0, tl = -1;
#pragma unroll 2
  for (int it = threadIdx.x; it < items; it += NT, ++u) {
    const int t = it >> LOGR1, k1 = it & (R1 - 1);
    if (t != tl) {
      tl = t;
      ra = f2_line(t, q0, np, R2);
      rb = f2_line(t + np, q0, np, R2);
    }
    if (q0 == 0 && t == 0) {
      if (k1 == 0) {
        split(0, 0, 0, 0, false);
        split(0, R1 >> 1, 0, R1 >> 1, false);
      } else if (k1 < (R1 >> 1)) {
        split(0, k1, 0, R1 - k1, true);
      } else {
        const int j = k1 - (R1 >> 1);
        split(np, j, np, R1 - 1 - j, true);
      }
    } else {
      if (UPI > 1 && u % UPI != 0 && (u & 3) != 0) W = cmul(W, wstep);
      else W = tw2(tw2L, ((unsigned)ra + ((unsigned)k1 << logR2)) & lmask);
      split_w(t, ra, k1, t + np, rb, R1 - 1 - k1, true, W);
    }
  }
}

// The spectrum X[k2 + R2 k1] is stored at row k2, column k1 of the output (the
// same place the row was read); the chirp is I1's.
template <int R1, bool TC>
__global__ void __launch_bounds__(NT, 2) k_fwd_rows(const float2* __restrict__ in, float2* __restrict__ out,
                                                    int logR2, int logL, const float2* __restrict__ tw3L, Tw2 tw2L,
                                                    const float2* __restrict__ tw, TcArgs tca) {
  extern __shared__ float2 smem[];
  float2* st3 = smem;                              // [TW3_SN], w = exp(-2 pi i / L)
  float2* stw = smem + TW3_SN;
  float2* sm = stw + stage_table_size(R1);
  constexpr int LSTR = line_stride(R1);
  constexpr int LOGR1 = ilog2c(R1);
  load_tw3(st3, tw3L);
  const int R2 = 1 << logR2;
  const int nl = min(TILE / R1, R2);   // 2 * pairs
  const int np = nl >> 1;
  load_twiddles<R1>(stw, tw);
  tc::Ctx tcc;
  if constexpr (TC) tc::setup(tcc, sm, tile_f2<R1, TC>(nl), tca);
  const int q0 = blockIdx.x * np;
  if constexpr (!TC && R1 >= 256) {
    if (threadIdx.x < 2 && np == 1 && blockIdx.x + PF_DIST < gridDim.x) {
      const int q = q0 + PF_DIST, row = threadIdx.x == 0 ? q : R2 - q;   // as in k_fwd_rows_inv
      prefetch_l2(in + ((size_t)row << LOGR1), R1 * (unsigned)sizeof(float2));
    }
    f2_stage1<R1, LSTR>(in, sm, st3, q0, np, R2, nl);
    __syncthreads();
    Stages<R1, 16, false, LSTR>::run(sm, nl, stw);        // the stages after the first
  } else {
    f2_load<R1, LSTR>(in, sm, st3, q0, np, R2, nl * R1);
    __syncthreads();
    fft_lines<R1, false, TC>(sm, nl, stw, &tcc);
    if constexpr (TC) tc::teardown(tcc);
  }
  f2_split<R1, LSTR>(sm, q0, np, R2, logR2, logL, tw2L, [&](int, int row, int k1, float2 X) {
    out[((unsigned)row << LOGR1) + (unsigned)k1] = X;
  });
}

// Length-J (= 64 = 16 x 4) inverse DFT of every (slot, c) run of a row tile
// (row stride R1 + R1/16, run c at c (J + J/16)), four lanes of one warp per
// run (run = threadIdx.x / 4, lane t4): the Stockham radix-16 step (outputs of
// butterfly t4 to 16 t4 + k) in registers, the exchange through the run's own
// line with warp-level barriers, the radix-4 step (butterflies t4 + 4q, outputs
// to t' + 16 j), then twk[slot][m1] = e^{2 pi i k2 m1 / M} and the store of
// element (k2 = row_of(slot), m1, c) at ((m1 G + g) R2 + k2) nl_c + ci,
// c = g nl_c + ci, nl_c = min(8192 / R2, NCH) (the column pass's blocks).
// The run's first read takes element o of the tile (its offset in the padded
// layout) from load(o); the runs' stores go to sm.
template <int R1, int J, class RowOf, class Load>
__device__ __forceinline__ void j_runs_load(float2* sm, const float2* stwj, const float2* twk,
                                            float2* __restrict__ out, int nl, int logR2, RowOf row_of, Load load) {
  static_assert(J == 64, "radix-16 x radix-4 runs");
  constexpr int NCH = R1 / J;
  constexpr int LSTR = R1 + R1 / 16;
  constexpr int LOGNCH = ilog2c(NCH);
  const int lognl = min(13 - logR2, LOGNCH);
  const int run = (int)threadIdx.x >> 2, t4 = (int)threadIdx.x & 3;
  if (run < nl * NCH) {                            // whole warps (8 runs each) in or out
    const int slot = run >> LOGNCH, c = run & (NCH - 1);
    const int lo = slot * LSTR + c * (J + J / 16);
    float2* line = sm + lo;
    float2 v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = load(lo + pidx(0, t4 + 4 * i, 0));
    Dft<16, true>::run(v);
    __syncwarp();                                  // the run is read before it is overwritten
#pragma unroll
    for (int k = 0; k < 16; ++k) line[pidx(0, 16 * t4 + k, 0)] = v[k];
    __syncwarp();
    const unsigned k2 = (unsigned)row_of(slot);
    const unsigned g = (unsigned)c >> lognl, ci = (unsigned)c & ((1u << lognl) - 1);
    const unsigned ofs0 = (((g << logR2) + k2) << lognl) + ci;
    const int mstep = LOGNCH + logR2;              // log2 of the m1 stride (G R2 nl_c)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int t = t4 + 4 * q;
      float2 w[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) w[j] = line[t + 17 * j];   // element t + 16 j (t < 16)
#pragma unroll
      for (int j = 1; j < 4; ++j) w[j] = cmul(w[j], cconj(stwj[(j - 1) * 16 + t]));
      Dft<4, true>::run(w);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int m1 = t + 16 * j;
        out[ofs0 + ((unsigned)m1 << mstep)] = cmul(w[j], twk[slot * J + m1]);
      }
    }
  }
}

// The runs of the tile held in sm.
template <int R1, int J, class RowOf>
__device__ __forceinline__ void j_runs(float2* sm, const float2* stwj, const float2* twk, float2* __restrict__ out,
                                       int nl, int logR2, RowOf row_of) {
  j_runs_load<R1, J>(sm, stwj, twk, out, nl, logR2, row_of, [&](int o) { return sm[o]; });
}

// ---------------------------------------------------------------------------
// F2f: F2 with the chirp and the first factor of every sub-channel's inverse
// ---------------------------------------------------------------------------

// When R2 divides M, row k2 holds for sub-channel c the J = M/R2 bins
// c M + k2 + R2 j (j < J) at columns c J + j, and with m = m1 + J m2
//   v_c[m] = sum_k2 e^{2 pi i k2 m2 / R2} e^{2 pi i k2 m1 / M}
//            sum_j Y_c[k2 + R2 j] e^{2 pi i j m1 / J}
// (times 1/M, applied on detection).  The inner sum is a length-J inverse DFT
// within the row, so F2f applies the chirp (Eq. 4) to the split spectrum in
// shared memory, transforms every (row, sub-channel) run of J bins, scales by
// e^{2 pi i k2 m1 / M} and stores element (k2, m1, c) blocked for the column
// pass (Ic): with nl = min(TILE/R2, NCH) sub-channels per Ic CTA and
// c = g nl + ci, at ((m1 G + g) R2 + k2) nl + ci, so that each Ic CTA reads one
// contiguous block (its stores here are runs of 4 sub-channels, 32 bytes).
// The row stride R1 + R1/16 makes each run a line of stride J + J/16.
template <int R1, int J, bool CTAB>
__global__ void __launch_bounds__(NT, 2) k_fwd_rows_inv(const float2* __restrict__ in, float2* __restrict__ out,
                                                        int logR2, int logL, const float2* __restrict__ tw3L,
                                                        Tw2 tw2L, const float2* __restrict__ tw,
                                                        const float2* __restrict__ twJ,
                                                        const ChirpAnchor* __restrict__ anc, int clog,
                                                        const float2* __restrict__ ctab) {
  static_assert(J >= 16 && J % 16 == 0 && R1 % (4 * J) == 0 && R1 >= NT, "row layout of the fused pass");
  constexpr int NCH = R1 / J;                 // sub-channels
  constexpr int LSTR = R1 + R1 / 16;
  constexpr int LOGJ = ilog2c(J), LOGNCH = ilog2c(NCH), LOGR1 = ilog2c(R1);
  extern __shared__ float2 smem[];
  float2* st3 = smem;                              // [TW3_SN], w = exp(-2 pi i / L)
  float2* stw = st3 + TW3_SN;
  float2* stwj = stw + stage_table_size(R1);
  float2* twk = stwj + stage_table_size(J);        // [nl][J]: e^{2 pi i k2 m1 / M}
  const int R2 = 1 << logR2;
  const int nl = min(TILE / R1, R2);
  const int np = nl >> 1;
  float2* sm = twk + nl * J;
  load_tw3(st3, tw3L);
  load_twiddles<R1>(stw, tw);
  load_twiddles<J>(stwj, twJ);
  const int q0 = blockIdx.x * np;
  if (threadIdx.x < 4 && np == 1 && blockIdx.x + PF_DIST < gridDim.x) {
    // the two rows of CTA blockIdx.x + PF_DIST (q and its mirror R2 - q), and
    // with the per-bin chirp table the same rows of the table
    const int q = q0 + PF_DIST, row = (threadIdx.x & 1) == 0 ? q : R2 - q;
    if (threadIdx.x < 2) prefetch_l2(in + ((size_t)row << LOGR1), R1 * (unsigned)sizeof(float2));
    else if (CTAB) prefetch_l2(ctab + ((size_t)row << LOGR1), R1 * (unsigned)sizeof(float2));
  }
  f2_stage1<R1, LSTR>(in, sm, st3, q0, np, R2, nl);
  // e^{2 pi i k2 m1 / M} = conj(w^{k2 m1 NCH}), k2 m1 NCH < L
  for (int i = threadIdx.x; i < nl * J; i += NT) {
    const unsigned k2 = (unsigned)f2_line(i >> LOGJ, q0, np, R2), m1 = (unsigned)(i & (J - 1));
    twk[i] = cconj(tw3(st3, (k2 * m1) << LOGNCH));
  }
  __syncthreads();
  Stages<R1, 16, false, LSTR>::run(sm, nl, stw);          // the stages after the first
  f2_split<R1, LSTR>(sm, q0, np, R2, logR2, logL, tw2L, [&](int slot, int row, int k1, float2 X) {
    if constexpr (CTAB) {
      // the chirp of bin row + R2 k1 from the plan's table (row layout: consecutive lanes, consecutive words)
      sm[pidx(slot, k1, LSTR)] = cmul(X, __ldg(ctab + ((size_t)row << LOGR1) + k1));
    } else {
      const unsigned k = (unsigned)row + ((unsigned)k1 << logR2);
      const ChirpAnchor a = anc[k >> clog];   // every row spans the band: L1/L2-resident table
      sm[pidx(slot, k1, LSTR)] = cmul(X, chirp_from(a, clog, k));
    }
  });
  __syncthreads();
  j_runs<R1, J>(sm, stwj, twk, out, nl, logR2, [&](int slot) { return f2_line(slot, q0, np, R2); });
}

// ---------------------------------------------------------------------------
// Ir: per-trial row pass of batched plans with M = 64 R2
// ---------------------------------------------------------------------------

// A batched plan shares F2's spectrum X[k2 + R2 k1] (row k2, column k1) among
// its trials, so the chirp cannot move into F2.  For each trial a CTA takes
// nl = min(TILE/R1, R2) consecutive rows, applies the trial's chirp (Eq. 4) as
// it loads them and runs F2f's length-64 runs and blocked store; the column
// pass (Ic) then completes the trial's sub-channel inverses.
template <int R1, int J>
__global__ void __launch_bounds__(NT, 2) k_inv_rows_chirp(const float2* __restrict__ in, float2* __restrict__ out,
                                                          int logR2, const float2* __restrict__ tw3L,
                                                          const float2* __restrict__ twJ,
                                                          const ChirpAnchor* __restrict__ anc, int clog) {
  static_assert(J == 64 && R1 % (4 * J) == 0 && R1 >= NT, "row layout of the fused pass");
  constexpr int NCH = R1 / J;
  constexpr int LSTR = R1 + R1 / 16;
  constexpr int LOGJ = ilog2c(J), LOGNCH = ilog2c(NCH), LOGR1 = ilog2c(R1);
  extern __shared__ float2 smem[];
  float2* st3 = smem;                              // [TW3_SN], w = exp(-2 pi i / L)
  float2* stwj = st3 + TW3_SN;
  float2* twk = stwj + stage_table_size(J);        // [nl][J]: e^{2 pi i k2 m1 / M}
  const int R2 = 1 << logR2;
  const int nl = min(TILE / R1, R2);
  float2* sm = twk + nl * J;
  load_tw3(st3, tw3L);
  load_twiddles<J>(stwj, twJ);
  const int r0 = blockIdx.x * nl;
  const int tot = nl * R1;
  // rows r0 .. r0 + nl - 1 are contiguous: 16-byte loads of columns k1, k1 + 1
  const float4* in4 = reinterpret_cast<const float4*>(in) + ((size_t)r0 << (LOGR1 - 1));
  constexpr int H = EPT / 2;
  float4 r[H];
#pragma unroll
  for (int u = 0; u < H; ++u) {
    const int idx = 2 * ((int)threadIdx.x + u * NT);
    if (idx < tot) r[u] = __ldg(in4 + (idx >> 1));
  }
#pragma unroll
  for (int u = 0; u < H; ++u) {
    const int idx = 2 * ((int)threadIdx.x + u * NT);
    if (idx < tot) {
      const int slot = idx >> LOGR1, k1 = idx & (R1 - 1);
      const unsigned ka = (unsigned)(r0 + slot) + ((unsigned)k1 << logR2), kb = ka + (1u << logR2);
      const ChirpAnchor a = anc[ka >> clog], b = anc[kb >> clog];
      float2* p = sm + pidx(slot, k1, LSTR);        // k1 even: no pad between the two
      p[0] = cmul(make_float2(r[u].x, r[u].y), chirp_from(a, clog, ka));
      p[1] = cmul(make_float2(r[u].z, r[u].w), chirp_from(b, clog, kb));
    }
  }
  __syncthreads();   // st3 and the tile
  // e^{2 pi i k2 m1 / M} = conj(w^{k2 m1 NCH}), k2 m1 NCH < L
  for (int i = threadIdx.x; i < nl * J; i += NT) {
    const unsigned k2 = (unsigned)(r0 + (i >> LOGJ)), m1 = (unsigned)(i & (J - 1));
    twk[i] = cconj(tw3(st3, (k2 * m1) << LOGNCH));
  }
  __syncthreads();
  j_runs<R1, J>(sm, stwj, twk, out, nl, logR2, [&](int slot) { return r0 + slot; });
}

// exp(-2 pi i r) for the phase r = u 2^-32 (mod 1) held as a Q0.32 word u: the
// same final sine and cosine as chirp_from.
__device__ __forceinline__ float2 chirp_q32(unsigned u) {
  const float r = (float)(int)u * 2.3283064365386963e-10f;   // 2^-32
  float s, c;
  __sincosf(6.2831853071795865f * r, &s, &c);
  return make_float2(c, -s);
}

// IrK, table form: Ir for the ntr trials of one batched launch with the rows
// resident.  CTA b (one per SM, R2 / nl of them) copies its nl rows of the
// shared spectrum and their table words (stored in the spectrum's row layout)
// into shared memory once, in the tile's padded layout, then runs every trial
// of the launch on them: each length-64 run applies the trial's chirp as it
// first reads its bins from those copies, and its F2f steps and blocked store
// for the column pass go to out + t out_tstride.  A run is read and written
// by the same four lanes, so the trials need no block barrier.  The rows are
// read from L2 or HBM once per launch instead of once per trial (per trial and
// segment, passes and decimation: 51.3 us one trial per CTA at two CTAs per
// SM, 48.2 with the rows resident and a chirped tile per trial).
template <int R1, int J>
__global__ void __launch_bounds__(NT, 1) k_inv_rows_chirp_res(const float2* __restrict__ in,
                                                              float2* __restrict__ out, long long out_tstride,
                                                              int logR2, const float2* __restrict__ tw3L,
                                                              const float2* __restrict__ twJ, MultiChirp mc,
                                                              int ntr) {
  static_assert(J == 64 && R1 % (4 * J) == 0 && R1 >= NT, "row layout of the fused pass");
  constexpr int NCH = R1 / J;
  constexpr int LSTR = R1 + R1 / 16;
  constexpr int LOGJ = ilog2c(J), LOGNCH = ilog2c(NCH), LOGR1 = ilog2c(R1);
  extern __shared__ float2 smem[];
  float2* st3 = smem;                              // [TW3_SN], w = exp(-2 pi i / L)
  float2* stwj = st3 + TW3_SN;
  float2* twk = stwj + stage_table_size(J);        // [nl][J]: e^{2 pi i k2 m1 / M}
  const int R2 = 1 << logR2;
  const int nl = min(TILE / R1, R2);
  const int tot = nl * R1;
  float2* rows = twk + nl * J;                     // [nl * LSTR], the tile's layout
  float2* sm = rows + nl * LSTR;                   // [nl * LSTR], the runs' exchange
  unsigned* tabw = reinterpret_cast<unsigned*>(sm + nl * LSTR);   // [nl * LSTR], the rows' table words
  const int r0 = blockIdx.x * nl;
  load_tw3(st3, tw3L);
  load_twiddles<J>(stwj, twJ);
  const float4* in4 = reinterpret_cast<const float4*>(in) + ((size_t)r0 << (LOGR1 - 1));
  const uint2* a2 = reinterpret_cast<const uint2*>(mc.atab) + ((size_t)r0 << (LOGR1 - 1));
  for (int i = threadIdx.x; i < tot / 2; i += NT) {
    const int idx = 2 * i, o = pidx(idx >> LOGR1, idx & (R1 - 1), LSTR);   // k1 even: o + 1 is k1 + 1
    const float4 rv = __ldg(in4 + i);
    const uint2 w = __ldg(a2 + i);
    rows[o] = make_float2(rv.x, rv.y);
    rows[o + 1] = make_float2(rv.z, rv.w);
    tabw[o] = w.x;
    tabw[o + 1] = w.y;
  }
  __syncthreads();   // st3
  for (int i = threadIdx.x; i < nl * J; i += NT) {
    const unsigned k2 = (unsigned)(r0 + (i >> LOGJ)), m1 = (unsigned)(i & (J - 1));
    twk[i] = cconj(tw3(st3, (k2 * m1) << LOGNCH));
  }
  __syncthreads();   // twk, the rows and their table words
  for (int t = 0; t < ntr; ++t) {
    const unsigned nm = __ldg(mc.nmul + t);
    j_runs_load<R1, J>(sm, stwj, twk, out + (size_t)t * out_tstride, nl, logR2, [&](int slot) { return r0 + slot; },
                       [&](int o) { return cmul(rows[o], chirp_q32(nm * tabw[o])); });
    __syncwarp();    // the run's last reads of sm come before the next trial's writes
  }
}

// IrK, anchor form: Ir for the ntr trials of one batched launch, one trial per
// CTA.  blockIdx.y is the row tile (nl rows of the shared spectrum) and
// blockIdx.x the trial, so the CTAs that read the same rows are adjacent in
// launch order and find them in L2 after the first.  Trial t's output (the
// blocked layout of F2f) goes to out + t out_tstride.  The anchor chirp costs
// about 20 more instructions per bin than the table's, and two CTAs per SM
// hide them better than the rows-resident form's one (per trial and segment,
// 32 trials per launch: 55.1 us here, 57.8 with the rows and each trial's
// anchors resident).
template <int R1, int J>
__global__ void __launch_bounds__(NT, 2) k_inv_rows_chirp_multi(const float2* __restrict__ in,
                                                                float2* __restrict__ out, long long out_tstride,
                                                                int logR2, const float2* __restrict__ tw3L,
                                                                const float2* __restrict__ twJ, MultiChirp mc) {
  static_assert(J == 64 && R1 % (4 * J) == 0 && R1 >= NT, "row layout of the fused pass");
  constexpr int NCH = R1 / J;
  constexpr int LSTR = R1 + R1 / 16;
  constexpr int LOGJ = ilog2c(J), LOGNCH = ilog2c(NCH), LOGR1 = ilog2c(R1);
  extern __shared__ float2 smem[];
  float2* st3 = smem;                              // [TW3_SN], w = exp(-2 pi i / L)
  float2* stwj = st3 + TW3_SN;
  float2* twk = stwj + stage_table_size(J);        // [nl][J]: e^{2 pi i k2 m1 / M}
  const int R2 = 1 << logR2;
  const int nl = min(TILE / R1, R2);
  float2* sm = twk + nl * J;
  const int t = blockIdx.x;
  const int r0 = blockIdx.y * nl;
  const int tot = nl * R1;
  if (t == 0 && threadIdx.x == 0) {
    // trials run fastest in launch order: the first trial's CTA of a row tile
    // warms L2 with the rows of a later tile
    const unsigned rn = blockIdx.y + max(1u, (unsigned)PF_DIST / gridDim.x);
    if (rn < gridDim.y) prefetch_l2(in + (((size_t)rn * nl) << LOGR1), (unsigned)tot * (unsigned)sizeof(float2));
  }
  load_tw3(st3, tw3L);
  load_twiddles<J>(stwj, twJ);
  // rows r0 .. r0 + nl - 1 are contiguous: 16-byte loads of columns k1, k1 + 1
  const float4* in4 = reinterpret_cast<const float4*>(in) + ((size_t)r0 << (LOGR1 - 1));
  constexpr int H = EPT / 2;
  float4 r[H];
#pragma unroll
  for (int u = 0; u < H; ++u) {
    const int idx = 2 * ((int)threadIdx.x + u * NT);
    if (idx < tot) r[u] = __ldg(in4 + (idx >> 1));
  }
  const ChirpAnchor* anc = mc.anc[t];
  const int clog = __ldg(mc.clog + t);
#pragma unroll
  for (int u = 0; u < H; ++u) {
    const int idx = 2 * ((int)threadIdx.x + u * NT);
    if (idx < tot) {
      const int slot = idx >> LOGR1, k1 = idx & (R1 - 1);
      const unsigned ka = (unsigned)(r0 + slot) + ((unsigned)k1 << logR2), kb = ka + (1u << logR2);
      const ChirpAnchor a = anc[ka >> clog], b = anc[kb >> clog];
      float2* p = sm + pidx(slot, k1, LSTR);
      p[0] = cmul(make_float2(r[u].x, r[u].y), chirp_from(a, clog, ka));
      p[1] = cmul(make_float2(r[u].z, r[u].w), chirp_from(b, clog, kb));
    }
  }
  __syncthreads();   // st3 and the tile
  for (int i = threadIdx.x; i < nl * J; i += NT) {
    const unsigned k2 = (unsigned)(r0 + (i >> LOGJ)), m1 = (unsigned)(i & (J - 1));
    twk[i] = cconj(tw3(st3, (k2 * m1) << LOGNCH));
  }
  __syncthreads();
  j_runs<R1, J>(sm, stwj, twk, out + (size_t)t * out_tstride, nl, logR2, [&](int slot) { return r0 + slot; });
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
__global__ void __launch_bounds__(NT, 2) k_inv_cols(const float2* __restrict__ in, float2* __restrict__ out,
                                                    int logQ1, int logM, int logR1, int logR2, int nchan,
                                                    const ChirpAnchor* __restrict__ anc, int clog,
                                                    const float2* __restrict__ tw, TcArgs tca) {
  extern __shared__ float2 smem[];
  ChirpAnchor* sanc = reinterpret_cast<ChirpAnchor*>(smem);   // [ANC_STAGE]
  float2* stw = smem + ANC_BYTES / sizeof(float2);
  float2* sm = stw + stage_table_size(Q2);
  constexpr int LSTR = col_stride<Q2>();
  constexpr int LOGQ2 = ilog2c(Q2);
  const int Q1 = 1 << logQ1;
  const int nl = min(TILE / Q2, nchan * Q1);
  const int lognl = __ffs(nl) - 1;
  const int tot = nl * Q2;
  load_twiddles<Q2>(stw, tw);
  tc::Ctx tcc;
  if constexpr (TC) tc::setup(tcc, sm, tile_f2<Q2, TC, LSTR>(nl), tca);
  const int tile = blockIdx.x;
  const int l0 = tile * nl;
  const int s = logR2 - logQ1;                 // j2 = j2lo + 2^s j2hi
  const int logrun = LOGQ2 - s;                // run length M / R2 (>= 1)
  // the CTA's bins lie in the sub-channels of its lines: stage their anchors
  long long a_lo = 0;
  bool staged = false;
  if (anc) {
    const long long c0 = l0 >> logQ1, c1 = (l0 + nl - 1) >> logQ1;
    a_lo = (c0 << logM) >> clog;
    const long long na = ((((c1 + 1) << logM) - 1) >> clog) - a_lo + 1;
    staged = na <= ANC_STAGE;
    if (staged)
      for (int i = threadIdx.x; i < (int)na; i += NT) sanc[i] = anc[a_lo + i];
  }
  // line l = l0 + (rest >> s) (l0 a multiple of nl), c = l / Q1, j1 = l mod Q1:
  // global offset k1 + k2 R1 with k1 = c M/R2 + j2hi, k2 = j1 + Q1 j2lo; bin
  // k = k2 + k1 R2; shared slot (rest >> s, j2lo + 2^s j2hi)
  const unsigned runm = (1u << logrun) - 1, sm1 = (1u << s) - 1;
  const Lin<EPT> gofs([&](unsigned idx) {
    const unsigned rest = idx >> logrun, l = (unsigned)l0 + (rest >> s);
    const unsigned k1 = ((l >> logQ1) << (logM - logR2)) + (idx & runm);
    return k1 + (((l & (Q1 - 1)) + ((rest & sm1) << logQ1)) << logR1);
  });
  const Lin<EPT> kbin([&](unsigned idx) {
    const unsigned rest = idx >> logrun, l = (unsigned)l0 + (rest >> s);
    const unsigned k1 = ((l >> logQ1) << (logM - logR2)) + (idx & runm);
    return (l & (Q1 - 1)) + ((rest & sm1) << logQ1) + (k1 << logR2);
  });
  const Lin<EPT> slot([&](unsigned idx) {
    const unsigned rest = idx >> logrun;
    return (unsigned)pidx((int)(rest >> s), (int)((rest & sm1) + ((idx & runm) << s)), LSTR);
  });
  float2 r[EPT];
#pragma unroll
  for (int u = 0; u < EPT; ++u)
    if ((int)threadIdx.x + u * NT < tot) r[u] = in[gofs(u)];
  if (anc) __syncthreads();   // staged anchors visible
#pragma unroll
  for (int u = 0; u < EPT; ++u) {
    if ((int)threadIdx.x + u * NT < tot) {
      if (anc) {
        const unsigned k = kbin(u);
        ChirpAnchor a;
        if (staged) a = sanc[(int)((long long)(k >> clog) - a_lo)];
        else a = anc[k >> clog];
        r[u] = cmul(r[u], chirp_from(a, clog, k));
      }
      sm[slot(u)] = r[u];
    }
  }
  __syncthreads();
  fft_lines<Q2, true, TC, LSTR>(sm, nl, stw, &tcc);
  if constexpr (TC) tc::teardown(tcc);
  // element (line b, m2) goes to c M + j1 + Q1 m2 with l0 + b = c Q1 + j1
  const Lin<EPT> oofs([&](unsigned idx) {
    const unsigned l = (unsigned)l0 + (idx & (nl - 1));
    return ((l >> logQ1) << logM) + (l & (Q1 - 1)) + ((idx >> lognl) << logQ1);
  });
  const Lin<EPT> oslot([&](unsigned idx) { return (unsigned)pidx((int)(idx & (nl - 1)), (int)(idx >> lognl), LSTR); });
#pragma unroll
  for (int u = 0; u < EPT; ++u)
    if ((int)threadIdx.x + u * NT < tot) out[oofs(u)] = sm[oslot(u)];
}

// ---------------------------------------------------------------------------
// I2: inverse row FFTs, discard, detect, sum over sub-channels
// ---------------------------------------------------------------------------

template <int Q1, bool TC>
__global__ void __launch_bounds__(NT, 2) k_inv_rows(const float2* __restrict__ buf, float* __restrict__ P,
                                                    float2* __restrict__ vout, long long vstride,
                                                    long long vofs, int logQ2, int logM, int nchan,
                                                    int m_lo, int m_hi, float scale,
                                                    const float2* __restrict__ tw3M,
                                                    const float2* __restrict__ tw, TcArgs tca) {
  extern __shared__ float2 smem[];
  float2* st3 = smem;                              // [TW3_SN], w = exp(+2 pi i / M)
  float2* stw = smem + TW3_SN;
  float2* sm = stw + stage_table_size(Q1);
  load_tw3(st3, tw3M);
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
  // slot = c b2 + bb (row m2_0 + bb of sub-channel c), element j1: global
  // offset c M + (m2_0 + bb) Q1 + j1
  const Lin<EPT> gofs([&](unsigned idx) {
    const unsigned sl = idx >> LOGQ1;
    return ((sl >> logb2) << logM) + (((unsigned)m2_0 + (sl & (b2 - 1))) << LOGQ1) + (idx & (Q1 - 1));
  });
  const Lin<EPT> slot([&](unsigned idx) { return (unsigned)pidx((int)(idx >> LOGQ1), (int)(idx & (Q1 - 1)), LSTR); });
  float2 r[EPT];
#pragma unroll
  for (int u = 0; u < EPT; ++u)
    if ((int)threadIdx.x + u * NT < tot) r[u] = buf[gofs(u)];
  __syncthreads();   // st3 filled
  // element j1 = e of row m2 carries I1's twiddle exp(+2 pi i j1 m2 / M); the
  // sub-channels of a row share it, so a thread reuses it while j1 m2 repeats
  {
    unsigned last = 0xffffffffu;
    float2 w = make_float2(1.f, 0.f);
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      const int idx = threadIdx.x + u * NT;
      if (idx < tot) {
        const int sl = idx >> LOGQ1, e = idx & (Q1 - 1);
        const unsigned ex = (unsigned)e * (unsigned)(m2_0 + (sl & (b2 - 1)));
        if (ex != last) {
          w = tw3(st3, ex);
          last = ex;
        }
        sm[slot(u)] = cmul(r[u], w);
      }
    }
  }
  __syncthreads();
  fft_lines<Q1, true, TC>(sm, nl, stw, &tcc);
  if constexpr (TC) tc::teardown(tcc);
  // Detect and sum over sub-channels.  The tile's no = b2 Q1 samples
  // (m = m2_0 + bb + Q2 m1) are shared by G = NT / no thread groups when no < NT;
  // group g sums sub-channels g, g + G, ..., and the G partial sums are added in
  // group order through shared memory.  P = scale^2 sum_c |v_c|^2.
  const int no = b2 * Q1;
  const float s2 = scale * scale;
  auto sample = [&](int o, int& m, int& bb, int& m1) {
    m1 = o >> logb2;
    bb = o & (b2 - 1);
    m = m2_0 + bb + (m1 << logQ2);
    return m >= m_lo && m < m_hi;
  };
  auto partial = [&](int bb, int m1, int m, int c0, int dc) {
    float p0 = 0.f, p1 = 0.f;
    for (int c = c0; c < nchan; c += dc) {
      const float2 v = sm[pidx((c << logb2) + bb, m1, LSTR)];
      p0 = fmaf(v.x, v.x, p0);
      p1 = fmaf(v.y, v.y, p1);
      if (vout) vout[(size_t)c * vstride + vofs + (m - m_lo)] = cscale(v, scale);
    }
    return p0 + p1;
  };
  if (no < NT && nchan > 1) {
    const int G = min(NT / no, nchan);
    const int tpg = NT / G;
    const int g = threadIdx.x / tpg, o = threadIdx.x - g * tpg;
    int m = 0, bb = 0, m1 = 0;
    const bool ok = o < no && sample(o, m, bb, m1);
    const float p = ok ? partial(bb, m1, m, g, G) : 0.f;
    __syncthreads();   // every read of the tile done
    float* red = reinterpret_cast<float*>(sm);   // [G][no]
    if (o < no) red[g * no + o] = p;
    __syncthreads();
    if (g == 0 && ok) {
      float q = red[o];
      for (int j = 1; j < G; ++j) q += red[j * no + o];
      P[m - m_lo] = q * s2;
    }
  } else {
    for (int o = threadIdx.x; o < no; o += NT) {
      int m, bb, m1;
      if (sample(o, m, bb, m1)) P[m - m_lo] = partial(bb, m1, m, 0, 1) * s2;
    }
  }
}


// ---------------------------------------------------------------------------
// Ic: column pass after F2f: inverse length-R2 FFTs, discard, detect, sum
// ---------------------------------------------------------------------------

// A CTA takes nl = min(TILE/R2, NCH) adjacent sub-channels c0.. of one m1 (one
// contiguous block of F2f's output, rows k2 of nl elements), transforms them along k2
// (v_c[m1 + J m2], m2 < R2), keeps the valid span m_lo <= m < m_hi, and detects.
// With G = NCH / nl > 1 the CTAs of one m1 each write their group's partial
// sum over sub-channels to part[g][m1][m2]; the last of the G to finish (an
// atomic ticket per m1, no waiting) adds the G partials in group order into P
// and clears the ticket.  P = scale^2 sum_c |v_c|^2.
template <int R2>
__global__ void __launch_bounds__(NT, 2) k_inv_cols_det(const float2* __restrict__ in, float* __restrict__ P,
                                                        float* __restrict__ part, int* __restrict__ cnt,
                                                        float2* __restrict__ vout, long long vstride,
                                                        long long vofs, int logR1, int lognch, int logJ,
                                                        int m_lo, int m_hi, float scale,
                                                        const float2* __restrict__ tw, TrialStride ts) {
  extern __shared__ float2 smem[];
  __shared__ int s_last;
  // batched launches: blockIdx.y is the trial, with its own input, P, partials and tickets
  in += blockIdx.y * ts.in;
  P += blockIdx.y * ts.P;
  part += blockIdx.y * ts.part;
  cnt += blockIdx.y * ts.cnt;
  float2* stw = smem;
  float2* sm = smem + stage_table_size(R2);
  constexpr int LSTR = col_stride<R2>();
  const int nl = min(TILE / R2, 1 << lognch);
  const int lognl = __ffs(nl) - 1;
  const int logG = lognch - lognl;
  const int tot = nl * R2;
  load_twiddles<R2>(stw, tw);
  const int m1 = blockIdx.x >> logG, gi = blockIdx.x & ((1 << logG) - 1);
  const float2* blk = in + (size_t)blockIdx.x * tot;   // block m1 G + g
  if (threadIdx.x < 4) {
    // the block of CTA blockIdx.x + PF_DIST (in launch order, the next trial's
    // blocks after this trial's last), in four quarters
    const unsigned nx = gridDim.x, lin = blockIdx.y * nx + blockIdx.x + PF_DIST;
    if (lin < nx * gridDim.y) {
      const float2* nb = in - blockIdx.y * ts.in + (size_t)(lin / nx) * ts.in + (size_t)(lin % nx) * tot;
      const unsigned qb = (unsigned)tot * (unsigned)sizeof(float2) / 4;
      if (ts.in != 0 || lin / nx == blockIdx.y)
        prefetch_l2(reinterpret_cast<const char*>(nb) + threadIdx.x * qb, qb);
    }
  }
  {
    // The first radix-16 stage straight from global memory: butterfly t of line
    // ci (sub-channels fastest, so consecutive lanes read consecutive elements)
    // reads element k2 = t + NB j of the block's rows, j < 16, and writes its
    // outputs to 16 t + j as the Stockham stage would.
    constexpr int NB = R2 / 16;
    const int ci = (int)threadIdx.x & (nl - 1), t = (int)threadIdx.x >> lognl;
    if (t < NB) {
      float2 v[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = blk[(t + NB * j) * nl + ci];
      Dft<16, true>::run(v);
      float2* dst = sm + ci * LSTR + pidx(0, 16 * t, 0);      // element 16 t + j
#pragma unroll
      for (int j = 0; j < 16; ++j) dst[j] = v[j];
    }
  }
  __syncthreads();
  Stages<R2, 16, true, LSTR>::run(sm, nl, stw);            // the stages after the first
  const float s2 = scale * scale;
  constexpr int NLMAX = TILE / R2 < NT ? TILE / R2 : NT;   // nl <= NLMAX
  constexpr int MPT = (R2 + NT - 1) / NT;                 // outputs per thread
#pragma unroll
  for (int q = 0; q < MPT; ++q) {
    const int m2 = (int)threadIdx.x + q * NT;
    if (m2 < R2) {
      const int m = m1 + (m2 << logJ);
      const bool ok = m >= m_lo && m < m_hi;
      float p0 = 0.f, p1 = 0.f;
      auto acc = [&](int b) {
        const float2 v = sm[pidx(b, m2, LSTR)];
        p0 = fmaf(v.x, v.x, p0);
        p1 = fmaf(v.y, v.y, p1);
      };
      if constexpr (NLMAX <= 16) {
#pragma unroll
        for (int b = 0; b < NLMAX; ++b)
          if (b < nl) acc(b);
      } else {
        for (int b = 0; b < nl; ++b) acc(b);
      }
      if (vout && ok)
        for (int b = 0; b < nl; ++b)
          vout[(size_t)((gi << lognl) + b) * vstride + vofs + (m - m_lo)] = cscale(sm[pidx(b, m2, LSTR)], scale);
      if (logG == 0) {
        if (ok) P[m - m_lo] = (p0 + p1) * s2;
      } else {
        part[((((size_t)gi << logJ) + m1) << ilog2c(R2)) + m2] = p0 + p1;
      }
    }
  }
  if (logG == 0) return;
  // release: the barrier orders every thread's partials before thread 0's fence
  // and ticket; acquire: the last group's thread 0 fences after its ticket and
  // the barrier orders the CTA's L2 loads of the other groups' partials after it
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const int t = atomicAdd(cnt + m1, 1);
    s_last = t == (1 << logG) - 1;
    if (s_last) {
      cnt[m1] = 0;   // every group has taken its ticket
      __threadfence();
    }
  }
  __syncthreads();
  if (!s_last) return;
  // the G partials of an output are loaded together, then added in group order
  constexpr int GMAX = 16;
  const size_t gstride = (size_t)1 << (logJ + ilog2c(R2));   // part[g + 1] - part[g]
#pragma unroll
  for (int q = 0; q < MPT; ++q) {
    const int m2 = (int)threadIdx.x + q * NT;
    const int m = m1 + (m2 << logJ);
    if (m2 >= R2 || m < m_lo || m >= m_hi) continue;
    const float* src = part + (((size_t)m1) << ilog2c(R2)) + m2;
    float acc = 0.f;
    if (logG <= 4) {
      float v[GMAX];
#pragma unroll
      for (int g = 0; g < GMAX; ++g) v[g] = g < (1 << logG) ? __ldcg(src + g * gstride) : 0.f;
#pragma unroll
      for (int g = 0; g < GMAX; ++g)
        if (g < (1 << logG)) acc += v[g];
    } else {
      for (int g = 0; g < (1 << logG); ++g) acc += __ldcg(src + g * gstride);
    }
    P[m - m_lo] = acc * s2;
  }
}


// ---------------------------------------------------------------------------
// Host launchers (one CTA per tile)
// ---------------------------------------------------------------------------

// Stage twiddle tables + padded tile (+ the tensor-core extras).
template <int R, bool TC, int LS = line_stride(R)>
size_t smem_bytes(int nl) {
  return ((size_t)stage_table_size(R) + (size_t)tile_f2<R, TC, LS>(nl)) * sizeof(float2) +
         (TC ? (size_t)tc::EXTRA_BYTES : 0);
}

#define POND_FOR_R(X) X(4) X(8) X(16) X(32) X(64) X(128) X(256) X(512) X(1024) X(2048) X(4096)

// Largest dynamic shared memory over the line lengths 4..4096.
template <bool TC>
size_t max_smem_t() {
  size_t m = 0;
#define MAXS(R) m = std::max(m, std::max(smem_bytes<R, TC>(TILE / R), smem_bytes<R, TC, col_stride<R>()>(TILE / R)));
  POND_FOR_R(MAXS)
#undef MAXS
  return m;
}

template <bool TC>
cudaError_t set_attributes_t() {
  // I1 adds its staged anchors, F2 its twiddle table (the larger of the two)
  const int max_smem = (int)max_smem_t<TC>() + (ANC_BYTES > TW3_BYTES ? ANC_BYTES : TW3_BYTES);
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
cudaError_t launch_fwd_cols_t(const Geom& g, SegIn in, float2* out, const float2* tw, cudaStream_t st) {
  const int R2 = 1 << g.logR2, R1 = 1 << g.logR1;
  const int nl = std::min(TILE / R2, R1);
  const unsigned grid = (unsigned)(R1 / nl);
  switch (R2) {
#define CASE(R) case R: k_fwd_cols<R, TC><<<grid, NT, smem_bytes<R, TC, col_stride<R>()>(nl), st>>>(in, out, g.logR1, tw, g.tc_fwd); break;
    POND_FOR_R(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <bool TC>
cudaError_t launch_fwd_rows_t(const Geom& g, const float2* in, float2* out, const float2* tw3L, Tw2 tw2L, const float2* tw,
                              cudaStream_t st) {
  const int R2 = 1 << g.logR2, R1 = 1 << g.logR1;
  const int nl = std::min(TILE / R1, R2);
  const unsigned grid = (unsigned)(R2 / nl);
  switch (R1) {
#define CASE(R) case R: k_fwd_rows<R, TC><<<grid, NT, smem_bytes<R, TC>(nl) + TW3_BYTES, st>>>(in, out, g.logR2, g.logL, tw3L, tw2L, tw, g.tc_fwd); break;
    POND_FOR_R(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <bool TC>
cudaError_t launch_inv_cols_t(const Geom& g, const float2* in, float2* out, const ChirpAnchor* anc,
                              int clog, const float2* tw, cudaStream_t st) {
  const int Q2 = 1 << g.logQ2, Q1 = 1 << g.logQ1;
  const int lines = g.nchan * Q1;
  const int nl = std::min(TILE / Q2, lines);
  const unsigned grid = (unsigned)(lines / nl);
  switch (Q2) {
#define CASE(R) case R: k_inv_cols<R, TC><<<grid, NT, smem_bytes<R, TC, col_stride<R>()>(nl) + ANC_BYTES, st>>>(in, out, g.logQ1, g.logM, g.logR1, g.logR2, g.nchan, anc, clog, tw, g.tc_inv); break;
    POND_FOR_R(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <bool TC>
cudaError_t launch_inv_rows_t(const Geom& g, const float2* buf, float* P, float2* vout, long long vstride,
                              long long vofs, int m_lo, int m_hi, const float2* tw3M, const float2* tw,
                               cudaStream_t st) {
  const int Q2 = 1 << g.logQ2, Q1 = 1 << g.logQ1;
  const int b2 = std::min(TILE / (Q1 * g.nchan), Q2);
  const int nl = g.nchan * b2;
  const unsigned grid = (unsigned)(Q2 / b2);
  const float scale = 1.0f / (float)(1u << g.logM);
  switch (Q1) {
#define CASE(R) case R: k_inv_rows<R, TC><<<grid, NT, smem_bytes<R, TC>(nl) + TW3_BYTES, st>>>(buf, P, vout, vstride, vofs, g.logQ2, g.logM, g.nchan, m_lo, m_hi, scale, tw3M, tw, g.tc_inv); break;
    POND_FOR_R(CASE)
#undef CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Tensor-core instantiations (kernels_tc.cu).
cudaError_t launch_fwd_cols_tc(const Geom& g, SegIn in, float2* out, const float2* tw, cudaStream_t st);
cudaError_t launch_fwd_rows_tc(const Geom& g, const float2* in, float2* out, const float2* tw3L, Tw2 tw2L, const float2* tw,
                               cudaStream_t st);
cudaError_t launch_inv_cols_tc(const Geom& g, const float2* in, float2* out, const ChirpAnchor* anc,
                               int clog, const float2* tw, cudaStream_t st);
cudaError_t launch_inv_rows_tc(const Geom& g, const float2* buf, float* P, float2* vout, long long vstride,
                               long long vofs, int m_lo, int m_hi, const float2* tw3M, const float2* tw,
                               cudaStream_t st);

}  // namespace pond
