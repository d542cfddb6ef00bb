// In-shared-memory FFT building blocks for the segment passes.
//
// A CTA holds a tile of TILE complex FP32 samples in shared memory: `nl` lines
// of R samples each (R a power of two, 4..4096).  All lines are transformed
// at once by radix-16 Stockham stages (one butterfly per thread per stage),
// followed by one radix-2/4/8 stage when log2(R) is not a multiple of 4.
// Stockham stage with radix r after sub-transforms of length Ls: butterfly t
// reads x[t + j R/r], j < r, multiplies input j by w^{j (t mod Ls)} with
// w = exp(-+2 pi i / (Ls r)), takes an r-point DFT and writes output j to
// (t / Ls) Ls r + (t mod Ls) + j Ls.  After the last stage the line holds its
// DFT in natural order.
//
// Shared-memory layout: line b, element e lives at b*LSTR + e + e/16 with
// LSTR = R + R/16 + 1 (odd) by default, so that both line-major and
// element-major sweeps of 8-byte elements avoid bank conflicts; a pass whose
// epilogue sweeps a few lines at a time may use R + R/16 + 16/nl instead
// (the stages sweep along lines and accept any stride).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pond {

constexpr int TILE = 8192;          // complex samples per CTA tile
constexpr int NT = TILE / 16;       // threads per FFT CTA
constexpr int TW_LOG = 13;          // twiddle table holds exp(-2 pi i m / 2^13)
constexpr int TW_N = 1 << TW_LOG;

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n >> 1); }
__host__ __device__ constexpr int line_stride(int R) { return R + R / 16 + 1; }
__device__ __forceinline__ int pidx(int line, int e, int lstr) { return line * lstr + e + (e >> 4); }

// The passes' CTAs start in launch order as earlier ones end (two resident per
// SM); CTA b asks L2 for the tile of CTA b + PF_DIST, which starts a fraction
// of a CTA lifetime later.  Measured on the full-rate plan (Msamples/s, two
// segment streams): none 104.1k; distance 1: 109.0k, 8: 109.9k, 16: 110.5k,
// 38: 111.2k, 76: 111.1k, 152: 110.2k, 304: 108.8k, 608: 105.6k.
constexpr int PF_DIST = 38;
// Ask L2 to fetch [p, p + bytes) (16-byte aligned, bytes a multiple of 16):
// no registers, no completion to wait for.
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Ask L2 for the whole 16-byte words of bytes [lo, hi) of p, in pieces of at
// most 64 KiB (rounded inward: nothing outside the range is touched).
__device__ __forceinline__ void prefetch_range(const int8_t* p, long long lo, long long hi) {
  uintptr_t s = ((uintptr_t)(p + lo) + 15) & ~(uintptr_t)15;
  const uintptr_t e = (uintptr_t)(p + hi) & ~(uintptr_t)15;
  for (; s < e; s += 65536) {
    const uintptr_t n = e - s < 65536 ? e - s : 65536;
    prefetch_l2(reinterpret_cast<const void*>(s), (unsigned)n);
  }
}

// Complex arithmetic on a (re, im) pair.  Component-wise sums, differences and
// real scalings are packed FP32x2 instructions (sm_100 and later: one issue
// for both components, each rounded as the scalar form).  The product stays
// scalar: its packed form needs the operands' components broadcast and swapped
// and issued no fewer instructions.
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  float2 r;
  asm("{.reg .b64 pa, pb, pd;\n\t"
      "mov.b64 pa, {%2, %3};\n\t"
      "mov.b64 pb, {%4, %5};\n\t"
      "sub.rn.f32x2 pd, pa, pb;\n\t"
      "mov.b64 {%0, %1}, pd;}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// multiply by -i (forward transform) or +i (inverse)
template <bool INV> __device__ __forceinline__ float2 rot90(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
// multiply by exp(-+ i pi/4) (the 8th root of unity of the transform direction)
template <bool INV> __device__ __forceinline__ float2 rot45(float2 a) {
  const float h = 0.70710678118654752f;
  return INV ? make_float2(h * (a.x - a.y), h * (a.x + a.y)) : make_float2(h * (a.x + a.y), h * (a.y - a.x));
}
template <bool INV> __device__ __forceinline__ float2 rot135(float2 a) {
  return rot90<INV>(rot45<INV>(a));
}

template <bool INV>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

// The odd outputs d02 +- rot90(d13) mix components, so they stay scalar.
template <bool INV>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 s02 = cadd(a0, a2), d02 = csub(a0, a2);
  const float2 s13 = cadd(a1, a3), d13 = csub(a1, a3);
  a0 = cadd(s02, s13);
  a2 = csub(s02, s13);
  if (INV) {   // rot90 = (-y, x)
    a1 = make_float2(d02.x - d13.y, d02.y + d13.x);
    a3 = make_float2(d02.x + d13.y, d02.y - d13.x);
  } else {     // rot90 = (y, -x)
    a1 = make_float2(d02.x + d13.y, d02.y - d13.x);
    a3 = make_float2(d02.x - d13.y, d02.y + d13.x);
  }
}

// r-point DFT of x (natural order in and out).
template <int RAD, bool INV> struct Dft;

template <bool INV> struct Dft<2, INV> {
  static __device__ __forceinline__ void run(float2* x) { dft2<INV>(x[0], x[1]); }
};

template <bool INV> struct Dft<4, INV> {
  static __device__ __forceinline__ void run(float2* x) { dft4<INV>(x[0], x[1], x[2], x[3]); }
};

// 8 = 4 (even/odd halves) x 2: X[k] = E[k] + w8^k O[k], X[k+4] = E[k] - w8^k O[k]
template <bool INV> struct Dft<8, INV> {
  static __device__ __forceinline__ void run(float2* x) {
    float2 e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
    float2 o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
    dft4<INV>(e0, e1, e2, e3);
    dft4<INV>(o0, o1, o2, o3);
    o1 = rot45<INV>(o1);
    o2 = rot90<INV>(o2);
    o3 = rot135<INV>(o3);
    x[0] = cadd(e0, o0); x[4] = csub(e0, o0);
    x[1] = cadd(e1, o1); x[5] = csub(e1, o1);
    x[2] = cadd(e2, o2); x[6] = csub(e2, o2);
    x[3] = cadd(e3, o3); x[7] = csub(e3, o3);
  }
};

// 16 = 4 x 4 with n = 4 n1 + n2, k = k1 + 4 k2:
// A[n2][k1] = DFT4_{n1} x[4 n1 + n2];  A *= w16^{n2 k1};  X[k1 + 4 k2] = DFT4_{n2} A[n2][k1]
template <bool INV> struct Dft<16, INV> {
  static __device__ __forceinline__ float2 tw16(float2 a, int e) {
    const float c1 = 0.92387953251128674f, s1 = 0.38268343236508978f;
    const float sg = INV ? 1.f : -1.f;   // sign of the imaginary part of w16
    switch (e) {
      case 1: return cmul(a, make_float2(c1, sg * s1));
      case 2: return rot45<INV>(a);
      case 3: return cmul(a, make_float2(s1, sg * c1));
      case 4: return rot90<INV>(a);
      case 6: return rot135<INV>(a);
      case 9: return cmul(a, make_float2(-c1, -sg * s1));
      default: return a;
    }
  }
  static __device__ __forceinline__ void run(float2* x) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(x[n2], x[n2 + 4], x[n2 + 8], x[n2 + 12]);
    // x[n2 + 4 k1] = A[n2][k1]
#pragma unroll
    for (int n2 = 1; n2 < 4; ++n2)
#pragma unroll
      for (int k1 = 1; k1 < 4; ++k1) x[n2 + 4 * k1] = tw16(x[n2 + 4 * k1], n2 * k1);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(x[4 * k1], x[4 * k1 + 1], x[4 * k1 + 2], x[4 * k1 + 3]);
    // x[4 k1 + k2] = X[k1 + 4 k2]: transpose the 4x4 digit order
    float2 y[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) y[k1 + 4 * k2] = x[4 * k1 + k2];
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = y[i];
  }
};

// Radix schedule of a length-R line: radix-16 stages, then one radix-2/4/8
// stage last when log2(R) is not a multiple of 4.  Stage s has radix RAD_s and
// follows sub-transforms of length LS_s = product of the earlier radices.
// Twiddles of a stage with LS > 1 live in a table laid out [j-1][k]
// (j = 1..RAD-1, k < LS): entry w^{j k}, w = exp(-2 pi i / (LS RAD)); threads
// with consecutive k read consecutive words.  The tables of all stages of R
// are concatenated in stage order; stage_table_size<R>() counts the entries.
__host__ __device__ constexpr int stage_radix(int R, int LS) {
  return (R / LS >= 16) ? 16 : R / LS;
}
__host__ __device__ constexpr int stage_table_offset(int R, int LS_target) {
  int off = 0;
  for (int ls = 1; ls < LS_target; ls *= stage_radix(R, ls))
    if (ls > 1) off += (stage_radix(R, ls) - 1) * ls;
  return off;
}
__host__ __device__ constexpr int stage_table_size(int R) { return stage_table_offset(R, R); }

// Copy the concatenated stage tables of R (global, FP64-built) into shared memory.
template <int R>
__device__ __forceinline__ void load_twiddles(float2* stw, const float2* __restrict__ gtw) {
  constexpr int NTW = stage_table_size(R);
  constexpr int PER = (NTW + NT - 1) / NT;
  if constexpr (NTW > 0) {
    float2 w[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int m = threadIdx.x + u * NT;
      if (m < NTW) w[u] = __ldg(gtw + m);
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int m = threadIdx.x + u * NT;
      if (m < NTW) stw[m] = w[u];
    }
  }
}

template <int R, int RAD, int LS, bool INV, int LSTR = line_stride(R)>
__device__ __forceinline__ void stockham_stage(float2* s, int nl, const float2* stw) {
  constexpr int NB = R / RAD;        // butterflies per line
  constexpr int BPT = 16 / RAD;      // butterflies per thread for a full tile
  constexpr int LOGNB = ilog2c(NB);
  const int total = nl * NB;
  float2 v[BPT][RAD];
#pragma unroll
  for (int u = 0; u < BPT; ++u) {
    const int bf = threadIdx.x + u * NT;
    if (bf < total) {
      const int line = bf >> LOGNB, t = bf & (NB - 1);
      if constexpr (NB % 16 == 0) {
        // (t + j NB) / 16 = t / 16 + j NB / 16: constant offsets per j
        const float2* p = s + line * LSTR + t + (t >> 4);
#pragma unroll
        for (int j = 0; j < RAD; ++j) v[u][j] = p[j * (NB + NB / 16)];
      } else {
#pragma unroll
        for (int j = 0; j < RAD; ++j) v[u][j] = s[pidx(line, t + j * NB, LSTR)];
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < BPT; ++u) {
    const int bf = threadIdx.x + u * NT;
    if (bf < total) {
      const int line = bf >> LOGNB, t = bf & (NB - 1);
      const int k = t & (LS - 1);
      if constexpr (LS > 1) {
        const float2* tws = stw + stage_table_offset(R, LS) + k;
#pragma unroll
        for (int j = 1; j < RAD; ++j) {
          const float2 w = tws[(j - 1) * LS];
          v[u][j] = cmul(v[u][j], INV ? cconj(w) : w);
        }
      }
      Dft<RAD, INV>::run(v[u]);
      const int base = (t / LS) * (LS * RAD) + k;
      if constexpr (LS % 16 == 0) {
        float2* p = s + line * LSTR + base + (base >> 4);
#pragma unroll
        for (int j = 0; j < RAD; ++j) p[j * (LS + LS / 16)] = v[u][j];
      } else if constexpr (LS == 1 && RAD == 16) {
        float2* p = s + line * LSTR + base + (base >> 4);   // base = 16 t: 17 t + j
#pragma unroll
        for (int j = 0; j < RAD; ++j) p[j] = v[u][j];
      } else {
#pragma unroll
        for (int j = 0; j < RAD; ++j) s[pidx(line, base + j * LS, LSTR)] = v[u][j];
      }
    }
  }
  __syncthreads();
}

template <int R, int LS, bool INV, int LSTR = line_stride(R)> struct Stages {
  static __device__ __forceinline__ void run(float2* s, int nl, const float2* stw) {
    if constexpr (LS < R) {
      constexpr int RAD = stage_radix(R, LS);
      stockham_stage<R, RAD, LS, INV, LSTR>(s, nl, stw);
      Stages<R, LS * RAD, INV, LSTR>::run(s, nl, stw);
    }
  }
};

// The stages of R with LS < LS_STOP (all but the last when LS_STOP is the last
// stage's LS): a pass that takes the last stage itself runs these first.
template <int R, int LS, bool INV, int LSTR, int LS_STOP> struct StagesUntil {
  static __device__ __forceinline__ void run(float2* s, int nl, const float2* stw) {
    if constexpr (LS < LS_STOP) {
      constexpr int RAD = stage_radix(R, LS);
      stockham_stage<R, RAD, LS, INV, LSTR>(s, nl, stw);
      StagesUntil<R, LS * RAD, INV, LSTR, LS_STOP>::run(s, nl, stw);
    }
  }
};

// Transform the nl lines of length R held in shared memory s (stw: stage tables).
template <int R, bool INV>
__device__ __forceinline__ void block_fft(float2* s, int nl, const float2* stw) {
  Stages<R, 1, INV>::run(s, nl, stw);
}

}  // namespace pond
