// The three-pass schedule's column pass (Ic) on the tensor cores, split-BF16.
//
// Ic takes, for one m1 and four adjacent sub-channels c, the R2 = 2048 values
// x[k2] left by the row pass and forms each sub-channel's inverse transform
// v[m2] = sum_k2 x[k2] e^{+2 pi i k2 m2 / 2048}, then detects and sums over the
// sub-channels.  With k2 = a + 32 b (a < 32, b < 64) and m2 = p + 64 q
// (p < 64, q < 32) the transform splits into two dense DFT-matrix products
// with a twiddle between them (the four-step factorisation):
//   Y[a][p] = sum_b x[a + 32 b] e^{2 pi i b p / 64}            (first factor)
//   Y'[a][p] = Y[a][p] e^{2 pi i a p / 2048}                   (twiddle, FP32)
//   v[p + 64 q] = sum_a Y'[a][p] e^{2 pi i a q / 32}           (second factor)
// Both factors run as tcgen05.mma products (M = 128 rows, BF16 operands, FP32
// accumulators in tensor memory) in real block form: with A = [Re | Im] of the
// inputs along K and C, S the cosine and sine matrices of the factor,
//   Re out = Re in . C - Im in . S,   Im out = Re in . S + Im in . C,
// the minus sign taken by the MMA's negate-B flag.  Operands are split
// a = a_hi + a_lo (data) and c = c_hi + c_mid (matrices) into BF16 parts and
// the three-term product a_lo c_hi + a_hi c_mid + a_hi c_hi accumulates in
// FP32, as the radix-16 tensor-core stages do.
//
// First factor: row r = 4 a + c (128 rows: 32 a x 4 sub-channels), K = b; row r
// of the input block is x[r + 128 b] in the row pass's blocked layout (k2 nl +
// ci with nl = 4), so a warp's loads are 1 KiB runs.  Each thread writes its
// row into its own tensor-memory lane (the A operand), and the matrices C, S
// of the 64-point factor sit in shared memory.  Second factor: rows (p, c) in
// two groups of 128 (p < 32, p >= 32), K = a; the first factor's outputs are
// twiddled and written, split, straight into the canonical K-major layout of
// a shared-memory A operand (the transpose between the factors).  Detection
// then reads each row's 32 outputs from tensor memory, adds |v|^2 over the
// four sub-channels with two lane exchanges, and the partial sums over
// sub-channel groups are merged as in the FP32 pass.
#pragma once
#include "passes.cuh"

namespace pond {
namespace tcc {

constexpr int IC_R2 = 2048;
// Operand block (host-built, copied to shared memory by every CTA):
//   64-point factor: C64, S64 [p][b] (cos, sin 2 pi b p / 64), parts hi, mid;
//   32-point factor: C32, S32 [q][a], parts hi, mid;
//   twiddle tables T0[i] = e^{2 pi i i / 2048} (i < 64), T1[j] = e^{2 pi i 64 j / 2048} (j < 32).
constexpr int W64_PART = 64 * 64 * 2;
constexpr int W32_PART = 32 * 32 * 2;
constexpr int OFF_C64_HI = 0, OFF_C64_MID = W64_PART, OFF_S64_HI = 2 * W64_PART, OFF_S64_MID = 3 * W64_PART;
constexpr int OFF_W32 = 4 * W64_PART;
constexpr int OFF_C32_HI = OFF_W32, OFF_C32_MID = OFF_W32 + W32_PART, OFF_S32_HI = OFF_W32 + 2 * W32_PART,
              OFF_S32_MID = OFF_W32 + 3 * W32_PART;
constexpr int OFF_T0 = OFF_W32 + 4 * W32_PART;
constexpr int OFF_T1 = OFF_T0 + 64 * 8;
constexpr int OPS_BYTES = OFF_T1 + 32 * 8;           // 41,728 bytes
// Second factor's A operand in shared memory: two groups of 128 rows x 64 K, parts hi, lo.
constexpr int A3_GROUP = 128 * 64 * 2;
constexpr int A3_PART = 2 * A3_GROUP;
constexpr int SMEM_BYTES = 128 + OPS_BYTES + 2 * A3_PART + 64;   // about 106 KiB: two CTAs per SM
// Tensor memory: D (first factor: Re 0..63, Im 64..127; second factor: group h
// at 64 h, Re then Im), A of the first factor (hi 128..191, lo 192..255).
constexpr uint32_t COL_A_HI = 128, COL_A_LO = 192, TMEM_COLS = 256;
static_assert(OPS_BYTES % 128 == 0, "the A operand starts on a 128-byte boundary");
static_assert(SMEM_BYTES > tc::MIN_SMEM_BYTES, "at most two CTAs per SM, so the TMEM allocation never waits");

// Byte offset of element (row, k) of a K-major no-swizzle operand with K = 64
// (8-row x 16-byte core matrices; core matrix (row/8, k/8) at row/8 * 1024 + k/8 * 128).
__host__ __device__ constexpr int off_k64(int row, int k) {
  return (row >> 3) * 1024 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}
// The same for K = 32 (core matrix (row/8, k/8) at row/8 * 512 + k/8 * 128).
__host__ __device__ constexpr int off_k32(int row, int k) {
  return (row >> 3) * 512 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B (both
// K-major), B negated when negb (bit 14), N >> 3 in bits 17-22, M = 128.
__host__ __device__ constexpr uint32_t idesc(int n, bool negb) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (negb ? (1u << 14) : 0u) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(128 >> 4) << 24);
}

// Shared-memory descriptor of a K-major no-swizzle operand: leading byte offset
// (between K-adjacent core matrices) 128, stride byte offset sbo (between
// 8-row groups), descriptor version 1.
__device__ __forceinline__ uint64_t desc(uint32_t addr, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
      "r"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t* r) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
               "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}
// 16 consecutive columns of this thread's lane (the caller waits with tmem_ld_wait).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// x = hi + lo with hi, lo BF16 (round to nearest): two values per packed word.
__device__ __forceinline__ void split2(float x0, float x1, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}
__device__ __forceinline__ void split1(float x, unsigned short& hi, unsigned short& lo) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
  hi = *reinterpret_cast<const unsigned short*>(&h);
  lo = *reinterpret_cast<const unsigned short*>(&l);
}

// First factor: D[:, 0:64] = Re out, D[:, 64:128] = Im out over K = 128
// (Re x at K 0..63, Im x at 64..127; A in TMEM, two K per column), terms
// a_lo c_hi, a_hi c_mid, a_hi c_hi (smallest first).
__device__ __forceinline__ void issue_first(uint32_t tmem, uint32_t ops) {
#pragma unroll
  for (int o = 0; o < 2; ++o) {
    uint32_t acc = 0;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const uint32_t ap = t == 0 ? COL_A_LO : COL_A_HI;
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const bool cosm = (o == i);                    // Re.C, Im.C; else Re.S (+) or Im.S (-)
        const uint32_t m = cosm ? (t == 1 ? OFF_C64_MID : OFF_C64_HI) : (t == 1 ? OFF_S64_MID : OFF_S64_HI);
        const uint32_t id = idesc(64, o == 0 && i == 1);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          mma_ts(tmem + 64 * o, tmem + ap + 32 * i + 8 * s, desc(ops + m + 256 * s, 1024), id, acc);
          acc = 1;
        }
      }
    }
  }
}

// Second factor, row group h: D[:, 64 h + 0..31] = Re out, D[:, 64 h + 32..63]
// = Im out over K = 64 (Re Y' at K 0..31, Im Y' at 32..63; A in shared memory).
__device__ __forceinline__ void issue_second(uint32_t tmem, uint32_t a3, uint32_t ops) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
#pragma unroll
    for (int o = 0; o < 2; ++o) {
      uint32_t acc = 0;
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        const uint32_t ap = a3 + (t == 0 ? A3_PART : 0) + h * A3_GROUP;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const bool cosm = (o == i);
          const uint32_t m = cosm ? (t == 1 ? OFF_C32_MID : OFF_C32_HI) : (t == 1 ? OFF_S32_MID : OFF_S32_HI);
          const uint32_t id = idesc(32, o == 0 && i == 1);
#pragma unroll
          for (int s = 0; s < 2; ++s) {
            mma_ss(tmem + 64 * h + 32 * o, desc(ap + (2 * i + s) * 256, 1024), desc(ops + m + 256 * s, 512), id, acc);
            acc = 1;
          }
        }
      }
    }
  }
}

}  // namespace tcc

// Ic on the tensor cores for R2 = 2048 and four sub-channels per CTA (the
// blocked layout of the row pass with nl = 4); same grid, outputs, partial
// sums, tickets and trial strides as k_inv_cols_det.  Every wait for the MMAs
// is bounded (2 s); when one gives up the CTA sets the plan's error flag,
// skips its remaining MMAs and still finishes.
__global__ void __launch_bounds__(NT, 2) k_inv_cols_det_tc(const float2* __restrict__ in, float* __restrict__ P,
                                                           float* __restrict__ part, int* __restrict__ cnt,
                                                           float2* __restrict__ vout, long long vstride,
                                                           long long vofs, int lognch, int m_lo, int m_hi,
                                                           float scale, const uint4* __restrict__ ops_g,
                                                           int* __restrict__ err, TrialStride ts) {
  using namespace tcc;
  extern __shared__ unsigned char dsm[];
  __shared__ int s_last;
  in += blockIdx.y * ts.in;
  P += blockIdx.y * ts.P;
  part += blockIdx.y * ts.part;
  cnt += blockIdx.y * ts.cnt;
  constexpr int LOGJ = 6, LOGR2 = 11, NL = 4;
  unsigned char* ops = tc::align128(dsm);
  unsigned char* a3 = ops + OPS_BYTES;
  unsigned char* tail = a3 + 2 * A3_PART;
  const uint32_t bar = tc::smem_addr(tail);
  uint32_t* slot = reinterpret_cast<uint32_t*>(tail + 8);
  int* fail = reinterpret_cast<int*>(tail + 16);
  const int logG = lognch - 2;
  const int m1 = blockIdx.x >> logG, gi = blockIdx.x & ((1 << logG) - 1);
  const float2* blk = in + (size_t)blockIdx.x * (IC_R2 * NL);
  if (threadIdx.x < 4) {
    // the block of CTA blockIdx.x + PF_DIST in launch order, as the FP32 column pass does
    const unsigned nx = gridDim.x, lin = blockIdx.y * nx + blockIdx.x + PF_DIST;
    if (lin < nx * gridDim.y && (ts.in != 0 || lin / nx == blockIdx.y)) {
      const float2* nb = in - blockIdx.y * ts.in + (size_t)(lin / nx) * ts.in + (size_t)(lin % nx) * (IC_R2 * NL);
      constexpr unsigned QB = IC_R2 * NL * (unsigned)sizeof(float2) / 4;
      prefetch_l2(reinterpret_cast<const char*>(nb) + threadIdx.x * QB, QB);
    }
  }
  const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
  const int L = warp & 3, Q = warp >> 2;
  const int row = 32 * L + lane;                   // this thread's MMA row and TMEM lane
  // the thread's sixteen inputs: row `row`, b = 16 Q .. 16 Q + 15
  float2 x[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) x[i] = __ldg(blk + row + 128 * (16 * Q + i));
  for (int i = threadIdx.x; i < OPS_BYTES / 16; i += NT) reinterpret_cast<uint4*>(ops)[i] = __ldg(ops_g + i);
  if (warp == 0) tc::tmem_alloc(tc::smem_addr(slot), TMEM_COLS);
  if (threadIdx.x == 0) {
    tc::mbar_init(bar, 1);
    *fail = 0;
  }
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *slot;
  const uint32_t lane_base = tmem + ((uint32_t)(32 * L) << 16);
  {  // the first factor's A row: K = b (Re), 64 + b (Im), two K per column
    uint32_t hr[8], hm[8], lr[8], lm[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      tcc::split2(x[2 * j].x, x[2 * j + 1].x, hr[j], lr[j]);
      tcc::split2(x[2 * j].y, x[2 * j + 1].y, hm[j], lm[j]);
    }
    const uint32_t c0 = 8 * Q;
    tcc::tmem_st8(lane_base + COL_A_HI + c0, hr);
    tcc::tmem_st8(lane_base + COL_A_HI + 32 + c0, hm);
    tcc::tmem_st8(lane_base + COL_A_LO + c0, lr);
    tcc::tmem_st8(lane_base + COL_A_LO + 32 + c0, lm);
    tc::tmem_store_wait();
  }
  tc::fence_before_sync();
  __syncthreads();
  const uint32_t ops_s = tc::smem_addr(ops), a3_s = tc::smem_addr(a3);
  if (threadIdx.x == 0) {
    tc::fence_after_sync();
    tcc::issue_first(tmem, ops_s);
    tc::mma_commit(bar);
  }
  if (!tc::mbar_wait(bar, 0)) {
    *fail = 1;
    if (err) atomicExch(err, 1);
  }
  tc::fence_after_sync();
  {  // twiddle the first factor's outputs and write them, split, as the second factor's A rows
    float dr[16], di[16];
    tcc::tmem_ld16(lane_base + 16 * Q, dr);
    tcc::tmem_ld16(lane_base + 64 + 16 * Q, di);
    const int a = row >> 2, c = row & 3;
    const float2* t0 = reinterpret_cast<const float2*>(ops + OFF_T0);
    const float2* t1 = reinterpret_cast<const float2*>(ops + OFF_T1);
    unsigned short* ah = reinterpret_cast<unsigned short*>(a3);
    unsigned short* al = reinterpret_cast<unsigned short*>(a3 + A3_PART);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int p = 16 * Q + i;
      const int e = a * p;                            // < 2048
      const float2 y = cmul(make_float2(dr[i], di[i]), cmul(t0[e & 63], t1[e >> 6]));
      const int r = ((p & 31) << 2) | c, h = p >> 5;
      const int ore = (h * A3_GROUP + off_k64(r, a)) >> 1, oim = (h * A3_GROUP + off_k64(r, 32 + a)) >> 1;
      unsigned short hv, lv;
      tcc::split1(y.x, hv, lv);
      ah[ore] = hv;
      al[ore] = lv;
      tcc::split1(y.y, hv, lv);
      ah[oim] = hv;
      al[oim] = lv;
    }
  }
  tc::fence_before_sync();
  tc::fence_async_smem();
  __syncthreads();
  const bool skip = *fail != 0;
  if (threadIdx.x == 0 && !skip) {
    tc::fence_after_sync();
    tcc::issue_second(tmem, a3_s, ops_s);
    tc::mma_commit(bar);
  }
  if (!skip && !tc::mbar_wait(bar, 1)) {
    *fail = 1;
    if (err) atomicExch(err, 1);
  }
  tc::fence_after_sync();
  const float s2 = scale * scale;
  {  // detection: row (p, c) of group h holds v_c[p + 64 q] for q = 16 qh .. 16 qh + 15
    const int h = Q >> 1, qh = Q & 1;
    float vr[16], vi[16];
    tcc::tmem_ld16(lane_base + 64 * h + 16 * qh, vr);
    tcc::tmem_ld16(lane_base + 64 * h + 32 + 16 * qh, vi);
    const int p = 32 * h + (row >> 2), c = row & 3;
    float pw[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) pw[i] = fmaf(vr[i], vr[i], vi[i] * vi[i]);
    if (vout) {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int m = m1 + ((p + 64 * (16 * qh + i)) << LOGJ);
        if (m >= m_lo && m < m_hi)
          vout[(size_t)((gi << 2) + c) * vstride + vofs + (m - m_lo)] = make_float2(vr[i] * scale, vi[i] * scale);
      }
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      pw[i] += __shfl_xor_sync(0xffffffffu, pw[i], 1);
      pw[i] += __shfl_xor_sync(0xffffffffu, pw[i], 2);
    }
    if (c == 0) {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int m2 = p + 64 * (16 * qh + i);
        const int m = m1 + (m2 << LOGJ);
        if (logG == 0) {
          if (m >= m_lo && m < m_hi) P[m - m_lo] = pw[i] * s2;
        } else {
          part[((((size_t)gi << LOGJ) + m1) << LOGR2) + m2] = pw[i];
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, TMEM_COLS);
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
  constexpr int MPT = IC_R2 / NT;
  const size_t gstride = (size_t)1 << (LOGJ + LOGR2);
#pragma unroll
  for (int q = 0; q < MPT; ++q) {
    const int m2 = (int)threadIdx.x + q * NT;
    const int m = m1 + (m2 << LOGJ);
    if (m < m_lo || m >= m_hi) continue;
    const float* src = part + (((size_t)m1) << LOGR2) + m2;
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

}  // namespace pond
