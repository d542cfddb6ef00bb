// Radix-16 DFT stages on the 5th-generation tensor cores (tcgen05), split-BF16.
//
// A radix-16 butterfly is a product with the 16-point DFT matrix W16.  In real
// form a butterfly's 16 complex inputs are one row of 32 reals
// x = [Re x_0..Re x_15, Im x_0..Im x_15] and its outputs are x B^T with the
// 32 x 32 block matrix B = [[C, S], [-S, C]] (C = cos 2 pi jm/16,
// S = sin 2 pi jm/16; the inverse transform uses -S).  Each CTA stacks its
// 512 butterflies as four 128-row matrices X_g and computes D_g = X_g B^T with
// tcgen05.mma (M = 128, N = 32, K = 16 per instruction, BF16 operands, FP32
// accumulator in tensor memory).  Data are split x = x_hi + x_lo into two BF16
// numbers (about 16 significant bits); B is held as three BF16 parts
// b_hi + b_mid + b_lo (about 24 bits).  The three-term product is
// X_hi B_hi + X_hi B_mid + X_lo B_hi; the five-term product adds X_hi B_lo and
// X_lo B_mid, which leaves the data split as the only BF16 rounding.  Twiddle
// factors and everything outside the 16-point DFTs stay FP32.
//
// Row m of X_g is thread 128 g + m's butterfly, so each thread writes its own
// A row straight into its tensor-memory lane (tcgen05.st, two K per 32-bit
// column) and reads its 32 outputs back from the same lane (tcgen05.ld); the
// MMA takes A from tensor memory and B (the W16 parts) from shared memory.
// The shared-memory B operand uses the canonical K-major layout without
// swizzle: 8-row x 16-byte core matrices, 128 bytes each; core matrix
// (row/8, k/8) of a 32-column operand sits at (row/8) * 512 + (k/8) * 128
// bytes, so the descriptor's K-direction stride (leading byte offset) is 128
// and its row-group stride (stride byte offset) is 512.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_block.cuh"
#include "pond_internal.h"

namespace pond {
namespace tc {

constexpr int ROWS = 128;                    // MMA M
constexpr int NCOL = 32;                     // MMA N (real outputs per butterfly)
constexpr int GROUPS = 4;                    // 512 butterflies per CTA
constexpr unsigned long long WAIT_NS = 2000000000ull;   // an MMA wait gives up after 2 s

// Byte offset of element (row, k) of a 32-column K-major operand.
__device__ __forceinline__ int op_offset(int row, int k) {
  return (row >> 3) * 512 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start >> 4 in bits 0-13, leading byte
// offset >> 4 in bits 16-29, stride byte offset >> 4 in bits 32-45, descriptor
// version 1 in bits 46-47, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  const uint64_t lbo = 128, sbo = 512;
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((lbo >> 4) << 16) | ((sbo >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A
// and B (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 in bits 17-22,
// M >> 4 in bits 24-28.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NCOL >> 3) << 17) |
                           ((uint32_t)(ROWS >> 4) << 24);

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for the barrier phase `parity` to complete; false when limit_ns passes first.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned long long limit_ns = WAIT_NS) {
  unsigned long long t0 = 0;
  for (unsigned i = 0;; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    const unsigned long long t = globaltimer_ns();
    if (i == 0) t0 = t;
    else if (t - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate));
}

// D (TMEM) (+)= A (TMEM, 128 lanes x 16 BF16 = 8 columns of packed pairs) x B^T (shared).
__device__ __forceinline__ void mma_bf16_ts(uint32_t tmem_d, uint32_t tmem_a, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem_d),
      "r"(tmem_a), "l"(bdesc), "r"(IDESC), "r"(accumulate));
}

// 16 consecutive TMEM columns of this thread's lane from 16 registers.
__device__ __forceinline__ void tmem_store16(uint32_t taddr, const uint32_t* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
      "%14, %15, %16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_store_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 32 consecutive accumulator columns of this thread's lane.
__device__ __forceinline__ void tmem_load32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Per-CTA state of the tensor-core stages.  Tensor memory holds, per row group
// g, the accumulator D_g in columns [32 g, 32 g + 32) and the A operands in
// columns D_COLS + 32 g: X_hi (16 columns of packed BF16 pairs), then X_lo.
struct Ctx {
  uint32_t b_s;       // shared-window address of the W16 parts
  uint32_t bar_s;     // MMA completion barrier
  uint32_t tmem;      // base of the CTA's TMEM_ALLOC columns
  uint32_t phase;
  int* fail;          // CTA flag (shared): a wait expired, skip further MMAs
  int terms;
  int* err;           // plan-wide flag (global)
};

constexpr int D_COLS = GROUPS * NCOL;          // 128 accumulator columns
constexpr int TMEM_ALLOC = 2 * D_COLS;         // + 128 columns of A operands
constexpr int W_BYTES = TC_W_BYTES;            // W16 hi, mid, lo: 6 KiB
// Extra dynamic shared memory of a tensor-core kernel after its tile: alignment
// slack (the no-swizzle operand needs 16-byte alignment; it is placed on a
// 128-byte core-matrix boundary), the W16 parts, the barrier, the TMEM address
// slot and the fail flag.  Kept small: F2 at R = 4096 then still fits two CTAs
// per SM (115,712 bytes each).
constexpr int EXTRA_BYTES = 128 + W_BYTES + 64;
// Smallest dynamic shared memory of a tensor-core pass: with more than a third
// of the SM's shared memory per CTA at most two CTAs (2 x 256 TMEM columns)
// share an SM, so tcgen05.alloc never waits.  MIN_TILE_F2 counts the float2
// entries of stage tables + tile that reach it.
constexpr int MIN_SMEM_BYTES = 78 * 1024;
constexpr int MIN_TILE_F2 = (MIN_SMEM_BYTES - EXTRA_BYTES + 7) / 8;

__device__ __forceinline__ unsigned char* align128(void* p) {
  const uint32_t off = (128u - (smem_addr(p) & 127u)) & 127u;
  return static_cast<unsigned char*>(p) + off;
}

// Allocate tensor memory, initialise the barrier and copy the W16 parts.
// `tile` holds tile_f2 float2 entries followed by EXTRA_BYTES; all threads call.
__device__ __forceinline__ void setup(Ctx& c, float2* tile, int tile_f2, const TcArgs& ta) {
  unsigned char* x = align128(tile + tile_f2);
  unsigned char* bar = x + W_BYTES;
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 8);
  c.fail = reinterpret_cast<int*>(bar + 16);
  for (int i = threadIdx.x; i < W_BYTES / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(x)[i] = __ldg(ta.w + i);
  if (threadIdx.x < 32) tmem_alloc(smem_addr(slot), TMEM_ALLOC);
  if (threadIdx.x == 0) {
    mbar_init(smem_addr(bar), 1);
    *c.fail = 0;
  }
  fence_async_smem();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  c.b_s = smem_addr(x);
  c.bar_s = smem_addr(bar);
  c.tmem = *slot;
  c.phase = 0;
  c.terms = ta.terms;
  c.err = ta.err;
}

// Release tensor memory once every thread's TMEM accesses are done.
__device__ __forceinline__ void teardown(const Ctx& c) {
  fence_before_sync();
  __syncthreads();
  if (threadIdx.x < 32) {
    fence_after_sync();
    tmem_dealloc(c.tmem, TMEM_ALLOC);
  }
}

// TMEM address of this thread's lane (row) in column col.
__device__ __forceinline__ uint32_t lane_addr(const Ctx& c, int col) {
  return c.tmem + ((uint32_t)(((threadIdx.x >> 5) & 3) * 32) << 16) + (uint32_t)col;
}

// This thread's A row from 16 complex values: K 0..15 real parts, 16..31
// imaginary parts, two K per column, split into X_hi and X_lo.
__device__ __forceinline__ void store_row(const Ctx& c, const float2* v) {
  uint32_t h[16], l[16];
#pragma unroll
  for (int cc = 0; cc < 16; ++cc) {
    const int j = (cc & 7) * 2;
    const float x0 = cc < 8 ? v[j].x : v[j].y;
    const float x1 = cc < 8 ? v[j + 1].x : v[j + 1].y;
    const __nv_bfloat162 hb = __floats2bfloat162_rn(x0, x1);
    const float2 hf = __bfloat1622float2(hb);
    const __nv_bfloat162 lb = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
    h[cc] = *reinterpret_cast<const uint32_t*>(&hb);
    l[cc] = *reinterpret_cast<const uint32_t*>(&lb);
  }
  const int a0 = D_COLS + (threadIdx.x >> 7) * NCOL;
  tmem_store16(lane_addr(c, a0), h);
  tmem_store16(lane_addr(c, a0 + 16), l);
  tmem_store_wait();
}

// D_g = sum over the product terms of X_part W_part^T for the four row groups,
// smallest terms first.  Terms (X part, W part): 3 -> lo.hi, hi.mid, hi.hi;
// 5 -> lo.mid, hi.lo, lo.hi, hi.mid, hi.hi (W16 parts hi, mid, lo).
__device__ __forceinline__ void issue(const Ctx& c) {
  const int nt = c.terms == 5 ? 5 : 3;
  const uint32_t xs = nt == 5 ? 0x05u : 0x01u;   // bit t: X part of term t
  const uint32_t ws = nt == 5 ? 0x49u : 0x04u;   // 2 bits per term: W part of term t
#pragma unroll
  for (int g = 0; g < GROUPS; ++g) {
#pragma unroll
    for (int t = 0; t < 5; ++t) {
      if (t < nt) {
        const uint32_t xp = (xs >> t) & 1u, wp = (ws >> (2 * t)) & 3u;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          const uint32_t at = c.tmem + D_COLS + g * NCOL + xp * 16 + s * 8;
          const uint64_t bd = smem_desc(c.b_s + wp * (NCOL * 64) + s * 256);
          mma_bf16_ts(c.tmem + g * NCOL, at, bd, (t | s) != 0);
        }
      }
    }
  }
  mma_commit(c.bar_s);
}

// One radix-16 Stockham stage (same data movement as stockham_stage) whose
// 16-point DFTs run on the tensor cores; one butterfly per thread, whose row
// of A and D is the thread's own TMEM lane.
template <int R, int LS, bool INV, int LSTR = line_stride(R)>
__device__ __forceinline__ void stage16(float2* s, int nl, const float2* stw, Ctx& c) {
  constexpr int NB = R / 16;
  constexpr int LOGNB = ilog2c(NB);
  const int total = nl * NB;
  const int bf = threadIdx.x;
  const bool act = bf < total;
  const int line = bf >> LOGNB, t = bf & (NB - 1);
  const int k = t & (LS - 1);
  float2 v[16];
  if (act) {
    if constexpr (NB % 16 == 0) {
      const float2* p = s + line * LSTR + t + (t >> 4);
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = p[j * (NB + NB / 16)];
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] = s[pidx(line, t + j * NB, LSTR)];
    }
    if constexpr (LS > 1) {
      const float2* tws = stw + stage_table_offset(R, LS) + k;
#pragma unroll
      for (int j = 1; j < 16; ++j) {
        const float2 w = tws[(j - 1) * LS];
        v[j] = cmul(v[j], INV ? cconj(w) : w);
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = make_float2(0.f, 0.f);
  }
  store_row(c, v);
  fence_before_sync();
  __syncthreads();   // every input is read and every A row stored
  const bool skip = *c.fail != 0;
  if (threadIdx.x == 0 && !skip) {
    fence_after_sync();
    issue(c);
  }
  if (!skip && !mbar_wait(c.bar_s, c.phase)) {
    *c.fail = 1;
    if (c.err) atomicExch(c.err, 1);
  }
  c.phase ^= 1u;
  fence_after_sync();
  float d[32];
  tmem_load32(lane_addr(c, (threadIdx.x >> 7) * NCOL), d);
  if (act) {
    const int base = (t / LS) * (LS * 16) + k;
    if constexpr (LS % 16 == 0) {
      float2* p = s + line * LSTR + base + (base >> 4);
#pragma unroll
      for (int j = 0; j < 16; ++j) p[j * (LS + LS / 16)] = make_float2(d[j], d[16 + j]);
    } else if constexpr (LS == 1) {
      float2* p = s + line * LSTR + base + (base >> 4);
#pragma unroll
      for (int j = 0; j < 16; ++j) p[j] = make_float2(d[j], d[16 + j]);
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j) s[pidx(line, base + j * LS, LSTR)] = make_float2(d[j], d[16 + j]);
    }
  }
  __syncthreads();
}

}  // namespace tc

template <int R, int LS, bool INV, bool TC, int LSTR> struct StagesSel {
  static __device__ __forceinline__ void run(float2* s, int nl, const float2* stw, tc::Ctx* c) {
    if constexpr (LS < R) {
      constexpr int RAD = stage_radix(R, LS);
      if constexpr (TC && RAD == 16) tc::stage16<R, LS, INV, LSTR>(s, nl, stw, *c);
      else stockham_stage<R, RAD, LS, INV, LSTR>(s, nl, stw);
      StagesSel<R, LS * RAD, INV, TC, LSTR>::run(s, nl, stw, c);
    }
  }
};

// block_fft with the radix-16 stages on the tensor cores when TC (the radix-2/4/8
// stage of a length that is not a power of 16 stays on the FP32 path).
template <int R, bool INV, bool TC, int LSTR = line_stride(R)>
__device__ __forceinline__ void fft_lines(float2* s, int nl, const float2* stw, tc::Ctx* c) {
  StagesSel<R, 1, INV, TC, LSTR>::run(s, nl, stw, c);
}

}  // namespace pond
