// Incoherent dedispersion modes of PONDER (Sec. 3.4): FFT filterbank with AID or
// CID detection and integration, per-channel Eq. 3 shifts with the channel sum,
// and the fold.
//
// Filterbank pass (k_fb_power<R>, R = 2 nchan).  A CTA owns a run of whole
// integration groups (spectra s0 .. s0 + S_cta).  Each line of its tile is one
// length-R complex FFT carrying two real blocks of R samples, z = a + i b:
//   AID: a, b are consecutive spectra's blocks of the (added) stream;
//   CID: a = N, b = S of one spectrum (one 2-byte load per complex sample).
// With A = Z[k] and C = Z[(R - k) mod R] the blocks' spectra are
// X_a = (A + conj C) / 2 and X_b = (A - conj C) / (2 i), so
//   |X_a|^2 = ((A.x + C.x)^2 + (A.y - C.y)^2) / 4,
//   |X_b|^2 = ((A.x - C.x)^2 + (A.y + C.y)^2) / 4,
//   Re(X_a conj X_b) = (A.x C.y + A.y C.x) / 2.
// A thread owns channels k and adds the spectra in order in registers; when an
// integration group is complete it writes row t of the time-major filterbank
// F[t][k] (all threads write one row together: coalesced).
//
// Shift-and-sum pass (k_incoh_sum).  A CTA owns DD_TD consecutive outputs; lane
// j of a warp takes channel 32 g + j, so one load reads 32 adjacent channels of
// one row (their delays differ by a sample at most within most groups).  Each
// lane sums its channel groups in order, the warp reduces its lanes, and the
// CTA adds its warps in order: a fixed order, so runs are bit-identical.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <vector>

#include "../../include/pond.h"
#include "fft_block.cuh"
#include "pond_internal.h"

namespace pond {
namespace {

constexpr double K_DM_S = 1.0 / 2.41e-4;   // s MHz^2, the coherent mode's constant
constexpr int FB_MIN_NCH = 64, FB_MAX_NCH = 2048;
constexpr int FB_MAX_LOGNINT = 16;
constexpr int DD_TD = 32;                  // outputs per shift-and-sum CTA
constexpr int DD_WARPS = 8;

enum FbForm { FB_AID1 = 0, FB_AID2 = 1, FB_CID = 2 };

struct FbArgs {
  const int8_t* x;       // input bytes (16-byte aligned)
  long long n_spec;      // spectra used: T nint
  long long s_cta;       // spectra per CTA: max(spectra per pass, nint)
  int lognint;
  int form;
  float* F;              // [T][nch]
};

__device__ __forceinline__ float s8(unsigned w, int byte) { return (float)(signed char)((w >> (8 * byte)) & 0xffu); }

// Four consecutive real samples x[q .. q+3] of the (added) stream, q a multiple of 4.
__device__ __forceinline__ void load_real4(const FbArgs& a, long long q, float (&v)[4]) {
  if (a.form == FB_AID1) {
    const unsigned w = __ldg(reinterpret_cast<const unsigned*>(a.x + q));
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = s8(w, i);
  } else {
    const uint2 w = __ldg(reinterpret_cast<const uint2*>(a.x + 2 * q));
    v[0] = s8(w.x, 0) + s8(w.x, 1);
    v[1] = s8(w.x, 2) + s8(w.x, 3);
    v[2] = s8(w.y, 0) + s8(w.y, 1);
    v[3] = s8(w.y, 2) + s8(w.y, 3);
  }
}

// ONE = false: one CTA per SM: with the pass loop around the stages, their
// per-thread indices stay live across passes and need more than the 64
// registers that two 512-thread CTAs per SM allow (at 64 the kernel spills).
// ONE = true (a CTA's spectra fit one tile pass, as with nint = 1): no pass
// loop and no running sums across passes, two CTAs per SM.
template <int R, bool ONE>
__global__ void __launch_bounds__(NT, ONE ? 2 : 1) k_fb_power(FbArgs a, const float2* __restrict__ tw) {
  constexpr int NCH = R / 2;
  constexpr int NL = TILE / R;                 // lines per pass
  constexpr int LSTR = line_stride(R);
  constexpr int QPL = R / 4;                   // 4-sample quads per line
  constexpr int QPT = TILE / 4 / NT;           // quads per thread per pass
  constexpr int KPT = NCH > NT ? NCH / NT : 1; // channels per thread
  extern __shared__ float2 smem[];
  float2* stw = smem;
  float2* sm = smem + stage_table_size(R);
  // running sums in shared memory, one per channel (each owned by one thread):
  // nothing but the pass offset stays in registers across the FFT stages
  float* acc = reinterpret_cast<float*>(sm + NL * LSTR);
  load_twiddles<R>(stw, tw);
  const int spl = a.form == FB_CID ? 1 : 2;    // spectra per line
  const long long s0 = (long long)blockIdx.x * a.s_cta;
  const int len = (int)min(a.s_cta, a.n_spec - s0);   // spectra of this CTA
  if (threadIdx.x == 0 && blockIdx.x + PF_DIST < gridDim.x) {
    // L2 prefetch of the input bytes of CTA blockIdx.x + PF_DIST (contiguous
    // spectra): AID 362.8k -> 402.4k, CID 272.3k -> 287.2k Msamples/s
    const long long bps = a.form == FB_AID1 ? 1 : 2;
    const long long n0 = (long long)(blockIdx.x + PF_DIST) * a.s_cta;
    const long long n1 = min(n0 + a.s_cta, a.n_spec);
    prefetch_range(a.x, n0 * R * bps, n1 * R * bps);
  }
  if (!ONE)
    for (int k = threadIdx.x; k < NCH; k += NT) acc[k] = 0.f;
  for (int p = 0; p < len; p += spl * NL) {
    // load: line l holds spectra s0 + p + spl l (+ 1)
#pragma unroll
    for (int u = 0; u < QPT; ++u) {
      const int q = (int)threadIdx.x + u * NT;
      const int l = q / QPL, n0 = 4 * (q % QPL);
      const int r = p + spl * l;               // spectrum within the CTA
      const long long sa = s0 + r;
      float re[4] = {0.f, 0.f, 0.f, 0.f}, im[4] = {0.f, 0.f, 0.f, 0.f};
      if (a.form == FB_CID) {
        if (r < len) {
          const uint2 w = __ldg(reinterpret_cast<const uint2*>(a.x + 2 * (sa * R + n0)));
          re[0] = s8(w.x, 0); im[0] = s8(w.x, 1); re[1] = s8(w.x, 2); im[1] = s8(w.x, 3);
          re[2] = s8(w.y, 0); im[2] = s8(w.y, 1); re[3] = s8(w.y, 2); im[3] = s8(w.y, 3);
        }
      } else {
        if (r < len) load_real4(a, sa * R + n0, re);
        if (r + 1 < len) load_real4(a, (sa + 1) * R + n0, im);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) sm[pidx(l, n0 + i, LSTR)] = make_float2(re[i], im[i]);
    }
    __syncthreads();
    Stages<R, 1, false, LSTR>::run(sm, NL, stw);
    // detect and integrate: thread-owned channels, spectra in order; a complete
    // group (spectrum index = -1 mod nint; s0 is a multiple of nint) is written
    // as row t of F by all threads together
    const int nmask = (1 << a.lognint) - 1;
#pragma unroll
    for (int u = 0; u < KPT; ++u) {
      const int k = (int)threadIdx.x + u * NT;
      if (k < NCH) {
        float s = ONE ? 0.f : acc[k];
        for (int l = 0; l < NL; ++l) {
          const int r = p + spl * l;
          if (r >= len) break;
          const float2 A = sm[pidx(l, k, LSTR)];
          const float2 C = sm[pidx(l, (R - k) & (R - 1), LSTR)];
          if (a.form == FB_CID) {
            s += 0.5f * (A.x * C.y + A.y * C.x);
            if ((r & nmask) == nmask) {
              a.F[((s0 + r) >> a.lognint) * NCH + k] = s;
              s = 0.f;
            }
          } else {
            const float ar = A.x + C.x, ai = A.y - C.y, br = A.x - C.x, bi = A.y + C.y;
            s += 0.25f * (ar * ar + ai * ai);
            if ((r & nmask) == nmask) {
              a.F[((s0 + r) >> a.lognint) * NCH + k] = s;
              s = 0.f;
            }
            if (r + 1 < len) {
              s += 0.25f * (br * br + bi * bi);
              if (((r + 1) & nmask) == nmask) {
                a.F[((s0 + r + 1) >> a.lognint) * NCH + k] = s;
                s = 0.f;
              }
            }
          }
        }
        if (!ONE) acc[k] = s;
      }
    }
    if (ONE) break;    // the CTA's spectra fit one pass
    __syncthreads();   // the next pass's loads overwrite the tile
  }
}

// D[i] = sum_k F[t_first + i + d_k][k], i < n_out (nch a multiple of 32).
__global__ void __launch_bounds__(DD_WARPS * 32) k_incoh_sum(const float* __restrict__ F, int nch,
                                                             const int* __restrict__ d, long long t_first,
                                                             long long n_out, float* __restrict__ D) {
  extern __shared__ int sd[];
  __shared__ float red[DD_WARPS][DD_TD];
  for (int k = threadIdx.x; k < nch; k += blockDim.x) sd[k] = __ldg(d + k);
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long i0 = (long long)blockIdx.x * DD_TD;
  const int td = (int)min((long long)DD_TD, n_out - i0);
  float part[DD_TD];
#pragma unroll
  for (int t = 0; t < DD_TD; ++t) part[t] = 0.f;
  for (int g = w; g < nch / 32; g += DD_WARPS) {
    const int k = g * 32 + lane;
    const float* p = F + (t_first + i0 + sd[k]) * nch + k;
#pragma unroll
    for (int t = 0; t < DD_TD; ++t)
      if (t < td) part[t] += __ldg(p + (long long)t * nch);
  }
#pragma unroll
  for (int t = 0; t < DD_TD; ++t) {
    float v = part[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[w][t] = v;
  }
  __syncthreads();
  if ((int)threadIdx.x < td) {
    float s = 0.f;
#pragma unroll
    for (int v = 0; v < DD_WARPS; ++v) s += red[v][threadIdx.x];
    D[i0 + threadIdx.x] = s;
  }
}

// Fluctuation spectrum of the series (Sec. 3.5): chunks of L samples, two per
// complex line (z = c_j + i c_{j+1}), A[f] = sum_j |X_j[f]|^2 for f = 0 .. L/2,
// j over the J complete chunks.  One CTA: each thread owns bins f and adds the
// chunks in order in FP64, so the result needs no merge and is deterministic.
template <int L>
__global__ void __launch_bounds__(NT, 1) k_ips_spectrum(const float* __restrict__ c, long long J,
                                                        const float2* __restrict__ tw, double* __restrict__ out) {
  constexpr int NL = TILE / L;                 // lines per pass (2 chunks each)
  constexpr int LSTR = line_stride(L);
  constexpr int QPL = L / 4;
  constexpr int QPT = TILE / 4 / NT;
  constexpr int NF = L / 2 + 1;                // bins 0 .. L/2
  constexpr int FPT = (NF + NT - 1) / NT;
  extern __shared__ float2 smem[];
  float2* stw = smem;
  float2* sm = smem + stage_table_size(L);
  load_twiddles<L>(stw, tw);
  double acc[FPT];
#pragma unroll
  for (int u = 0; u < FPT; ++u) acc[u] = 0.0;
  for (long long p = 0; p < J; p += 2 * NL) {
#pragma unroll
    for (int u = 0; u < QPT; ++u) {
      const int q = (int)threadIdx.x + u * NT;
      const int l = q / QPL, n0 = 4 * (q % QPL);
      const long long ja = p + 2 * l;
      float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
      if (ja < J) a = __ldg(reinterpret_cast<const float4*>(c + ja * L + n0));
      if (ja + 1 < J) b = __ldg(reinterpret_cast<const float4*>(c + (ja + 1) * L + n0));
      sm[pidx(l, n0, LSTR)] = make_float2(a.x, b.x);
      sm[pidx(l, n0 + 1, LSTR)] = make_float2(a.y, b.y);
      sm[pidx(l, n0 + 2, LSTR)] = make_float2(a.z, b.z);
      sm[pidx(l, n0 + 3, LSTR)] = make_float2(a.w, b.w);
    }
    __syncthreads();
    Stages<L, 1, false, LSTR>::run(sm, NL, stw);
#pragma unroll
    for (int u = 0; u < FPT; ++u) {
      const int f = (int)threadIdx.x + u * NT;
      if (f < NF) {
        for (int l = 0; l < NL; ++l) {
          const long long ja = p + 2 * l;
          if (ja >= J) break;
          const float2 A = sm[pidx(l, f, LSTR)];
          const float2 C = sm[pidx(l, (L - f) & (L - 1), LSTR)];
          const float ar = A.x + C.x, ai = A.y - C.y, br = A.x - C.x, bi = A.y + C.y;
          acc[u] += (double)(0.25f * (ar * ar + ai * ai));
          if (ja + 1 < J) acc[u] += (double)(0.25f * (br * br + bi * bi));
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < FPT; ++u) {
    const int f = (int)threadIdx.x + u * NT;
    if (f < NF) out[f] = acc[u];
  }
}

template <int L>
size_t ips_smem_bytes() {
  return ((size_t)stage_table_size(L) + (size_t)(TILE / L) * line_stride(L)) * sizeof(float2);
}

template <int R>
size_t fb_smem_bytes() {
  return ((size_t)stage_table_size(R) + (size_t)(TILE / R) * line_stride(R)) * sizeof(float2) +
         (size_t)(R / 2) * sizeof(float);
}

}  // namespace
}  // namespace pond

// ---------------------------------------------------------------------------
// Host side: plan, launches and the C ABI.
// ---------------------------------------------------------------------------

struct pond_incoh_s {
  int device = 0;
  pond_incoh_opts o{};
  int nch = 0, logR = 0, lognint = 0, form = 0;
  double ts = 0.0, inc = 0.0;
  std::vector<int> delay;
  int dmin = 0, dmax = 0;
  int* d_delay = nullptr;
  float2* stw = nullptr;
  float2* stwL = nullptr;    // stage tables of the fluctuation FFT (ips_len)
  double* ips = nullptr;     // accumulated fluctuation spectrum [ips_len / 2 + 1]
  long long ips_chunks = 0;
  float* F = nullptr;
  size_t F_cap = 0;          // floats
  float* D = nullptr;
  size_t D_cap = 0;
  double* psum = nullptr;
  int* phits = nullptr;
  double* prof_sum = nullptr;
  long long* prof_hits = nullptr;
  cudaEvent_t ev[5] = {};
  cudaStream_t st = nullptr; // stream of the last run
  bool ran = false;
  long long T = 0, t_first = 0, n_out = 0;
  double in_bytes = 0.0;
  int launches = 0;
};

namespace {

using pond::FbArgs;

int err(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  return pond::set_error(code, buf);
}

#define ICK(call)                                                                                   \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess)                                                                          \
      return err(e_ == cudaErrorMemoryAllocation ? POND_E_OOM : POND_E_CUDA, "%s: %s", #call,        \
                 cudaGetErrorString(e_));                                                           \
  } while (0)

// Keeps a product rounded on its own (no fused multiply-add with what follows), so
// the FP64 channel frequencies match a plain evaluation of the same expression.
double rounded(double x) {
  volatile double v = x;
  return v;
}

template <int R>
cudaError_t fb_attr() {
  cudaError_t e = cudaFuncSetAttribute(pond::k_fb_power<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)pond::fb_smem_bytes<R>());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(pond::k_fb_power<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)pond::fb_smem_bytes<R>());
  return e;
}

template <int R>
cudaError_t fb_launch(const FbArgs& a, const float2* tw, cudaStream_t st) {
  const long long blocks = (a.n_spec + a.s_cta - 1) / a.s_cta;
  const long long per_pass = (long long)(a.form == pond::FB_CID ? 1 : 2) * (pond::TILE / R);
  if (a.s_cta <= per_pass)
    pond::k_fb_power<R, true><<<(unsigned)blocks, pond::NT, pond::fb_smem_bytes<R>(), st>>>(a, tw);
  else
    pond::k_fb_power<R, false><<<(unsigned)blocks, pond::NT, pond::fb_smem_bytes<R>(), st>>>(a, tw);
  return cudaGetLastError();
}

template <int L>
cudaError_t ips_attr() {
  return cudaFuncSetAttribute(pond::k_ips_spectrum<L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)pond::ips_smem_bytes<L>());
}

template <int L>
cudaError_t ips_launch(const float* c, long long J, const float2* tw, double* out, cudaStream_t st) {
  pond::k_ips_spectrum<L><<<1, pond::NT, pond::ips_smem_bytes<L>(), st>>>(c, J, tw, out);
  return cudaGetLastError();
}

cudaError_t ips_dispatch(int logL, bool attr, const float* c, long long J, const float2* tw, double* out,
                         cudaStream_t st) {
  switch (logL) {
#define IPS_CASE(K) \
  case K: return attr ? ips_attr<1 << K>() : ips_launch<1 << K>(c, J, tw, out, st);
    IPS_CASE(6) IPS_CASE(7) IPS_CASE(8) IPS_CASE(9) IPS_CASE(10) IPS_CASE(11) IPS_CASE(12)
#undef IPS_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t fb_dispatch(int logR, bool attr, const FbArgs& a, const float2* tw, cudaStream_t st) {
  switch (logR) {
#define FB_CASE(L) \
  case L: return attr ? fb_attr<1 << L>() : fb_launch<1 << L>(a, tw, st);
    FB_CASE(7) FB_CASE(8) FB_CASE(9) FB_CASE(10) FB_CASE(11) FB_CASE(12)
#undef FB_CASE
    default: return cudaErrorInvalidValue;
  }
}

bool pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }
int ilog2(long long v) {
  int l = 0;
  while ((1ll << l) < v) ++l;
  return l;
}

void release(pond_incoh_t h) {
  cudaFree(h->d_delay);
  cudaFree(h->stw);
  cudaFree(h->stwL);
  cudaFree(h->ips);
  cudaFree(h->F);
  cudaFree(h->D);
  cudaFree(h->psum);
  cudaFree(h->phits);
  cudaFree(h->prof_sum);
  cudaFree(h->prof_hits);
  for (auto& e : h->ev)
    if (e) cudaEventDestroy(e);
}

int wait_last(pond_incoh_t h) {
  ICK(cudaSetDevice(h->device));
  if (h->ran) ICK(cudaStreamSynchronize(h->st));
  return POND_OK;
}

}  // namespace

extern "C" int pond_incoh_create(pond_incoh_t* out, const pond_incoh_opts* o) {
  if (!out || !o) return err(POND_E_ARG, "pond_incoh_create: null pointer");
  *out = nullptr;
  for (int r : o->reserved)
    if (r) return err(POND_E_ARG, "pond_incoh_create: reserved fields must be zero");
  const double half = std::fabs(o->bw_mhz) / 2.0;
  if (!(o->bw_mhz != 0.0) || !(o->f0_mhz > half) || !std::isfinite(o->f0_mhz) ||
      !(std::fabs(o->fs_hz - 2.0 * std::fabs(o->bw_mhz) * 1e6) <= 1e-9 * o->fs_hz))
    return err(POND_E_ARG, "pond_incoh_create: need f0 > |bw|/2 > 0 and fs = 2 |bw| 1e6");
  if (!(o->dm >= 0.0) || !std::isfinite(o->dm) || !(o->period_s > 0.0) || !std::isfinite(o->period_s))
    return err(POND_E_ARG, "pond_incoh_create: need dm >= 0 and period > 0");
  if (o->nbins < 1 || o->nbins > pond::MAX_NBINS)
    return err(POND_E_ARG, "pond_incoh_create: nbins must be 1..%d", pond::MAX_NBINS);
  if (!((o->mode == POND_INCOH_AID && (o->input_channels == 1 || o->input_channels == 2)) ||
        (o->mode == POND_INCOH_CID && o->input_channels == 2)))
    return err(POND_E_ARG, "pond_incoh_create: AID takes 1 or 2 input channels, CID takes 2");
  if (!pow2(o->nchan) || o->nchan < pond::FB_MIN_NCH || o->nchan > pond::FB_MAX_NCH)
    return err(POND_E_NCHAN, "pond_incoh_create: nchan must be a power of two in %d..%d", pond::FB_MIN_NCH,
               pond::FB_MAX_NCH);
  if (!pow2(o->nint) || o->nint > (1 << pond::FB_MAX_LOGNINT))
    return err(POND_E_ARG, "pond_incoh_create: nint must be a power of two in 1..%d", 1 << pond::FB_MAX_LOGNINT);
  if (o->ips_len != 0 && (!pow2(o->ips_len) || o->ips_len < 64 || o->ips_len > 4096))
    return err(POND_E_ARG, "pond_incoh_create: ips_len must be 0 or a power of two in 64..4096");
  pond_incoh_t h = new pond_incoh_s;
  h->device = o->device;
  h->o = *o;
  h->nch = o->nchan;
  h->logR = ilog2(2ll * o->nchan);
  h->lognint = ilog2(o->nint);
  h->form = o->mode == POND_INCOH_CID ? pond::FB_CID : (o->input_channels == 2 ? pond::FB_AID2 : pond::FB_AID1);
  h->ts = 2.0 * o->nchan * o->nint / o->fs_hz;
  h->inc = h->ts / o->period_s;
  h->delay.resize(o->nchan);
  const double df = std::fabs(o->bw_mhz) / o->nchan;
  const double base = o->bw_mhz > 0 ? o->f0_mhz - half : o->f0_mhz + half;
  for (int k = 0; k < o->nchan; ++k) {
    const double kd = rounded((double)k * df);
    const double f = o->bw_mhz > 0 ? base + kd : base - kd;
    const double delay_s = pond::K_DM_S * o->dm * (std::pow(f, -2.0) - std::pow(o->f0_mhz, -2.0));
    h->delay[k] = (int)std::floor(delay_s / h->ts + 0.5);
  }
  h->dmin = *std::min_element(h->delay.begin(), h->delay.end());
  h->dmax = *std::max_element(h->delay.begin(), h->delay.end());
  auto bail = [&](int rc) {
    release(h);
    delete h;
    return rc;
  };
  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) != cudaSuccess || o->device < 0 || o->device >= dev_count)
    return bail(err(POND_E_CUDA, "pond_incoh_create: no CUDA device %d", o->device));
  cudaError_t e = cudaSetDevice(o->device);
  if (e == cudaSuccess) e = pond::set_kernel_attributes();
  if (e == cudaSuccess) e = fb_dispatch(h->logR, true, FbArgs{}, nullptr, nullptr);
  if (e == cudaSuccess && o->ips_len) {
    const int logL = ilog2(o->ips_len);
    e = ips_dispatch(logL, true, nullptr, 0, nullptr, nullptr, nullptr);
    if (e == cudaSuccess)
      e = cudaMalloc(&h->stwL, std::max(1, pond::stage_tw_entries(o->ips_len)) * sizeof(float2));
    if (e == cudaSuccess) e = pond::launch_stage_tw(h->stwL, o->ips_len, nullptr);
    if (e == cudaSuccess) e = cudaMalloc(&h->ips, (o->ips_len / 2 + 1) * sizeof(double));
    if (e == cudaSuccess) e = cudaMemset(h->ips, 0, (o->ips_len / 2 + 1) * sizeof(double));
  }
  if (e == cudaSuccess) e = cudaMalloc(&h->d_delay, o->nchan * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&h->stw, std::max(1, pond::stage_tw_entries(1 << h->logR)) * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc(&h->psum, (size_t)pond::MAX_FOLD_PARTS * o->nbins * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&h->phits, (size_t)pond::MAX_FOLD_PARTS * o->nbins * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&h->prof_sum, o->nbins * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&h->prof_hits, o->nbins * sizeof(long long));
  for (auto& ev : h->ev)
    if (e == cudaSuccess) e = cudaEventCreate(&ev);
  if (e == cudaSuccess)
    e = cudaMemcpy(h->d_delay, h->delay.data(), o->nchan * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = pond::launch_stage_tw(h->stw, 1 << h->logR, nullptr);
  if (e == cudaSuccess) e = cudaMemset(h->prof_sum, 0, o->nbins * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(h->prof_hits, 0, o->nbins * sizeof(long long));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess)
    return bail(err(e == cudaErrorMemoryAllocation ? POND_E_OOM : POND_E_CUDA, "pond_incoh_create: %s",
                    cudaGetErrorString(e)));
  *out = h;
  return POND_OK;
}

extern "C" int pond_incoh_run(pond_incoh_t h, const int8_t* d_x, size_t nbytes, void* cuda_stream) {
  if (!h) return err(POND_E_ARG, "pond_incoh_run: null handle");
  const int ch = h->o.input_channels;
  if (nbytes % ch) return err(POND_E_ARG, "pond_incoh_run: %zu bytes split an N / S sample pair", nbytes);
  if (nbytes > 0 && (!d_x || (reinterpret_cast<uintptr_t>(d_x) & 15)))
    return err(POND_E_ARG, "pond_incoh_run: input must be a 16-byte aligned device pointer");
  ICK(cudaSetDevice(h->device));
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // a previous run on another stream must not still read the buffers this one rewrites
  if (h->ran && h->st != st) ICK(cudaStreamSynchronize(h->st));
  const long long R = 2ll * h->nch;
  const long long n = (long long)(nbytes / ch);
  const long long T = n / R / h->o.nint;
  const long long n_spec = T * h->o.nint;
  const long long t_first = std::max(0, -h->dmin);
  const long long n_out = std::max(0ll, T - std::max(0, h->dmax) - t_first);
  if ((size_t)(T * h->nch) > h->F_cap) {
    ICK(cudaStreamSynchronize(st));
    cudaFree(h->F);
    h->F = nullptr;
    h->F_cap = 0;
    ICK(cudaMalloc(&h->F, (size_t)T * h->nch * sizeof(float)));
    h->F_cap = (size_t)T * h->nch;
  }
  if ((size_t)n_out > h->D_cap) {
    ICK(cudaStreamSynchronize(st));
    cudaFree(h->D);
    h->D = nullptr;
    h->D_cap = 0;
    ICK(cudaMalloc(&h->D, (size_t)n_out * sizeof(float)));
    h->D_cap = (size_t)n_out;
  }
  int launches = 0;
  ICK(cudaEventRecord(h->ev[0], st));
  if (n_spec > 0) {
    FbArgs a{};
    a.x = d_x;
    a.n_spec = n_spec;
    const long long spp = (h->form == pond::FB_CID ? 1 : 2) * (long long)(pond::TILE / R);
    a.s_cta = std::max<long long>(spp, h->o.nint);
    a.lognint = h->lognint;
    a.form = h->form;
    a.F = h->F;
    ICK(fb_dispatch(h->logR, false, a, h->stw, st));
    ++launches;
  }
  ICK(cudaEventRecord(h->ev[1], st));
  if (n_out > 0) {
    const long long blocks = (n_out + pond::DD_TD - 1) / pond::DD_TD;
    pond::k_incoh_sum<<<(unsigned)blocks, pond::DD_WARPS * 32, h->nch * sizeof(int), st>>>(
        h->F, h->nch, h->d_delay, t_first, n_out, h->D);
    ICK(cudaGetLastError());
    ++launches;
  }
  ICK(cudaEventRecord(h->ev[2], st));
  ICK(cudaMemsetAsync(h->prof_sum, 0, h->o.nbins * sizeof(double), st));
  ICK(cudaMemsetAsync(h->prof_hits, 0, h->o.nbins * sizeof(long long), st));
  if (n_out > 0) {
    ICK(pond::launch_fold(h->D, n_out, t_first, h->inc, h->o.nbins, h->psum, h->phits, h->prof_sum, h->prof_hits,
                          st));
    launches += 2;
  }
  ICK(cudaEventRecord(h->ev[3], st));
  long long ips_chunks = 0;
  if (h->o.ips_len) {
    ips_chunks = n_out / h->o.ips_len;
    if (ips_chunks > 0) {
      ICK(ips_dispatch(ilog2(h->o.ips_len), false, h->D, ips_chunks, h->stwL, h->ips, st));
      ++launches;
    } else {
      ICK(cudaMemsetAsync(h->ips, 0, (h->o.ips_len / 2 + 1) * sizeof(double), st));
    }
  }
  ICK(cudaEventRecord(h->ev[4], st));
  h->ips_chunks = ips_chunks;
  h->st = st;
  h->ran = true;
  h->T = T;
  h->t_first = t_first;
  h->n_out = n_out;
  h->in_bytes = (double)n_spec * R * ch;
  h->launches = launches;
  return POND_OK;
}

extern "C" int pond_incoh_info_get(pond_incoh_t h, pond_incoh_info* info) {
  if (!h || !info) return err(POND_E_ARG, "pond_incoh_info_get: null pointer");
  if (int rc = wait_last(h)) return rc;
  *info = pond_incoh_info{};
  info->T = h->T;
  info->t_first = h->t_first;
  info->n_out = h->n_out;
  info->ips_chunks = h->ips_chunks;
  info->d_min = h->dmin;
  info->d_max = h->dmax;
  info->ts = h->ts;
  info->launches = h->launches;
  info->algo_bytes_filterbank = h->in_bytes + (double)h->T * h->nch * sizeof(float);
  info->algo_bytes_dedisperse = (double)h->n_out * h->nch * sizeof(float) + (double)h->n_out * sizeof(float);
  if (h->ran) {
    float ms[4] = {0.f, 0.f, 0.f, 0.f};
    for (int i = 0; i < 4; ++i) ICK(cudaEventElapsedTime(&ms[i], h->ev[i], h->ev[i + 1]));
    info->ms_filterbank = ms[0];
    info->ms_dedisperse = ms[1];
    info->ms_fold = ms[2];
    info->ms_ips = ms[3];
  }
  return POND_OK;
}

extern "C" int pond_incoh_filterbank(pond_incoh_t h, float* out, size_t cap, int64_t* T) {
  if (!h || !T) return err(POND_E_ARG, "pond_incoh_filterbank: null pointer");
  if (int rc = wait_last(h)) return rc;
  *T = h->T;
  const size_t need = (size_t)h->T * h->nch;
  if (cap < need) return err(POND_E_OVERRUN, "pond_incoh_filterbank: %zu floats needed, %zu given", need, cap);
  if (need > 0) {
    if (!out) return err(POND_E_ARG, "pond_incoh_filterbank: null output");
    ICK(cudaMemcpy(out, h->F, need * sizeof(float), cudaMemcpyDeviceToHost));
  }
  return POND_OK;
}

extern "C" int pond_incoh_series(pond_incoh_t h, float* out, size_t cap, int64_t* n_out, int64_t* t_first) {
  if (!h || !n_out || !t_first) return err(POND_E_ARG, "pond_incoh_series: null pointer");
  if (int rc = wait_last(h)) return rc;
  *n_out = h->n_out;
  *t_first = h->t_first;
  if (cap < (size_t)h->n_out)
    return err(POND_E_OVERRUN, "pond_incoh_series: %lld samples needed, %zu given", h->n_out, cap);
  if (h->n_out > 0) {
    if (!out) return err(POND_E_ARG, "pond_incoh_series: null output");
    ICK(cudaMemcpy(out, h->D, (size_t)h->n_out * sizeof(float), cudaMemcpyDeviceToHost));
  }
  return POND_OK;
}

extern "C" int pond_incoh_profile(pond_incoh_t h, double* sum, int64_t* hits) {
  if (!h || !sum || !hits) return err(POND_E_ARG, "pond_incoh_profile: null pointer");
  if (int rc = wait_last(h)) return rc;
  ICK(cudaMemcpy(sum, h->prof_sum, h->o.nbins * sizeof(double), cudaMemcpyDeviceToHost));
  ICK(cudaMemcpy(hits, h->prof_hits, h->o.nbins * sizeof(long long), cudaMemcpyDeviceToHost));
  return POND_OK;
}

extern "C" int pond_incoh_ips(pond_incoh_t h, double* out, int64_t* chunks) {
  if (!h || !out || !chunks) return err(POND_E_ARG, "pond_incoh_ips: null pointer");
  if (!h->o.ips_len) return err(POND_E_STATE, "pond_incoh_ips: the handle was created with ips_len = 0");
  if (int rc = wait_last(h)) return rc;
  *chunks = h->ips_chunks;
  ICK(cudaMemcpy(out, h->ips, (h->o.ips_len / 2 + 1) * sizeof(double), cudaMemcpyDeviceToHost));
  return POND_OK;
}

extern "C" int pond_incoh_delays(pond_incoh_t h, int32_t* out) {
  if (!h || !out) return err(POND_E_ARG, "pond_incoh_delays: null pointer");
  std::copy(h->delay.begin(), h->delay.end(), out);
  return POND_OK;
}

extern "C" int pond_incoh_destroy(pond_incoh_t h) {
  if (!h) return POND_OK;
  cudaSetDevice(h->device);
  if (h->ran) cudaStreamSynchronize(h->st);
  release(h);
  delete h;
  return POND_OK;
}
