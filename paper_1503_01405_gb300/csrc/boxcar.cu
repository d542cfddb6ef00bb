// Boxcar S/N single-pulse detector over the series of a batch of DM trials.
//
// The paper names automatic transient detection as future work (Sec. 5); this
// is the plain matched-filter search over the dedispersed series that the
// batched trials produce:
//   mu_d = median(T_d), sigma_d = 1.4826 median|T_d - mu_d| (exact order
//   statistics; an even count takes the FP64 mean of the two middle values),
//   S_w(d, t) = (sum_{i<w} T_d[t+i] - w mu_d) / (sigma_d sqrt(w)), w = 1..64
//   (powers of two), the sum accumulated in FP64 in index order,
//   s(d, t) = max_w S_w, w*(d, t) its smallest maximising width,
//   candidate: s >= threshold and no point within |dd| <= 2 trials and
//   |dt| <= w* samples has a larger s (an equal s wins when it comes earlier
//   in (trial, sample) order).
// Every floating-point step is one correctly rounded IEEE operation (explicit
// _rn intrinsics, no contraction), so the FP64 oracle reproduces each S value
// bit for bit and the integer decisions agree exactly.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "../../include/pond.h"
#include "pond_internal.h"

namespace pond {

constexpr int SEL_THREADS = 512;
constexpr int NW = 7;                       // widths 1, 2, 4, ..., 64
constexpr int WMAX = 64;
constexpr int BOX_THREADS = 256;

__device__ __forceinline__ unsigned f32_key(float v) {
  const unsigned u = __float_as_uint(v);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float f32_unkey(unsigned k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// k-th smallest (0-based) of n keys produced by key(i), MSB-first radix select
// with 8-bit digits; all threads of the CTA call it and get the same result.
template <typename K, int BITS, typename F>
__device__ K radix_select(long long n, long long k, F key, unsigned* hist, K* sh_prefix, long long* sh_k) {
  K prefix = 0, mask = 0;
  for (int shift = BITS - 8; shift >= 0; shift -= 8) {
    for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
      const K x = key(i);
      if ((x & mask) == prefix) atomicAdd(&hist[(unsigned)((x >> shift) & 0xff)], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      long long c = 0;
      int b = 0;
      for (; b < 255; ++b) {
        if (c + hist[b] > k) break;
        c += hist[b];
      }
      *sh_k = k - c;
      *sh_prefix = prefix | ((K)b << shift);
    }
    __syncthreads();
    k = *sh_k;
    prefix = *sh_prefix;
    mask |= (K)0xff << shift;
    __syncthreads();
  }
  return prefix;
}

// One CTA per trial: mu and sigma of series[d * stride + 0 .. n).
__global__ void __launch_bounds__(SEL_THREADS) k_robust_stats(const float* __restrict__ series, long long n,
                                                             long long stride, double* __restrict__ mu_out,
                                                             double* __restrict__ sig_out) {
  __shared__ unsigned hist[256];
  __shared__ unsigned long long shp;
  __shared__ long long shk;
  const float* T = series + (size_t)blockIdx.x * stride;
  auto k32 = [&](long long i) -> unsigned { return f32_key(T[i]); };
  unsigned* pu = reinterpret_cast<unsigned*>(&shp);
  double mu;
  {
    const float a = f32_unkey(radix_select<unsigned, 32>(n, (n - 1) / 2, k32, hist, pu, &shk));
    if (n % 2) {
      mu = (double)a;
    } else {
      const float b = f32_unkey(radix_select<unsigned, 32>(n, n / 2, k32, hist, pu, &shk));
      mu = __dmul_rn(__dadd_rn((double)a, (double)b), 0.5);
    }
  }
  // |T - mu| >= 0: its FP64 bit pattern orders like the value
  auto k64 = [&](long long i) -> unsigned long long {
    return (unsigned long long)__double_as_longlong(fabs(__dsub_rn((double)T[i], mu)));
  };
  double mad;
  {
    const double a = __longlong_as_double((long long)radix_select<unsigned long long, 64>(n, (n - 1) / 2, k64, hist,
                                                                                        &shp, &shk));
    if (n % 2) {
      mad = a;
    } else {
      const double b = __longlong_as_double((long long)radix_select<unsigned long long, 64>(n, n / 2, k64, hist,
                                                                                          &shp, &shk));
      mad = __dmul_rn(__dadd_rn(a, b), 0.5);
    }
  }
  if (threadIdx.x == 0) {
    mu_out[blockIdx.x] = mu;
    sig_out[blockIdx.x] = __dmul_rn(1.4826, mad);
  }
}

// s(d, t) and w*(d, t); grid (ceil(n / BOX_THREADS), ndm).
__global__ void __launch_bounds__(BOX_THREADS) k_boxcar(const float* __restrict__ series, long long n,
                                                       long long stride, const double* __restrict__ mu,
                                                       const double* __restrict__ sig, double* __restrict__ S,
                                                       unsigned char* __restrict__ W) {
  __shared__ float tile[BOX_THREADS + WMAX];
  const int d = blockIdx.y;
  const long long t0 = (long long)blockIdx.x * BOX_THREADS;
  const float* T = series + (size_t)d * stride;
  for (int i = threadIdx.x; i < BOX_THREADS + WMAX; i += BOX_THREADS)
    tile[i] = (t0 + i < n) ? T[t0 + i] : 0.f;
  __syncthreads();
  const long long t = t0 + threadIdx.x;
  if (t >= n) return;
  const double m = mu[d], sg = sig[d];
  double best = -INFINITY;
  int bw = 0;
  if (sg > 0) {
    double acc = 0.0;
    int done = 0;
#pragma unroll
    for (int q = 0; q < NW; ++q) {
      const int w = 1 << q;
      if (t + w > n) break;
      for (int i = done; i < w; ++i) acc = __dadd_rn(acc, (double)tile[threadIdx.x + i]);
      done = w;
      const double num = __dsub_rn(acc, __dmul_rn((double)w, m));
      const double s = __ddiv_rn(num, __dmul_rn(sg, __dsqrt_rn((double)w)));
      if (s > best) {
        best = s;
        bw = w;
      }
    }
  }
  S[(size_t)d * n + t] = best;
  W[(size_t)d * n + t] = (unsigned char)bw;
}

// Candidates: local maxima of s over |dd| <= 2 trials and |dt| <= w* samples.
__global__ void k_suppress(const double* __restrict__ S, const unsigned char* __restrict__ W, int ndm, long long n,
                           double thr, int radius, pond_cand* __restrict__ out, long long cap,
                           unsigned long long* __restrict__ count) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)ndm * n) return;
  const double s = S[idx];
  if (!(s >= thr)) return;
  const int d = (int)(idx / n);
  const long long t = idx - (long long)d * n;
  const int w = W[idx];
  const int d0 = max(0, d - radius), d1 = min(ndm - 1, d + radius);
  const long long a = max(0ll, t - w), b = min(n - 1, t + w);
  for (int dd = d0; dd <= d1; ++dd)
    for (long long tt = a; tt <= b; ++tt) {
      if (dd == d && tt == t) continue;
      const double o = S[(size_t)dd * n + tt];
      const bool earlier = dd < d || (dd == d && tt < t);
      if (o > s || (o == s && earlier)) return;
    }
  const unsigned long long k = atomicAdd(count, 1ull);
  if ((long long)k < cap) {
    pond_cand c;
    c.trial = d;
    c.width = w;
    c.index = t;
    c.snr = s;
    c.dm = 0.0;
    c.score = -1.f;
    c.reserved = 0;
    out[k] = c;
  }
}

int run_boxcar(const float* d_series, int ndm, long long n, long long stride, double thr, pond_cand* host_out,
               size_t cap, size_t* n_found, cudaStream_t st) {
  *n_found = 0;
  if (ndm <= 0 || n <= 0) return POND_OK;
  double *mu = nullptr, *sig = nullptr, *S = nullptr;
  unsigned char* W = nullptr;
  pond_cand* dc = nullptr;
  unsigned long long* cnt = nullptr;
  const long long dcap = std::max<long long>(1024, (long long)cap);
  auto cleanup = [&]() {
    cudaFree(mu);
    cudaFree(sig);
    cudaFree(S);
    cudaFree(W);
    cudaFree(dc);
    cudaFree(cnt);
  };
  cudaError_t e = cudaMalloc(&mu, ndm * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&sig, ndm * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&S, (size_t)ndm * n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&W, (size_t)ndm * n);
  if (e == cudaSuccess) e = cudaMalloc(&dc, dcap * sizeof(pond_cand));
  if (e == cudaSuccess) e = cudaMalloc(&cnt, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) {
    cleanup();
    return set_error(e == cudaErrorMemoryAllocation ? POND_E_OOM : POND_E_CUDA, cudaGetErrorString(e));
  }
  k_robust_stats<<<ndm, SEL_THREADS, 0, st>>>(d_series, n, stride, mu, sig);
  dim3 grid((unsigned)((n + BOX_THREADS - 1) / BOX_THREADS), (unsigned)ndm);
  k_boxcar<<<grid, BOX_THREADS, 0, st>>>(d_series, n, stride, mu, sig, S, W);
  const long long tot = (long long)ndm * n;
  k_suppress<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(S, W, ndm, n, thr, 2, dc, dcap, cnt);
  unsigned long long found = 0;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&found, cnt, sizeof found, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  std::vector<pond_cand> v;
  if (e == cudaSuccess) {
    v.resize((size_t)std::min<unsigned long long>(found, (unsigned long long)dcap));
    if (!v.empty()) e = cudaMemcpyAsync(v.data(), dc, v.size() * sizeof(pond_cand), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  cleanup();
  if (e != cudaSuccess) return set_error(POND_E_CUDA, cudaGetErrorString(e));
  if (found > (unsigned long long)dcap) return set_error(POND_E_OVERRUN, "boxcar: more candidates than capacity");
  std::sort(v.begin(), v.end(), [](const pond_cand& x, const pond_cand& y) {
    return x.trial != y.trial ? x.trial < y.trial : x.index < y.index;
  });
  *n_found = v.size();
  if (v.size() > cap) return set_error(POND_E_OVERRUN, "boxcar: more candidates than capacity");
  std::copy(v.begin(), v.end(), host_out);
  return POND_OK;
}

}  // namespace pond

extern "C" int pond_boxcar(const float* d_series, int32_t ndm, int64_t n, int64_t stride, double threshold,
                           pond_cand* out, size_t cap, size_t* n_found, void* cuda_stream) {
  if (!n_found || (cap > 0 && !out) || ndm < 0 || n < 0 || stride < n || (ndm > 0 && n > 0 && !d_series))
    return pond::set_error(POND_E_ARG, "pond_boxcar: bad argument");
  return pond::run_boxcar(d_series, ndm, n, stride, threshold, out, cap, n_found,
                          static_cast<cudaStream_t>(cuda_stream));
}
