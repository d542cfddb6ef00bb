// C ABI of the engine: planning, stream ingest, segment scheduling, outputs.
//
// The host side holds the overlap-save bookkeeping (PONDER Sec. 3.7): segment s
// starts at real sample s*S (S = 2 nchan S_c) and yields the channel samples
// g = s*S_c + m, n_past <= m < M - n_fut.  The last n_ov = N - S real samples
// of the stream seen so far are kept in a device carry buffer for the next
// segment.  Every arithmetic step on the data runs in the kernels of kernels.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/pond.h"
#include "fft_block.cuh"
#include "pond_internal.h"

using namespace pond;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(e_ == cudaErrorMemoryAllocation ? POND_E_OOM : POND_E_CUDA, "%s: %s (%s:%d)", #call, \
                  cudaGetErrorString(e_), __FILE__, __LINE__);                            \
  } while (0)

constexpr double K_DM = 1.0 / 2.41e-4;        // s MHz^2 (Eq. 1 constant)
constexpr long long STAGE_BYTES = 64ll << 20; // host-push staging chunk
constexpr long long TS_RING = 1ll << 22;      // time-series samples held on the device

enum Stage { ST_F1 = 0, ST_F2, ST_I1, ST_I2, ST_FOLD, ST_DEC, ST_COUNT };
const char* kStageName[POND_NSTAGE] = {"fwd_cols_unpack", "fwd_rows_split_chirp", "inv_cols",
                                       "inv_rows_detect", "fold", "decimate", "", ""};

int ilog2ll(long long v) {
  int r = 0;
  while ((1ll << r) < v) ++r;
  return r;
}

long long gcd_ll(long long a, long long b) {
  while (b) {
    long long t = a % b;
    a = b;
    b = t;
  }
  return a;
}

// Events bracketing the stages of one segment (timing mode).
struct SegEvents {
  cudaEvent_t e[ST_COUNT + 1];
};

}  // namespace

int pond::set_error(int code, const char* msg) { return fail(code, "%s", msg); }

struct pond_s {
  // parameters
  double f0, bw, fs, dm, period;
  int nbins;
  long long t_dec_ns;
  int epoch_day;
  double epoch_sec;
  int want_voltages, timing, device;
  // geometry
  Geom g;
  double dtc, inc;
  long long dec_num, dec_den;
  int sgn;
  // streams
  cudaStream_t st = nullptr, cst = nullptr;
  cudaEvent_t ev_done = nullptr, ev_caller = nullptr;
  cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_used[2] = {nullptr, nullptr};
  // device buffers
  float2* bufA = nullptr;
  float2* bufB = nullptr;
  float* P = nullptr;
  float2* tw = nullptr;                     // stage twiddle tables of R1, R2, Q1, Q2
  const float2 *stwR1 = nullptr, *stwR2 = nullptr, *stwQ1 = nullptr, *stwQ2 = nullptr;
  float2* tw2buf = nullptr;
  Tw2 twL, tw2L, twM;   // exp(-2 pi i e/L), exp(-2 pi i e/(2L)), exp(+2 pi i e/M)
  ChirpAnchor* anc = nullptr;
  long long nanc = 0;
  int clog = 0;
  double* prof_sum = nullptr;
  long long* prof_hits = nullptr;
  double* psum = nullptr;
  int* phits = nullptr;
  float* ts = nullptr;
  int* ts_cnt = nullptr;
  int8_t* carry[2] = {nullptr, nullptr};
  int carry_cur = 0;
  int8_t* stage[2] = {nullptr, nullptr};
  int stage_next = 0;
  float2* vbuf = nullptr;
  long long v_cap = 0;
  // stream state (real-sample indices)
  long long total_in = 0, seg_start = 0, carry_pos = 0, seg_index = 0;
  bool flushed = false;
  long long outputs = 0;
  // time series: samples [ts_drained, ts_written_hi) live in the device ring;
  // [ts_drained, ts_complete) are complete
  long long ts_first = -1, ts_drained = 0, ts_hi = 0, ts_complete = 0;
  std::vector<float> ts_host;
  std::vector<int32_t> ts_host_cnt;
  long long ts_host_first = 0;
  // voltages: device [v_base, v_base + v_len), host spill before that
  long long v_len = 0, v_base = -1;
  std::vector<std::vector<float>> v_host;
  long long v_host_first = -1;
  // timing
  std::vector<SegEvents> ev_pending;
  std::vector<cudaEvent_t> ev_pool;
  SegEvents ev_cur;
  double stage_ms[POND_NSTAGE] = {0};
  long long stage_launches[POND_NSTAGE] = {0};
};

namespace {

int validate(const pond_opts* o) {
  if (!o) return fail(POND_E_ARG, "null options");
  if (!(o->f0_mhz > 0) || !(o->bw_mhz != 0) || !(std::fabs(o->bw_mhz) < 2 * o->f0_mhz) || !(o->fs_hz > 0))
    return fail(POND_E_ARG, "bad band: f0=%g bw=%g fs=%g", o->f0_mhz, o->bw_mhz, o->fs_hz);
  if (std::fabs(o->fs_hz - 2.0 * std::fabs(o->bw_mhz) * 1e6) > 1e-6 * o->fs_hz)
    return fail(POND_E_ARG, "fs must equal 2|bw| (real Nyquist sampling)");
  if (o->fs_hz != std::floor(o->fs_hz) || o->fs_hz > 9e15) return fail(POND_E_ARG, "fs must be a whole number of Hz");
  if (!(o->dm >= 0) || !std::isfinite(o->dm)) return fail(POND_E_ARG, "DM must be >= 0");
  if (!(o->period_s > 0) || !std::isfinite(o->period_s)) return fail(POND_E_ARG, "period must be > 0");
  if (o->nbins < 1 || o->nbins > MAX_NBINS) return fail(POND_E_ARG, "nbins must be 1..%d", MAX_NBINS);
  if (o->nfft < 4 || (o->nfft & (o->nfft - 1))) return fail(POND_E_NFFT, "nfft must be a power of two");
  if (o->nchan < 1 || (o->nchan & (o->nchan - 1)) || (o->nfft / 2) % o->nchan)
    return fail(POND_E_NCHAN, "nchan must be a power of two dividing nfft/2");
  if (o->precision != POND_FP32) return fail(POND_E_UNIMPLEMENTED, "only POND_FP32 is built");
  return POND_OK;
}

int geometry(const pond_opts* o, Geom* g, double* dtc) {
  g->N = o->nfft;
  g->L = o->nfft / 2;
  g->nchan = o->nchan;
  g->M = g->L / o->nchan;
  g->logL = ilog2ll(g->L);
  g->logM = ilog2ll(g->M);
  *dtc = 2.0 * o->nchan / o->fs_hz;
  const double half = std::fabs(o->bw_mhz) / 2.0;
  const double f_lo = o->f0_mhz - half, f_hi = o->f0_mhz + half;
  const double past = K_DM * o->dm * (std::pow(o->f0_mhz, -2) - std::pow(f_hi, -2));
  const double fut = K_DM * o->dm * (std::pow(f_lo, -2) - std::pow(o->f0_mhz, -2));
  g->n_past = (long long)std::ceil(past / *dtc);
  g->n_fut = (long long)std::ceil(fut / *dtc);
  g->S_c = g->M - g->n_past - g->n_fut;
  if (g->S_c <= 0)
    return fail(POND_E_NFFT, "nfft %lld does not exceed the overlap (n_past %lld + n_fut %lld >= M %lld)",
                (long long)o->nfft, g->n_past, g->n_fut, g->M);
  g->S = 2ll * o->nchan * g->S_c;
  // forward passes: L = R1 * R2, 4 <= R <= 4096, with R2 <= M so that every
  // sub-channel spans whole columns of F2's row layout
  if (g->logL < 4 || g->logL > 24) return fail(POND_E_NFFT, "nfft must be in 2^5 .. 2^25");
  g->logR2 = std::min(g->logL / 2, g->logM);
  g->logR1 = g->logL - g->logR2;
  if (g->logR1 > 12) {
    g->logR1 = 12;
    g->logR2 = g->logL - 12;
  }
  // inverse passes: M = Q1 * Q2 with nchan * Q1 <= TILE and Q1 <= R2
  const int lognch = ilog2ll(o->nchan);
  g->logQ1 = std::min(std::min((g->logM + 1) / 2, 13 - lognch), std::min(12, g->logR2));
  g->logQ2 = g->logM - g->logQ1;
  if (g->logR2 < 2 || g->logR2 > g->logM || g->logQ1 < 2 || g->logQ2 < 2 || g->logQ2 > 12)
    return fail(POND_E_NCHAN, "unsupported nchan %d for nfft %lld (need M >= 16 and nchan*4 <= 8192)",
                o->nchan, (long long)o->nfft);
  return POND_OK;
}

// Record boundary event `i` (0 = before F1, i = after stage i-1) of the current segment.
int record(pond_t h, int i) {
  if (!h->timing) return POND_OK;
  cudaEvent_t e;
  if (!h->ev_pool.empty()) {
    e = h->ev_pool.back();
    h->ev_pool.pop_back();
  } else {
    CK(cudaEventCreate(&e));
  }
  CK(cudaEventRecord(e, h->st));
  h->ev_cur.e[i] = e;
  if (i == ST_COUNT) h->ev_pending.push_back(h->ev_cur);
  return POND_OK;
}

int collect_timing(pond_t h) {
  if (!h->timing) return POND_OK;
  CK(cudaStreamSynchronize(h->st));
  for (auto& se : h->ev_pending) {
    for (int i = 0; i < ST_COUNT; ++i) {
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, se.e[i], se.e[i + 1]));
      h->stage_ms[i] += ms;
      h->stage_launches[i] += 1;
    }
    for (int i = 0; i <= ST_COUNT; ++i) h->ev_pool.push_back(se.e[i]);
  }
  h->ev_pending.clear();
  return POND_OK;
}

// Move completed time-series samples from the device ring to the host vector.
int spill_ts(pond_t h) {
  if (h->ts_first < 0 || h->ts_complete <= h->ts_drained) return POND_OK;
  CK(cudaStreamSynchronize(h->st));
  const long long n = h->ts_complete - h->ts_drained;
  if (h->ts_host.empty()) h->ts_host_first = h->ts_drained;
  const size_t off = h->ts_host.size();
  h->ts_host.resize(off + n);
  h->ts_host_cnt.resize(off + n);
  long long j = h->ts_drained;
  long long done = 0;
  while (done < n) {
    const long long slot = j % TS_RING;
    const long long run = std::min(n - done, TS_RING - slot);
    CK(cudaMemcpyAsync(h->ts_host.data() + off + done, h->ts + slot, run * sizeof(float),
                       cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemcpyAsync(h->ts_host_cnt.data() + off + done, h->ts_cnt + slot, run * sizeof(int),
                       cudaMemcpyDeviceToHost, h->st));
    CK(cudaMemsetAsync(h->ts + slot, 0, run * sizeof(float), h->st));
    CK(cudaMemsetAsync(h->ts_cnt + slot, 0, run * sizeof(int), h->st));
    done += run;
    j += run;
  }
  CK(cudaStreamSynchronize(h->st));
  h->ts_drained = h->ts_complete;
  return POND_OK;
}

int spill_voltages(pond_t h) {
  if (!h->want_voltages || h->v_len == 0) return POND_OK;
  CK(cudaStreamSynchronize(h->st));
  if (h->v_host_first < 0) h->v_host_first = h->v_base;
  for (int c = 0; c < h->g.nchan; ++c) {
    auto& vec = h->v_host[c];
    const size_t off = vec.size();
    vec.resize(off + 2 * h->v_len);
    CK(cudaMemcpyAsync(vec.data() + off, h->vbuf + (size_t)c * h->v_cap, h->v_len * sizeof(float2),
                       cudaMemcpyDeviceToHost, h->st));
  }
  CK(cudaStreamSynchronize(h->st));
  h->v_base += h->v_len;
  h->v_len = 0;
  return POND_OK;
}

// Process one segment (index s) whose input is `in`; m_hi bounds the valid span.
int run_segment(pond_t h, SegIn in, long long s, long long m_hi) {
  const Geom& g = h->g;
  const long long g0 = s * g.S_c + g.n_past;     // first output of this segment
  const long long nv = m_hi - g.n_past;
  if (nv <= 0) return POND_OK;
  // time-series samples touched by this segment
  const long long j_lo = (g0 * h->dec_den) / h->dec_num;
  const long long j_hi = ((g0 + nv - 1) * h->dec_den) / h->dec_num;
  if (h->ts_first < 0) {
    h->ts_first = j_lo;
    h->ts_drained = j_lo;
    h->ts_complete = j_lo;
  }
  if (j_hi - h->ts_drained >= TS_RING) {
    int rc = spill_ts(h);
    if (rc) return rc;
  }
  float2* vout = nullptr;
  if (h->want_voltages) {
    if (h->v_base < 0) h->v_base = g0;
    if (h->v_len + nv > h->v_cap) {
      int rc = spill_voltages(h);
      if (rc) return rc;
    }
    vout = h->vbuf;
  }
  int rc;
  if ((rc = record(h, 0))) return rc;
  {  // F1 may load 8 bytes (4 columns of a row) at a time when both runs allow it
    const int nl1 = std::min(TILE >> g.logR2, 1 << g.logR1);
    in.vec8 = (nl1 % 4 == 0) && ((uintptr_t)in.a % 8 == 0) && (in.a_len % 8 == 0) &&
              (in.b_len == 0 || (uintptr_t)in.b % 8 == 0);
  }
  CK(launch_fwd_cols(g, in, h->bufA, h->twL, h->stwR2, h->st));
  if ((rc = record(h, 1 + ST_F1))) return rc;
  CK(launch_fwd_rows(g, h->bufA, h->bufB, h->tw2L, h->anc, h->clog, 1, h->stwR1, h->st));
  if ((rc = record(h, 1 + ST_F2))) return rc;
  CK(launch_inv_cols(g, h->bufB, h->bufA, h->twM, h->stwQ2, h->st));
  if ((rc = record(h, 1 + ST_I1))) return rc;
  CK(launch_inv_rows(g, h->bufA, h->P, vout, h->v_cap, h->v_len, (int)m_hi, h->stwQ1, h->st));
  if ((rc = record(h, 1 + ST_I2))) return rc;
  CK(launch_fold(h->P, nv, g0, h->inc, h->nbins, h->psum, h->phits, h->prof_sum, h->prof_hits, h->st));
  if ((rc = record(h, 1 + ST_FOLD))) return rc;
  CK(launch_decimate(h->P, nv, g0, h->dec_num, h->dec_den, j_lo, j_hi - j_lo + 1, h->ts, h->ts_cnt, TS_RING,
                     h->st));
  if ((rc = record(h, 1 + ST_DEC))) return rc;
  if (h->want_voltages) h->v_len += nv;
  h->ts_hi = std::max(h->ts_hi, j_hi + 1);
  // samples before the next segment's first output are complete
  const long long g_next = g0 + nv;
  h->ts_complete = std::max(h->ts_complete, (g_next * h->dec_den) / h->dec_num);
  h->outputs += nv;
  h->seg_index = s + 1;
  return POND_OK;
}

// Ingest n samples at device pointer d (already ordered on h->st).
int ingest_device(pond_t h, const int8_t* d, long long n) {
  const Geom& g = h->g;
  const long long end = h->total_in + n;
  while (h->seg_start + g.N <= end) {
    SegIn in;
    if (h->seg_start < h->total_in) {
      in.a = h->carry[h->carry_cur] + (h->seg_start - h->carry_pos);
      in.a_len = h->total_in - h->seg_start;
      in.b = d;
      in.b_len = g.N - in.a_len;
    } else {
      in.a = d + (h->seg_start - h->total_in);
      in.a_len = g.N;
      in.b = nullptr;
      in.b_len = 0;
    }
    const long long s = h->seg_start / g.S;
    int rc = run_segment(h, in, s, g.M - g.n_fut);
    if (rc) return rc;
    h->seg_start += g.S;
  }
  // keep [seg_start, end) for the next segment
  int8_t* dst = h->carry[1 - h->carry_cur];
  long long w = 0;
  if (h->seg_start < h->total_in) {
    const long long old = h->total_in - h->seg_start;
    CK(cudaMemcpyAsync(dst, h->carry[h->carry_cur] + (h->seg_start - h->carry_pos), old,
                       cudaMemcpyDeviceToDevice, h->st));
    w = old;
    if (n > 0) CK(cudaMemcpyAsync(dst + w, d, n, cudaMemcpyDeviceToDevice, h->st));
  } else if (end > h->seg_start) {
    CK(cudaMemcpyAsync(dst, d + (h->seg_start - h->total_in), end - h->seg_start, cudaMemcpyDeviceToDevice,
                       h->st));
  }
  h->carry_cur = 1 - h->carry_cur;
  h->carry_pos = h->seg_start;
  h->total_in = end;
  return POND_OK;
}

void destroy_all(pond_t h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st);
  cudaFree(h->bufA);
  cudaFree(h->bufB);
  cudaFree(h->P);
  cudaFree(h->tw);
  cudaFree(h->tw2buf);
  cudaFree(h->anc);
  cudaFree(h->prof_sum);
  cudaFree(h->prof_hits);
  cudaFree(h->psum);
  cudaFree(h->phits);
  cudaFree(h->ts);
  cudaFree(h->ts_cnt);
  cudaFree(h->carry[0]);
  cudaFree(h->carry[1]);
  cudaFree(h->stage[0]);
  cudaFree(h->stage[1]);
  cudaFree(h->vbuf);
  for (auto& se : h->ev_pending)
    for (int i = 0; i <= ST_COUNT; ++i) cudaEventDestroy(se.e[i]);
  for (auto e : h->ev_pool) cudaEventDestroy(e);
  for (int i = 0; i < 2; ++i) {
    if (h->ev_copied[i]) cudaEventDestroy(h->ev_copied[i]);
    if (h->ev_used[i]) cudaEventDestroy(h->ev_used[i]);
  }
  if (h->ev_done) cudaEventDestroy(h->ev_done);
  if (h->ev_caller) cudaEventDestroy(h->ev_caller);
  if (h->st) cudaStreamDestroy(h->st);
  if (h->cst) cudaStreamDestroy(h->cst);
  delete h;
}

int plan_impl(pond_t* out, const pond_opts* o) {
  int rc = validate(o);
  if (rc) return rc;
  pond_t h = new pond_s();
  h->f0 = o->f0_mhz;
  h->bw = o->bw_mhz;
  h->fs = o->fs_hz;
  h->dm = o->dm;
  h->period = o->period_s;
  h->nbins = o->nbins;
  h->epoch_day = o->epoch_mjd_day;
  h->epoch_sec = o->epoch_mjd_sec;
  h->want_voltages = o->want_voltages;
  h->timing = o->timing;
  h->device = o->device;
  h->sgn = o->bw_mhz > 0 ? 1 : -1;
  rc = geometry(o, &h->g, &h->dtc);
  if (rc) {
    delete h;
    return rc;
  }
  h->inc = h->dtc / o->period_s;
  const double tdec = o->t_dec_s > 0 ? o->t_dec_s : 61.44e-6;
  h->t_dec_ns = (long long)std::llround(tdec * 1e9);
  if (h->t_dec_ns <= 0) {
    delete h;
    return fail(POND_E_ARG, "t_dec must be >= 1 ns");
  }
  {  // D = t_dec fs / (2 nchan) channel samples, exact rational num/den
    long long num = h->t_dec_ns, den = 1000000000ll * 2 * o->nchan;
    long long fsi = (long long)o->fs_hz;
    long long gq = gcd_ll(fsi, den);
    fsi /= gq;
    den /= gq;
    long long g2 = gcd_ll(num, den);
    num /= g2;
    den /= g2;
    if (num > (1ll << 40) / std::max(1ll, fsi)) {
      delete h;
      return fail(POND_E_ARG, "t_dec too long");
    }
    num *= fsi;
    h->dec_num = num;
    h->dec_den = den;
  }
  const Geom& g = h->g;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    delete h;
    return fail(POND_E_CUDA, "no CUDA device");
  }
  if (o->device < 0 || o->device >= ndev) {
    delete h;
    return fail(POND_E_ARG, "device %d out of range", o->device);
  }
#define CKD(call)                   \
  do {                              \
    cudaError_t e_ = (call);        \
    if (e_ != cudaSuccess) {        \
      int c_ = fail(e_ == cudaErrorMemoryAllocation ? POND_E_OOM : POND_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
      destroy_all(h);               \
      return c_;                    \
    }                               \
  } while (0)
  CKD(cudaSetDevice(o->device));
  CKD(cudaDeviceGetAttribute(&h->g.sms, cudaDevAttrMultiProcessorCount, o->device));
  CKD(set_kernel_attributes());
  CKD(cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking));
  CKD(cudaStreamCreateWithFlags(&h->cst, cudaStreamNonBlocking));
  CKD(cudaEventCreateWithFlags(&h->ev_done, cudaEventDisableTiming));
  CKD(cudaEventCreateWithFlags(&h->ev_caller, cudaEventDisableTiming));
  for (int i = 0; i < 2; ++i) {
    CKD(cudaEventCreateWithFlags(&h->ev_copied[i], cudaEventDisableTiming));
    CKD(cudaEventCreateWithFlags(&h->ev_used[i], cudaEventDisableTiming));
  }
  CKD(cudaMalloc(&h->bufA, g.L * sizeof(float2)));
  CKD(cudaMalloc(&h->bufB, g.L * sizeof(float2)));
  CKD(cudaMalloc(&h->P, g.M * sizeof(float)));
  {
    const int n1 = stage_tw_entries(1 << g.logR1), n2 = stage_tw_entries(1 << g.logR2);
    const int n3 = stage_tw_entries(1 << g.logQ1), n4 = stage_tw_entries(1 << g.logQ2);
    CKD(cudaMalloc(&h->tw, (size_t)std::max(1, n1 + n2 + n3 + n4) * sizeof(float2)));
    h->stwR1 = h->tw;
    h->stwR2 = h->stwR1 + n1;
    h->stwQ1 = h->stwR2 + n2;
    h->stwQ2 = h->stwQ1 + n3;
  }
  {  // two-level twiddle tables for exponents below L, 2L and M
    auto nhi = [](int logn) { return logn > TW2_LOG ? (1ll << (logn - TW2_LOG)) : 1ll; };
    const long long total = 3ll * TW2_LO + nhi(g.logL) + nhi(g.logL + 1) + nhi(g.logM);
    CKD(cudaMalloc(&h->tw2buf, total * sizeof(float2)));
    float2* p = h->tw2buf;
    h->twL = {p, p + TW2_LO};
    p += TW2_LO + nhi(g.logL);
    h->tw2L = {p, p + TW2_LO};
    p += TW2_LO + nhi(g.logL + 1);
    h->twM = {p, p + TW2_LO};
  }
  const double du = o->fs_hz / (double)o->nfft * 1e-6;
  const double half = std::fabs(o->bw_mhz) / 2.0;
  const double alpha = K_DM * 1e6 * o->dm / (o->f0_mhz * o->f0_mhz);
  {  // anchor span: the quartic Taylor term alpha f0^2/(f0+f)^5 (du span/2)^4 <= 1e-9 cycles
    const double fmin = o->f0_mhz - half;
    const double c4 = alpha * o->f0_mhz * o->f0_mhz / std::pow(fmin, 5);
    h->clog = CHIRP_LOG_MAX;
    while (h->clog > 0 && c4 * std::pow(du * (double)(1ll << (h->clog - 1)), 4) > 1e-9) --h->clog;
  }
  h->nanc = (g.L + (1ll << h->clog) - 1) >> h->clog;
  CKD(cudaMalloc(&h->anc, h->nanc * sizeof(ChirpAnchor)));
  CKD(cudaMalloc(&h->prof_sum, h->nbins * sizeof(double)));
  CKD(cudaMalloc(&h->prof_hits, h->nbins * sizeof(long long)));
  CKD(cudaMalloc(&h->psum, (size_t)MAX_FOLD_PARTS * h->nbins * sizeof(double)));
  CKD(cudaMalloc(&h->phits, (size_t)MAX_FOLD_PARTS * h->nbins * sizeof(int)));
  CKD(cudaMalloc(&h->ts, TS_RING * sizeof(float)));
  CKD(cudaMalloc(&h->ts_cnt, TS_RING * sizeof(int)));
  CKD(cudaMalloc(&h->carry[0], g.N));
  CKD(cudaMalloc(&h->carry[1], g.N));
  if (h->want_voltages) {
    h->v_cap = std::max<long long>(4 * g.S_c, 1 << 16);
    CKD(cudaMalloc(&h->vbuf, (size_t)g.nchan * h->v_cap * sizeof(float2)));
    h->v_host.resize(g.nchan);
  }
  CKD(cudaMemsetAsync(h->prof_sum, 0, h->nbins * sizeof(double), h->st));
  CKD(cudaMemsetAsync(h->prof_hits, 0, h->nbins * sizeof(long long), h->st));
  CKD(cudaMemsetAsync(h->ts, 0, TS_RING * sizeof(float), h->st));
  CKD(cudaMemsetAsync(h->ts_cnt, 0, TS_RING * sizeof(int), h->st));
  CKD(launch_tables(h->anc, h->nanc, h->clog, du, half, o->f0_mhz, alpha, h->sgn, h->st));
  CKD(launch_stage_tw(const_cast<float2*>(h->stwR1), 1 << g.logR1, h->st));
  CKD(launch_stage_tw(const_cast<float2*>(h->stwR2), 1 << g.logR2, h->st));
  CKD(launch_stage_tw(const_cast<float2*>(h->stwQ1), 1 << g.logQ1, h->st));
  CKD(launch_stage_tw(const_cast<float2*>(h->stwQ2), 1 << g.logQ2, h->st));
  CKD(launch_tw2(const_cast<float2*>(h->twL.lo), const_cast<float2*>(h->twL.hi), g.logL, -1, h->st));
  CKD(launch_tw2(const_cast<float2*>(h->tw2L.lo), const_cast<float2*>(h->tw2L.hi), g.logL + 1, -1, h->st));
  CKD(launch_tw2(const_cast<float2*>(h->twM.lo), const_cast<float2*>(h->twM.hi), g.logM, +1, h->st));
  CKD(cudaStreamSynchronize(h->st));
#undef CKD
  *out = h;
  return POND_OK;
}

int caller_wait(pond_t h, cudaStream_t cs) {
  // the handle's stream waits for work the caller queued before this call
  CK(cudaEventRecord(h->ev_caller, cs));
  CK(cudaStreamWaitEvent(h->st, h->ev_caller, 0));
  return POND_OK;
}

int caller_release(pond_t h, cudaStream_t cs) {
  // the caller's later work waits for what this call queued
  CK(cudaEventRecord(h->ev_done, h->st));
  CK(cudaStreamWaitEvent(cs, h->ev_done, 0));
  return POND_OK;
}

}  // namespace

extern "C" {

int pond_plan(pond_t* out, double f0_mhz, double bw_mhz, double fs_hz, double dm, int64_t nfft, int32_t nchan,
              int32_t nbins, double period_s) {
  pond_opts o;
  memset(&o, 0, sizeof o);
  o.f0_mhz = f0_mhz;
  o.bw_mhz = bw_mhz;
  o.fs_hz = fs_hz;
  o.dm = dm;
  o.nfft = nfft;
  o.nchan = nchan;
  o.nbins = nbins;
  o.period_s = period_s;
  return pond_plan_ex(out, &o);
}

int pond_plan_ex(pond_t* out, const pond_opts* opts) {
  if (!out) return fail(POND_E_ARG, "null handle pointer");
  *out = nullptr;
  g_last_error.clear();
  return plan_impl(out, opts);
}

int pond_push_device(pond_t h, const int8_t* d_x, size_t n, void* cuda_stream) {
  if (!h) return fail(POND_E_ARG, "null handle");
  if (h->flushed) return fail(POND_E_STATE, "push after flush");
  if (n == 0) return POND_OK;
  if (!d_x) return fail(POND_E_ARG, "null data");
  CK(cudaSetDevice(h->device));
  cudaStream_t cs = (cudaStream_t)cuda_stream;
  int rc = caller_wait(h, cs);
  if (rc) return rc;
  rc = ingest_device(h, d_x, (long long)n);
  if (rc) return rc;
  return caller_release(h, cs);
}

int pond_push(pond_t h, const int8_t* x, size_t n) {
  if (!h) return fail(POND_E_ARG, "null handle");
  if (h->flushed) return fail(POND_E_STATE, "push after flush");
  if (n == 0) return POND_OK;
  if (!x) return fail(POND_E_ARG, "null data");
  CK(cudaSetDevice(h->device));
  if (!h->stage[0]) {
    CK(cudaMalloc(&h->stage[0], STAGE_BYTES));
    CK(cudaMalloc(&h->stage[1], STAGE_BYTES));
    CK(cudaEventRecord(h->ev_used[0], h->st));
    CK(cudaEventRecord(h->ev_used[1], h->st));
  }
  cudaEvent_t last = nullptr;
  for (size_t off = 0; off < n; off += STAGE_BYTES) {
    const long long len = std::min<long long>(STAGE_BYTES, (long long)(n - off));
    const int i = h->stage_next;
    h->stage_next ^= 1;
    CK(cudaStreamWaitEvent(h->cst, h->ev_used[i], 0));
    CK(cudaMemcpyAsync(h->stage[i], x + off, len, cudaMemcpyHostToDevice, h->cst));
    CK(cudaEventRecord(h->ev_copied[i], h->cst));
    CK(cudaStreamWaitEvent(h->st, h->ev_copied[i], 0));
    int rc = ingest_device(h, h->stage[i], len);
    if (rc) return rc;
    CK(cudaEventRecord(h->ev_used[i], h->st));
    last = h->ev_copied[i];
  }
  // the caller's buffer is free once the copies have landed
  if (last) CK(cudaEventSynchronize(last));
  return POND_OK;
}

int pond_flush(pond_t h) {
  if (!h) return fail(POND_E_ARG, "null handle");
  if (h->flushed) return POND_OK;
  CK(cudaSetDevice(h->device));
  const Geom& g = h->g;
  const long long total_c = h->total_in / (2ll * g.nchan);
  const long long g_end = total_c - g.n_fut;
  while (h->seg_start / (2ll * g.nchan) + g.n_past < g_end) {
    SegIn in;
    in.a = h->carry[h->carry_cur] + (h->seg_start - h->carry_pos);
    in.a_len = std::max(0ll, h->total_in - h->seg_start);
    in.b = nullptr;
    in.b_len = 0;
    const long long s = h->seg_start / g.S;
    const long long m_hi = std::min(g.M - g.n_fut, g_end - s * g.S_c);
    int rc = run_segment(h, in, s, m_hi);
    if (rc) return rc;
    h->seg_start += g.S;
  }
  h->flushed = true;
  if (h->ts_first >= 0) h->ts_complete = h->ts_hi;
  CK(cudaStreamSynchronize(h->st));
  return POND_OK;
}

int pond_sync(pond_t h) {
  if (!h) return fail(POND_E_ARG, "null handle");
  CK(cudaSetDevice(h->device));
  CK(cudaStreamSynchronize(h->st));
  return POND_OK;
}

int pond_reset(pond_t h) {
  if (!h) return fail(POND_E_ARG, "null handle");
  CK(cudaSetDevice(h->device));
  int rc = collect_timing(h);
  if (rc) return rc;
  CK(cudaStreamSynchronize(h->st));
  CK(cudaMemsetAsync(h->prof_sum, 0, h->nbins * sizeof(double), h->st));
  CK(cudaMemsetAsync(h->prof_hits, 0, h->nbins * sizeof(long long), h->st));
  CK(cudaMemsetAsync(h->ts, 0, TS_RING * sizeof(float), h->st));
  CK(cudaMemsetAsync(h->ts_cnt, 0, TS_RING * sizeof(int), h->st));
  CK(cudaStreamSynchronize(h->st));
  h->total_in = h->seg_start = h->carry_pos = h->seg_index = 0;
  h->carry_cur = 0;
  h->flushed = false;
  h->outputs = 0;
  h->ts_first = -1;
  h->ts_drained = h->ts_hi = h->ts_complete = 0;
  h->ts_host.clear();
  h->ts_host_cnt.clear();
  h->ts_host_first = 0;
  h->v_len = 0;
  h->v_base = -1;
  for (auto& v : h->v_host) v.clear();
  h->v_host_first = -1;
  return POND_OK;
}

int pond_profile(pond_t h, double* sum, int64_t* hits, pond_meta* meta) {
  if (!h) return fail(POND_E_ARG, "null handle");
  CK(cudaSetDevice(h->device));
  CK(cudaStreamSynchronize(h->st));
  if (sum) CK(cudaMemcpyAsync(sum, h->prof_sum, h->nbins * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  if (hits) CK(cudaMemcpyAsync(hits, h->prof_hits, h->nbins * sizeof(long long), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (meta) {
    meta->epoch_mjd_day = h->epoch_day;
    meta->epoch_mjd_sec = h->epoch_sec;
    meta->period_s = h->period;
    meta->dm = h->dm;
    meta->dtc_s = h->dtc;
    meta->first_g = h->g.n_past;
    meta->nsamples = h->outputs;
    meta->nbins = h->nbins;
  }
  return POND_OK;
}

int pond_timeseries(pond_t h, float* out, int32_t* counts, size_t cap, size_t* n_out, int64_t* first_index) {
  if (!h || !n_out || !first_index || (cap > 0 && !out)) return fail(POND_E_ARG, "null argument");
  CK(cudaSetDevice(h->device));
  *n_out = 0;
  *first_index = h->ts_host.empty() ? std::max(h->ts_drained, 0ll) : h->ts_host_first;
  if (h->ts_first < 0) return POND_OK;
  int rc = spill_ts(h);
  if (rc) return rc;
  const size_t n = std::min(cap, h->ts_host.size());
  if (n) {
    memcpy(out, h->ts_host.data(), n * sizeof(float));
    if (counts) memcpy(counts, h->ts_host_cnt.data(), n * sizeof(int32_t));
    *first_index = h->ts_host_first;
    h->ts_host.erase(h->ts_host.begin(), h->ts_host.begin() + n);
    h->ts_host_cnt.erase(h->ts_host_cnt.begin(), h->ts_host_cnt.begin() + n);
    h->ts_host_first += (long long)n;
  }
  *n_out = n;
  return POND_OK;
}

int pond_voltages(pond_t h, float* out_c, size_t cap, size_t* n_out, int64_t* first_g) {
  if (!h || !n_out || !first_g || (cap > 0 && !out_c)) return fail(POND_E_ARG, "null argument");
  if (!h->want_voltages) return fail(POND_E_STATE, "plan made without want_voltages");
  CK(cudaSetDevice(h->device));
  int rc = spill_voltages(h);
  if (rc) return rc;
  *n_out = 0;
  *first_g = h->v_host_first < 0 ? h->g.n_past : h->v_host_first;
  if (h->v_host_first < 0) return POND_OK;
  const size_t avail = h->v_host[0].size() / 2;
  const size_t n = std::min(cap, avail);
  for (int c = 0; c < h->g.nchan; ++c) {
    auto& vec = h->v_host[c];
    memcpy(out_c + (size_t)c * cap * 2, vec.data(), n * 2 * sizeof(float));
    vec.erase(vec.begin(), vec.begin() + 2 * n);
  }
  *n_out = n;
  h->v_host_first += (long long)n;
  return POND_OK;
}

int pond_stats(pond_t h, pond_stats_t* s) {
  if (!h || !s) return fail(POND_E_ARG, "null argument");
  CK(cudaSetDevice(h->device));
  int rc = collect_timing(h);
  if (rc) return rc;
  CK(cudaStreamSynchronize(h->st));
  memset(s, 0, sizeof *s);
  const Geom& g = h->g;
  s->samples_in = h->total_in;
  s->segments = h->seg_index;
  s->outputs = h->outputs;
  s->n_past = g.n_past;
  s->n_fut = g.n_fut;
  s->seg_step = g.S;
  s->nfft = (int32_t)g.N;
  s->nchan = g.nchan;
  s->kernel_launches = 7;   // F1, F2, I1, I2, fold partial, fold merge, decimate
  s->flushed = h->flushed;
  const double spec = (double)g.L * sizeof(float2);
  const double nv = (double)g.S_c;
  s->algo_bytes[ST_F1] = (double)g.N + spec;
  s->algo_bytes[ST_F2] = 2 * spec;
  s->algo_bytes[ST_I1] = 2 * spec;
  s->algo_bytes[ST_I2] = spec + nv * sizeof(float);
  s->algo_bytes[ST_FOLD] = nv * sizeof(float);
  s->algo_bytes[ST_DEC] = nv * sizeof(float);
  for (int i = 0; i < POND_NSTAGE; ++i) {
    s->stage_ms[i] = h->stage_ms[i];
    s->stage_launches[i] = h->stage_launches[i];
    s->stage_name[i] = kStageName[i];
  }
  return POND_OK;
}

const char* pond_strerror(int code) {
  switch (code) {
    case POND_OK: return "ok";
    case POND_E_ARG: return "invalid argument";
    case POND_E_NFFT: return "invalid or too short nfft";
    case POND_E_NCHAN: return "invalid nchan";
    case POND_E_OOM: return "out of memory";
    case POND_E_CUDA: return "CUDA error";
    case POND_E_STATE: return "invalid state";
    case POND_E_OVERRUN: return "output overrun";
    case POND_E_TIMEOUT: return "device wait timed out";
    case POND_E_UNIMPLEMENTED: return "not implemented";
    default: return "unknown error";
  }
}

const char* pond_last_error(void) { return g_last_error.c_str(); }

int pond_destroy(pond_t h) {
  if (!h) return POND_OK;
  cudaSetDevice(h->device);
  destroy_all(h);
  return POND_OK;
}

}  // extern "C"
