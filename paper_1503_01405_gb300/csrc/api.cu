// C ABI of the engine: planning, stream ingest, segment scheduling, outputs.
//
// The host side holds the overlap-save bookkeeping (PONDER Sec. 3.7): segment s
// of a lane starts at real sample s*S (S = 2 nchan S_c) and yields the channel
// samples g = s*S_c + m, n_past <= m < M - n_fut.  The last N - S real samples
// seen so far are kept in the lane's device carry buffer for its next segment.
//
// A plan holds one lane per FFT length.  A single-DM plan has one lane with one
// trial and also folds.  A batched plan holds many DM trials: trials with the
// same FFT length share a lane, whose segmentation takes the overlap of its
// largest DM; the lane's forward transform runs once per segment and each trial
// applies its own chirp in the first inverse pass.  All trials emit the common
// range of channel samples set by the largest DM of the plan.
//
// Every arithmetic step on the data runs in the kernels of kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <type_traits>
#include <tuple>
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

#define RC(call)           \
  do {                     \
    int rc_ = (call);      \
    if (rc_) return rc_;   \
  } while (0)

constexpr double K_DM = 1.0 / 2.41e-4;          // s MHz^2 (Eq. 1 constant)
constexpr long long STAGE_BYTES = 128ll << 20;  // host-push staging chunk
constexpr int NSTAGE = 2;                        // staging buffers: copies run up to one piece ahead
constexpr long long FIRST_STAGE_BYTES = 32ll << 20;  // first piece of a stream's host push
constexpr long long TS_RING_SINGLE = 1ll << 22; // time-series samples held on the device (one trial)
constexpr long long TS_RING_MULTI = 1ll << 19;  // ... per trial of a batched plan
constexpr int MAX_TRIALS = 4096;
constexpr int NSLOT = 2;                       // segments in flight (streams, FFT buffer sets)

// Stages in pipeline order (a segment runs F1, F2, I1, I2; F1, F2f, Ic; or, in
// batched plans, F1, F2 and per trial Ir, Ic; then fold / decimation).
enum Stage { ST_F1 = 0, ST_F2, ST_F2F, ST_IR, ST_I1, ST_I2, ST_IC, ST_FOLD, ST_DEC, ST_COUNT };
static_assert(ST_COUNT <= POND_NSTAGE, "stage slots");
const char* kStageName[POND_NSTAGE] = {"fwd_cols_unpack", "fwd_rows_split", "fwd_rows_chirp_inv",
                                       "inv_rows_chirp", "inv_cols_chirp", "inv_rows_detect",
                                       "inv_cols_detect", "fold", "decimate"};

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

// Events bracketing the stages of one segment (timing mode); unused slots stay null.
struct SegEvents {
  cudaEvent_t e[ST_COUNT + 1];
};

// One DM trial: its chirp anchors and its lane.
struct Trial {
  double dm = 0;
  int lane = 0;
  ChirpAnchor* anc = nullptr;
  int clog = 0;
  long long nanc = 0;
  float2* ctab = nullptr;   // per-bin inverse filter (POND_CHIRP_TABLE, single-DM three-pass plans)
};

// One FFT length: segmentation, buffers, stream state.
struct Lane {
  Geom g;
  double dm_max = 0;                        // largest DM of the lane (sets the overlap)
  std::vector<int> trials;
  // two buffer slots: consecutive segments alternate slots and streams
  float2* bufA[NSLOT] = {};
  float2* bufB[NSLOT] = {};
  float* P[NSLOT] = {};
  // fused schedule (F1, F2f, Ic; batched: F1, F2, per trial Ir, Ic): Ic's group
  // partials and per-m1 tickets per slot
  bool fused = false, fused_multi = false;
  bool ic_tc = false;                       // the column pass on the tensor cores (three-term split-BF16 plans)
  float* part[NSLOT] = {};
  int* cnt[NSLOT] = {};
  // per trial of the lane and slot: after that trial's fold / decimation of a segment
  std::vector<cudaEvent_t> ev_chain[NSLOT];
  float2* stw = nullptr;                    // stage twiddle tables of R1, R2, Q1, Q2
  const float2 *stwR1 = nullptr, *stwR2 = nullptr, *stwQ1 = nullptr, *stwQ2 = nullptr, *stwJ = nullptr;
  float2* tw2buf = nullptr;
  Tw2 tw2L;                                 // exp(-2 pi i e/(2L))
  float2* tw3L = nullptr;                   // three-level exp(-2 pi i e/L)
  float2* tw3M = nullptr;                   // three-level exp(+2 pi i e/M)
  int8_t* carry[2] = {nullptr, nullptr};
  int carry_cur = 0;
  long long seg_start = 0, carry_pos = 0, segments = 0;
  // batched lanes with several trials per launch (POND_TRIALS_MULTI_*)
  int mode = POND_TRIALS_PER_TRIAL;
  int kt = 1;                               // trials per launch
  float2* bufT[NSLOT] = {};                 // [kt][L] row-pass outputs
  float* Pm[NSLOT] = {};                    // [kt][M] detected power
  float* partm[NSLOT] = {};                 // [kt][G][M] column-pass group partials
  int* cntm[NSLOT] = {};                    // [kt][FUSED_J] column-pass tickets
  unsigned* atab = nullptr;                 // table form: Q0.32 phase of one DM step per bin (row layout)
  unsigned* d_nmul = nullptr;               // per lane trial: its DM in DM steps
  const ChirpAnchor** d_anc = nullptr;      // per lane trial: its anchor table
  int* d_clog = nullptr;
  int* d_rows = nullptr;                    // per lane trial: its series row (the caller's trial index)
  double dm_step = 0;                       // table form's DM step (0: no table)
  std::vector<int> cand_mode, cand_kt;      // autotuner candidates and their time per trial
  std::vector<int> cand_split;              // log2 Q1 of a four-pass candidate, else 0
  std::vector<double> cand_us;
  float2* stwq = nullptr;                   // Q1 and Q2 tables of a tuned split other than the built one
};

}  // namespace

int pond::set_error(int code, const char* msg) { return fail(code, "%s", msg); }

struct pond_s {
  // parameters
  double f0, bw, fs, period;
  int nchan, nbins;
  long long t_dec_ns;
  int epoch_day;
  double epoch_sec;
  int want_voltages, timing, device;
  bool multi = false;
  int schedule = POND_SCHEDULE_AUTO;
  int ch = 1;                               // bytes per real sample (2: N / S added in phase)
  double dtc = 0, inc = 0;
  FoldPhase fold_rule;                      // the fold's phase: constant period or a phase model
  long long dec_num = 1, dec_den = 1;
  int sgn = 1;
  // lanes and trials (trials in the caller's order)
  std::vector<Lane> lanes;
  std::vector<Trial> trials;
  long long g_first = 0, n_fut_max = 0;     // common emitted range: [g_first, total_c - n_fut_max)
  // streams
  cudaStream_t st = nullptr, cst = nullptr;
  // streams of segments s with s mod NSLOT = 1 .. NSLOT-1 (slot 0 runs on st);
  // joined into st by every call that reads results or hands a buffer back
  cudaStream_t sx[NSLOT] = {};
  cudaEvent_t ev_in = nullptr, ev_join[NSLOT] = {};
  cudaEvent_t ev_done = nullptr, ev_caller = nullptr;
  cudaEvent_t ev_copied[NSTAGE] = {}, ev_used[NSTAGE] = {};
  // side-stream work of the last two ingests (carry reuse) and of the segments
  // that read each staging buffer (staging reuse)
  cudaEvent_t ev_side[2][NSLOT] = {}, ev_used_x[NSTAGE][NSLOT] = {};
  int ingest_par = 0;
  // single-DM plans fold on their own stream: a segment's fold waits for its
  // detection (ev_pready), the next detection into the same P for the fold
  // (ev_pfree); the segment streams never wait for folds of other segments
  cudaStream_t sf = nullptr;
  cudaEvent_t ev_pready[NSLOT] = {}, ev_pfree[NSLOT] = {}, ev_fjoin = nullptr;
  // fold (single-DM plans)
  double* prof_sum = nullptr;
  long long* prof_hits = nullptr;
  double* psum = nullptr;                   // per-CTA fold partials, accumulated over the stream
  long long* phits = nullptr;
  // time series rings: [ntrial][ring] sums and counts
  long long ring = 0;
  float* ts = nullptr;
  int* ts_cnt = nullptr;
  // host-push staging
  int8_t* stage[NSTAGE] = {};
  int stage_next = 0;
  // voltages (single-DM plans, tests)
  float2* vbuf = nullptr;
  long long v_cap = 0;
  // stream state
  long long total_in = 0;
  bool flushed = false;
  long long outputs = 0;
  // time series: [ts_drained, ts_complete) complete on the device; ts_hi = one past the last touched
  long long ts_first = -1, ts_drained = 0, ts_hi = 0, ts_complete = 0;
  std::vector<std::vector<float>> ts_host;  // per trial
  std::vector<int32_t> ts_host_cnt;
  void* ts_pin = nullptr;                   // pinned staging of one ring row (ring * 4 B)
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
  long long launches = 0;
  double push_enqueue_ms = 0, push_wait_ms = 0;   // host times of the last pond_push
  // split-BF16 tensor-core stages: product terms (0 = FP32), W16 parts, MMA wait flag
  int tc_terms = 0;
  uint4* wdft = nullptr;
  int* tc_err = nullptr;
  uint4* ic_ops = nullptr;                  // operand block of the tensor-core column pass
};

namespace {

int validate(const pond_opts* o) {
  if (!o) return fail(POND_E_ARG, "null options");
  if (!(o->f0_mhz > 0) || !(o->bw_mhz != 0) || !(std::fabs(o->bw_mhz) < 2 * o->f0_mhz) || !(o->fs_hz > 0))
    return fail(POND_E_ARG, "bad band: f0=%g bw=%g fs=%g", o->f0_mhz, o->bw_mhz, o->fs_hz);
  if (std::fabs(o->fs_hz - 2.0 * std::fabs(o->bw_mhz) * 1e6) > 1e-6 * o->fs_hz)
    return fail(POND_E_ARG, "fs must equal 2|bw| (real Nyquist sampling)");
  if (o->fs_hz != std::floor(o->fs_hz) || o->fs_hz > 9e15) return fail(POND_E_ARG, "fs must be a whole number of Hz");
  if (o->ndm < 0 || o->ndm > MAX_TRIALS) return fail(POND_E_ARG, "ndm must be 0..%d", MAX_TRIALS);
  if (o->ndm > 0) {
    if (!o->dm_list) return fail(POND_E_ARG, "null dm_list");
    for (int i = 0; i < o->ndm; ++i)
      if (!(o->dm_list[i] >= 0) || !std::isfinite(o->dm_list[i])) return fail(POND_E_ARG, "DM must be >= 0");
    if (o->want_voltages) return fail(POND_E_ARG, "want_voltages needs a single-DM plan");
  } else {
    if (!(o->dm >= 0) || !std::isfinite(o->dm)) return fail(POND_E_ARG, "DM must be >= 0");
    if (!(o->period_s > 0) || !std::isfinite(o->period_s)) return fail(POND_E_ARG, "period must be > 0");
    if (o->nbins < 1 || o->nbins > MAX_NBINS) return fail(POND_E_ARG, "nbins must be 1..%d", MAX_NBINS);
  }
  if (o->nfft < 4 || (o->nfft & (o->nfft - 1))) return fail(POND_E_NFFT, "nfft must be a power of two");
  if (o->nchan < 1 || (o->nchan & (o->nchan - 1)) || (o->nfft / 2) % o->nchan)
    return fail(POND_E_NCHAN, "nchan must be a power of two dividing nfft/2");
  for (int i = 0; i < 4; ++i) {
    const long long n = o->nfft_choices[i];
    if (n != 0 && (n < 4 || (n & (n - 1)) || (n / 2) % o->nchan))
      return fail(POND_E_NFFT, "nfft_choices[%d] = %lld is not a usable power of two", i, n);
  }
  if (o->precision != POND_FP32 && o->precision != POND_SPLIT_BF16 && o->precision != POND_SPLIT_BF16_5T)
    return fail(POND_E_ARG, "precision must be POND_FP32, POND_SPLIT_BF16 or POND_SPLIT_BF16_5T");
  if (o->trial_mode < POND_TRIALS_AUTO || o->trial_mode > POND_TRIALS_FOUR_PASS)
    return fail(POND_E_ARG, "trial_mode %d is not a POND_TRIALS_* value", o->trial_mode);
  if (o->trials_per_launch < 0 || o->trials_per_launch > 128)
    return fail(POND_E_ARG, "trials_per_launch must be in 0 .. 128");
  if (o->chirp < POND_CHIRP_AUTO || o->chirp > POND_CHIRP_TABLE)
    return fail(POND_E_ARG, "chirp %d is not a POND_CHIRP_* value", o->chirp);
  if (o->schedule != POND_SCHEDULE_AUTO && o->schedule != POND_SCHEDULE_FOUR_PASS)
    return fail(POND_E_ARG, "schedule must be POND_SCHEDULE_AUTO or POND_SCHEDULE_FOUR_PASS");
  if (o->input_channels < 0 || o->input_channels > 2)
    return fail(POND_E_ARG, "input_channels must be 0 or 1 (one int8 stream) or 2 (N / S pairs added in phase)");
  if (o->inv_split < 0 || o->inv_split > 12) return fail(POND_E_ARG, "inv_split must be 0 (default) or 2 .. 12");
  if (o->phase_ncoef < 0 || o->phase_ncoef > 8) return fail(POND_E_ARG, "phase_ncoef must be 0 .. 8");
  if (o->phase_ncoef > 0) {
    if (o->ndm > 0) return fail(POND_E_ARG, "a phase model folds single-DM plans only");
    if (!std::isfinite(o->phase_tref_s)) return fail(POND_E_ARG, "phase_tref_s must be finite");
    for (int i = 0; i < o->phase_ncoef; ++i)
      if (!std::isfinite(o->phase_coef[i])) return fail(POND_E_ARG, "phase_coef[%d] must be finite", i);
  }
  return POND_OK;
}

// An inverse split M = Q1 Q2 (q = log2 Q1) the four-pass kernels take: I2's
// CTA holds Q1-point rows of every sub-channel (nchan Q1 <= TILE), I1's bins
// lie in runs of M / R2 columns (Q1 <= R2), and both lengths are 4 .. 4096.
bool split_ok(const Geom& g, int lognch, int q) {
  return q >= 2 && q <= 12 && q <= 13 - lognch && q <= g.logR2 && g.logM - q >= 2 && g.logM - q <= 12;
}

// Overlap-save geometry of an FFT length at the largest DM it must carry.
int geometry(const pond_opts* o, long long nfft, double dm, Geom* g) {
  g->N = nfft;
  g->L = nfft / 2;
  g->nchan = o->nchan;
  g->M = g->L / o->nchan;
  g->logL = ilog2ll(g->L);
  g->logM = ilog2ll(g->M);
  const double dtc = 2.0 * o->nchan / o->fs_hz;
  const double half = std::fabs(o->bw_mhz) / 2.0;
  const double f_lo = o->f0_mhz - half, f_hi = o->f0_mhz + half;
  const double past = K_DM * dm * (std::pow(o->f0_mhz, -2) - std::pow(f_hi, -2));
  const double fut = K_DM * dm * (std::pow(f_lo, -2) - std::pow(o->f0_mhz, -2));
  g->n_past = (long long)std::ceil(past / dtc);
  g->n_fut = (long long)std::ceil(fut / dtc);
  g->S_c = g->M - g->n_past - g->n_fut;
  if (g->S_c <= 0)
    return fail(POND_E_NFFT, "nfft %lld does not exceed the overlap at DM %g (n_past %lld + n_fut %lld >= M %lld)",
                nfft, dm, g->n_past, g->n_fut, g->M);
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
                o->nchan, nfft);
  if (o->inv_split) {
    if (!split_ok(*g, lognch, o->inv_split))
      return fail(POND_E_ARG, "inv_split %d is not admissible for nfft %lld, nchan %d (M = 2^%d, R2 = 2^%d)",
                  o->inv_split, nfft, o->nchan, g->logM, g->logR2);
    g->logQ1 = o->inv_split;
    g->logQ2 = g->logM - g->logQ1;
  }
  return POND_OK;
}

// Bins per chirp anchor (log2): the dropped quartic Taylor term
// alpha f0^2/(f0+f)^5 (du span/2)^4 stays below 1e-9 cycles.
int anchor_log(const pond_opts* o, long long nfft, double dm) {
  const double du = o->fs_hz / (double)nfft * 1e-6;
  const double half = std::fabs(o->bw_mhz) / 2.0;
  const double alpha = K_DM * 1e6 * dm / (o->f0_mhz * o->f0_mhz);
  // |c''''|/24 and |c'''|/6 at their band maximum (f0 + f = f0 - |bw|/2)
  const double c4 = alpha * o->f0_mhz * o->f0_mhz / std::pow(o->f0_mhz - half, 5);
  const double c3 = alpha * o->f0_mhz * o->f0_mhz / std::pow(o->f0_mhz - half, 4);
  int clog = CHIRP_LOG_MAX;
  // dropped quartic term <= 1e-9 cycles; the FP32 cubic term <= 1e-2 cycles
  // (so its rounding stays < 1e-9 cycles)
  while (clog > 0 && (c4 * std::pow(du * (double)(1ll << (clog - 1)), 4) > 1e-9 ||
                      c3 * std::pow(du * (double)(1ll << (clog - 1)), 3) > 1e-2))
    --clog;
  return clog;
}

int build_trial(pond_t h, const pond_opts* o, Trial* t) {
  const Lane& ln = h->lanes[t->lane];
  const long long nfft = ln.g.N;
  t->clog = anchor_log(o, nfft, t->dm);
  t->nanc = (ln.g.L + (1ll << t->clog) - 1) >> t->clog;
  CK(cudaMalloc(&t->anc, t->nanc * sizeof(ChirpAnchor)));
  const double du = o->fs_hz / (double)nfft * 1e-6;
  const double half = std::fabs(o->bw_mhz) / 2.0;
  const double alpha = K_DM * 1e6 * t->dm / (o->f0_mhz * o->f0_mhz);
  CK(launch_tables(t->anc, t->nanc, t->clog, du, half, o->f0_mhz, alpha, h->sgn, h->st));
  // single-DM three-pass plans take the chirp from the per-bin table unless the
  // anchors are asked for: with the table rows prefetched into L2 the fused row
  // pass then overlaps the other segment stream better (full rate: 116.6k
  // against 114.5k Msamples/s)
  if ((o->chirp == POND_CHIRP_TABLE || o->chirp == POND_CHIRP_AUTO) && ln.fused) {
    CK(cudaMalloc(&t->ctab, (size_t)ln.g.L * sizeof(float2)));
    CK(launch_chirp_c64(t->ctab, ln.g, du, half, o->f0_mhz, alpha, h->sgn, h->st));
  }
  return POND_OK;
}

int build_lane(pond_t h, Lane* ln) {
  if (h->tc_terms) {
    ln->g.tc_terms = h->tc_terms;
    ln->g.tc_fwd = {h->wdft, h->tc_terms, h->tc_err};
    ln->g.tc_inv = {h->wdft + TC_W_BYTES / 16, h->tc_terms, h->tc_err};
  }
  const Geom& g = ln->g;
  // three-pass lanes: FP32 plans with M = 64 R2, and three-term split-BF16 plans whose column
  // pass has a tensor-core form (R2 = 2048); the fused row pass itself is FP32 in both
  const bool three = h->schedule == POND_SCHEDULE_AUTO && fused_geometry(g) &&
                     (!h->tc_terms || (h->tc_terms == 3 && ic_tc_geometry(g)));
  ln->fused = !h->multi && three;
  ln->fused_multi = h->multi && three;
  ln->ic_tc = three && h->tc_terms == 3;
  for (int k = 0; k < NSLOT; ++k) {
    CK(cudaMalloc(&ln->bufA[k], g.L * sizeof(float2)));
    CK(cudaMalloc(&ln->bufB[k], g.L * sizeof(float2)));
    CK(cudaMalloc(&ln->P[k], g.M * sizeof(float)));
    if ((ln->fused || ln->fused_multi) && fused_groups(g) > 1) {
      CK(cudaMalloc(&ln->part[k], (size_t)fused_groups(g) * g.M * sizeof(float)));
      CK(cudaMalloc(&ln->cnt[k], FUSED_J * sizeof(int)));
      CK(cudaMemsetAsync(ln->cnt[k], 0, FUSED_J * sizeof(int), h->st));
    }
  }
  const int n1 = stage_tw_entries(1 << g.logR1), n2 = stage_tw_entries(1 << g.logR2);
  const int n3 = stage_tw_entries(1 << g.logQ1), n4 = stage_tw_entries(1 << g.logQ2);
  const int n5 = stage_tw_entries(FUSED_J);
  CK(cudaMalloc(&ln->stw, (size_t)std::max(1, n1 + n2 + n3 + n4 + n5) * sizeof(float2)));
  ln->stwR1 = ln->stw;
  ln->stwR2 = ln->stwR1 + n1;
  ln->stwQ1 = ln->stwR2 + n2;
  ln->stwQ2 = ln->stwQ1 + n3;
  ln->stwJ = ln->stwQ2 + n4;
  auto nhi = [](int logn) { return logn > TW2_LOG ? (1ll << (logn - TW2_LOG)) : 1ll; };
  const long long total = TW2_LO + nhi(g.logL + 1) + 2 * 768;
  CK(cudaMalloc(&ln->tw2buf, total * sizeof(float2)));
  float2* p = ln->tw2buf;
  ln->tw3L = p;
  ln->tw3M = p + 768;
  p += 2 * 768;
  ln->tw2L = {p, p + TW2_LO};
  CK(cudaMalloc(&ln->carry[0], g.N * h->ch));
  CK(cudaMalloc(&ln->carry[1], g.N * h->ch));
  CK(launch_stage_tw(const_cast<float2*>(ln->stwR1), 1 << g.logR1, h->st));
  CK(launch_stage_tw(const_cast<float2*>(ln->stwR2), 1 << g.logR2, h->st));
  CK(launch_stage_tw(const_cast<float2*>(ln->stwQ1), 1 << g.logQ1, h->st));
  CK(launch_stage_tw(const_cast<float2*>(ln->stwQ2), 1 << g.logQ2, h->st));
  CK(launch_stage_tw(const_cast<float2*>(ln->stwJ), FUSED_J, h->st));
  CK(launch_tw3(ln->tw3L, g.logL, -1, h->st));
  CK(launch_tw2(const_cast<float2*>(ln->tw2L.lo), const_cast<float2*>(ln->tw2L.hi), g.logL + 1, -1, h->st));
  CK(launch_tw3(ln->tw3M, g.logM, +1, h->st));
  return POND_OK;
}

void free_lane(Lane* ln) {
  for (int k = 0; k < NSLOT; ++k) {
    cudaFree(ln->bufA[k]);
    cudaFree(ln->bufB[k]);
    cudaFree(ln->P[k]);
    cudaFree(ln->part[k]);
    cudaFree(ln->cnt[k]);
    cudaFree(ln->bufT[k]);
    cudaFree(ln->Pm[k]);
    cudaFree(ln->partm[k]);
    cudaFree(ln->cntm[k]);
    for (auto e : ln->ev_chain[k]) cudaEventDestroy(e);
    ln->ev_chain[k].clear();
  }
  cudaFree(ln->atab);
  cudaFree(ln->d_nmul);
  cudaFree(ln->d_anc);
  cudaFree(ln->d_clog);
  cudaFree(ln->d_rows);
  cudaFree(ln->stw);
  cudaFree(ln->stwq);
  cudaFree(ln->tw2buf);
  cudaFree(ln->carry[0]);
  cudaFree(ln->carry[1]);
  *ln = Lane();
}

// Record boundary event i of the current segment (0 = before F1, i = after stage i-1).
// Order everything queued on the segment streams before later work on st.
int join_streams(pond_t h) {
  for (int k = 1; k < NSLOT; ++k) {
    CK(cudaEventRecord(h->ev_join[k], h->sx[k]));
    CK(cudaStreamWaitEvent(h->st, h->ev_join[k], 0));
  }
  CK(cudaEventRecord(h->ev_fjoin, h->sf));
  CK(cudaStreamWaitEvent(h->st, h->ev_fjoin, 0));
  return POND_OK;
}

// Work on the segment streams may read what st produced before this point.
int fork_streams(pond_t h) {
  CK(cudaEventRecord(h->ev_in, h->st));
  for (int k = 1; k < NSLOT; ++k) CK(cudaStreamWaitEvent(h->sx[k], h->ev_in, 0));
  CK(cudaStreamWaitEvent(h->sf, h->ev_in, 0));
  return POND_OK;
}

int record(pond_t h, int i, cudaStream_t cs, bool last = false) {
  if (!h->timing) return POND_OK;
  cudaEvent_t e;
  if (!h->ev_pool.empty()) {
    e = h->ev_pool.back();
    h->ev_pool.pop_back();
  } else {
    CK(cudaEventCreate(&e));
  }
  CK(cudaEventRecord(e, cs));
  h->ev_cur.e[i] = e;
  if (last) h->ev_pending.push_back(h->ev_cur);
  return POND_OK;
}

int collect_timing(pond_t h) {
  if (!h->timing) return POND_OK;
  RC(join_streams(h));
  CK(cudaStreamSynchronize(h->st));
  for (auto& se : h->ev_pending) {
    for (int i = 0; i < ST_COUNT; ++i) {
      if (!se.e[i + 1]) continue;
      int k = i;
      while (k >= 0 && !se.e[k]) --k;     // a skipped stage: time from the last boundary
      if (k < 0) continue;
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, se.e[k], se.e[i + 1]));
      h->stage_ms[i] += ms;
      h->stage_launches[i] += 1;
    }
    for (int i = 0; i <= ST_COUNT; ++i)
      if (se.e[i]) h->ev_pool.push_back(se.e[i]);
  }
  h->ev_pending.clear();
  return POND_OK;
}

// True when p is page-locked host memory (cudaMallocHost / cudaHostRegister):
// device-to-host copies can land there directly.
bool pinned_host(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

// Move n completed series samples, from ts_drained on, out of the device ring
// into row d of dst (dst(d) returns its first element) and the counts into
// cnt, and clear the ring slots they held.  Rows that are page-locked host
// memory receive the device-to-host copies directly; others go through the
// pinned row buffer (device-to-pageable copies are several times slower).
template <class DstRow>
int drain_ts(pond_t h, long long n, DstRow dst, int32_t* cnt) {
  const int ntr = (int)h->trials.size();
  const long long slot0 = h->ts_drained % h->ring;
  auto row = [&](auto* dev_row, auto* out) -> int {
    using T = typename std::remove_pointer<decltype(out)>::type;
    static_assert(sizeof(T) == sizeof(float), "4-byte ring rows");
    const bool direct = out && pinned_host(out);
    if (out && !direct && !h->ts_pin) CK(cudaMallocHost(&h->ts_pin, (size_t)h->ring * sizeof(float)));
    T* land = direct ? out : static_cast<T*>(h->ts_pin);
    long long done = 0, slot = slot0;
    while (done < n) {
      const long long run = std::min(n - done, h->ring - slot);
      if (out) CK(cudaMemcpyAsync(land + done, dev_row + slot, run * sizeof(T), cudaMemcpyDeviceToHost, h->st));
      CK(cudaMemsetAsync(dev_row + slot, 0, run * sizeof(T), h->st));
      done += run;
      slot = 0;
    }
    if (out && !direct) {
      CK(cudaStreamSynchronize(h->st));
      memcpy(out, h->ts_pin, n * sizeof(T));
    }
    return POND_OK;
  };
  for (int d = 0; d < ntr; ++d) RC(row(h->ts + (size_t)d * h->ring, dst(d)));
  // every trial's counts row is the same: the first is returned, all are cleared
  for (int d = 0; d < ntr; ++d) RC(row(h->ts_cnt + (size_t)d * h->ring, d == 0 ? cnt : (int32_t*)nullptr));
  CK(cudaStreamSynchronize(h->st));
  h->ts_drained += n;
  return POND_OK;
}

int spill_ts(pond_t h) {
  if (h->ts_first < 0 || h->ts_complete <= h->ts_drained) return POND_OK;
  RC(join_streams(h));
  CK(cudaStreamSynchronize(h->st));
  const long long n = h->ts_complete - h->ts_drained;
  const int ntr = (int)h->trials.size();
  if (h->ts_host[0].empty()) h->ts_host_first = h->ts_drained;
  const size_t off = h->ts_host[0].size();
  for (int d = 0; d < ntr; ++d) h->ts_host[d].resize(off + n);
  h->ts_host_cnt.resize(off + n);
  return drain_ts(h, n, [&](int d) { return h->ts_host[d].data() + off; }, h->ts_host_cnt.data() + off);
}

int spill_voltages(pond_t h) {
  if (!h->want_voltages || h->v_len == 0) return POND_OK;
  RC(join_streams(h));
  CK(cudaStreamSynchronize(h->st));
  if (h->v_host_first < 0) h->v_host_first = h->v_base;
  for (int c = 0; c < h->nchan; ++c) {
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

// The lane's next channel sample still to be produced (its next segment's first output).
long long lane_next_g(pond_t h, const Lane& ln) {
  return std::max(h->g_first, (ln.seg_start / ln.g.S) * ln.g.S_c + ln.g.n_past);
}

void update_complete(pond_t h) {
  if (h->ts_first < 0) return;
  long long gn = -1;
  for (const Lane& ln : h->lanes) {
    const long long x = lane_next_g(h, ln);
    gn = gn < 0 ? x : std::min(gn, x);
  }
  h->ts_complete = std::max(h->ts_complete, (gn * h->dec_den) / h->dec_num);
}

// Process segment s of lane li; g_end bounds the emitted channel samples.
// The column pass of a three-pass lane: FP32 or tensor-core form.
cudaError_t launch_ic(pond_t h, const Lane& ln, const float2* in, float* P, float* part, int* cnt, float2* vout,
                      long long vstride, long long vofs, int m_lo, int m_hi, cudaStream_t st, int ntr = 1) {
  if (ln.ic_tc)
    return launch_inv_cols_det_tc(ln.g, in, P, part, cnt, vout, vstride, vofs, m_lo, m_hi, h->ic_ops, h->tc_err, st,
                                  ntr);
  return launch_inv_cols_det(ln.g, in, P, part, cnt, vout, vstride, vofs, m_lo, m_hi, ln.stwR2, st, ntr);
}

int run_segment(pond_t h, int li, SegIn in, long long s, long long g_end) {
  Lane& ln = h->lanes[li];
  const Geom& g = ln.g;
  const long long m_lo = std::max(g.n_past, h->g_first - s * g.S_c);
  const long long m_hi = std::min(g.M - g.n_fut, g_end - s * g.S_c);
  ln.segments = s + 1;
  if (m_hi <= m_lo) return POND_OK;
  const long long g0 = s * g.S_c + m_lo;         // first output of this segment
  const long long nv = m_hi - m_lo;
  const long long j_lo = (g0 * h->dec_den) / h->dec_num;
  const long long j_hi = ((g0 + nv - 1) * h->dec_den) / h->dec_num;
  if (h->ts_first < 0) {
    h->ts_first = j_lo;
    h->ts_drained = j_lo;
    h->ts_complete = j_lo;
  }
  if (j_hi - h->ts_drained >= h->ring) RC(spill_ts(h));
  float2* vout = nullptr;
  if (h->want_voltages) {
    if (h->v_base < 0) h->v_base = g0;
    if (h->v_len + nv > h->v_cap) RC(spill_voltages(h));
    vout = h->vbuf;
  }
  {  // F1 may load 8 bytes (4 columns of a row), or one sample's N / S pairs, at a time when both runs allow it
    const int nl1 = std::min(TILE >> g.logR2, 1 << g.logR1);
    in.vec8 = in.ch == 1 && (nl1 % 4 == 0) && ((uintptr_t)in.a % 8 == 0) && (in.a_len % 8 == 0) &&
              (in.b_len == 0 || (uintptr_t)in.b % 8 == 0);
    in.pair4 = in.ch == 2 && ((uintptr_t)in.a % 4 == 0) && (in.a_len % 4 == 0) && (in.b_len % 4 == 0) &&
               (in.b_len == 0 || (uintptr_t)in.b % 4 == 0);
  }
  // consecutive segments alternate buffer slots and streams, so one segment's
  // passes fill the other's tail waves; fold / decimation stay in segment order.
  // With per-stage timing everything runs on st, so each stage's events
  // bracket that stage alone.
  const int slot = (int)(s % NSLOT);
  cudaStream_t cs = (slot && !h->timing) ? h->sx[slot] : h->st;
  float2 *bufA = ln.bufA[slot], *bufB = ln.bufB[slot];
  float* P = ln.P[slot];
  h->ev_cur = SegEvents{};
  RC(record(h, 0, cs));
  CK(launch_fwd_cols(g, in, bufA, ln.stwR2, cs));
  RC(record(h, 1 + ST_F1, cs));
  if (ln.fused) {
    // three passes: F2f takes the chirp and the first inverse factor, Ic the rest
    const Trial& t = h->trials[ln.trials[0]];
    CK(launch_fwd_rows_inv(g, bufA, bufB, ln.tw3L, ln.tw2L, ln.stwR1, ln.stwJ, t.anc, t.clog, t.ctab, cs));
    RC(record(h, 1 + ST_F2F, cs));
    // P of this slot is free once the fold of segment s - NSLOT has read it
    if (!h->timing) CK(cudaStreamWaitEvent(cs, h->ev_pfree[slot], 0));
    CK(launch_ic(h, ln, bufB, P, ln.part[slot], ln.cnt[slot], vout, h->v_cap, h->v_len, (int)m_lo, (int)m_hi, cs));
    RC(record(h, 1 + ST_IC, cs));
    // folds run in segment order on their own stream (on st with per-stage timing)
    cudaStream_t fs = h->timing ? cs : h->sf;
    if (!h->timing) {
      CK(cudaEventRecord(h->ev_pready[slot], cs));
      CK(cudaStreamWaitEvent(fs, h->ev_pready[slot], 0));
    }
    CK(launch_fold_dec(P, nv, g0, h->fold_rule, h->nbins, h->dec_num, h->dec_den, j_lo, j_hi - j_lo + 1,
                       h->ts + (size_t)ln.trials[0] * h->ring, h->ts_cnt + (size_t)ln.trials[0] * h->ring, h->ring,
                       h->psum, h->phits, fs));
    RC(record(h, 1 + ST_FOLD, fs));
    RC(record(h, 1 + ST_DEC, fs, true));
    if (!h->timing) CK(cudaEventRecord(h->ev_pfree[slot], fs));
    h->launches += 4;
  } else {
    CK(launch_fwd_rows(g, bufA, bufB, ln.tw3L, ln.tw2L, ln.stwR1, cs));
    RC(record(h, 1 + ST_F2, cs));
    h->launches += 2;
    if (ln.mode == POND_TRIALS_MULTI_ANCHOR || ln.mode == POND_TRIALS_MULTI_TABLE) {
      // kt trials per launch: the row pass with each trial's chirp, the column
      // pass with detection, then the decimation of every trial's series row
      const int ntr = (int)ln.trials.size();
      for (int b = 0, q0 = 0; q0 < ntr; ++b, q0 += ln.kt) {
        const int nq = std::min(ln.kt, ntr - q0);
        const MultiChirp mc{ln.atab, ln.d_nmul + q0, ln.d_anc + q0, ln.d_clog + q0};
        CK(launch_inv_rows_chirp_multi(g, bufB, ln.bufT[slot], nq, ln.tw3L, ln.stwJ, mc,
                                       ln.mode == POND_TRIALS_MULTI_TABLE, cs));
        if (b == 0) RC(record(h, 1 + ST_IR, cs));
        CK(launch_ic(h, ln, ln.bufT[slot], ln.Pm[slot], ln.partm[slot], ln.cntm[slot], nullptr, 0, 0, (int)m_lo,
                     (int)m_hi, cs, nq));
        if (b == 0) RC(record(h, 1 + ST_IC, cs));
        // the block's series rows are updated in segment order
        CK(cudaStreamWaitEvent(cs, ln.ev_chain[(slot + NSLOT - 1) % NSLOT][b], 0));
        if (h->dec_num < 64 * h->dec_den) {
          CK(launch_decimate_multi(ln.Pm[slot], g.M, nv, g0, h->dec_num, h->dec_den, j_lo, j_hi - j_lo + 1, h->ts,
                                   h->ts_cnt, h->ring, ln.d_rows + q0, nq, cs));
          h->launches += 1;
        } else {
          for (int q = 0; q < nq; ++q) {
            const int d = ln.trials[q0 + q];
            CK(launch_decimate(ln.Pm[slot] + (size_t)q * g.M, nv, g0, h->dec_num, h->dec_den, j_lo,
                               j_hi - j_lo + 1, h->ts + (size_t)d * h->ring, h->ts_cnt + (size_t)d * h->ring,
                               h->ring, cs));
          }
          h->launches += nq;
        }
        if (b == 0) RC(record(h, 1 + ST_DEC, cs, true));
        CK(cudaEventRecord(ln.ev_chain[slot][b], cs));
        h->launches += 2;
      }
    } else {
      for (size_t q = 0; q < ln.trials.size(); ++q) {
        const int d = ln.trials[q];
        const Trial& t = h->trials[d];
        if (ln.mode == POND_TRIALS_PER_TRIAL) {
          // the trial's chirp and the first inverse factor as Ir loads the shared spectrum's rows
          CK(launch_inv_rows_chirp(g, bufB, bufA, ln.tw3L, ln.stwJ, t.anc, t.clog, cs));
          if (q == 0) RC(record(h, 1 + ST_IR, cs));
          CK(launch_ic(h, ln, bufA, P, ln.part[slot], ln.cnt[slot], vout, h->v_cap, h->v_len, (int)m_lo,
                       (int)m_hi, cs));
          if (q == 0) RC(record(h, 1 + ST_IC, cs));
        } else {
          // four passes: every trial's chirp is applied as I1 loads the shared forward spectrum
          CK(launch_inv_cols(g, bufB, bufA, t.anc, t.clog, ln.stwQ2, cs));
          if (q == 0) RC(record(h, 1 + ST_I1, cs));
          CK(launch_inv_rows(g, bufA, P, vout, h->v_cap, h->v_len, (int)m_lo, (int)m_hi, ln.tw3M, ln.stwQ1, cs));
          if (q == 0) RC(record(h, 1 + ST_I2, cs));
        }
        // each trial's series row (and the fold partials) is updated in segment order
        CK(cudaStreamWaitEvent(cs, ln.ev_chain[(slot + NSLOT - 1) % NSLOT][q], 0));
        if (!h->multi) {
          // fold and decimation in one launch; the profile is merged when read
          CK(launch_fold_dec(P, nv, g0, h->fold_rule, h->nbins, h->dec_num, h->dec_den, j_lo, j_hi - j_lo + 1,
                             h->ts + (size_t)d * h->ring, h->ts_cnt + (size_t)d * h->ring, h->ring, h->psum,
                             h->phits, cs));
          RC(record(h, 1 + ST_FOLD, cs));
          RC(record(h, 1 + ST_DEC, cs, true));
        } else {
          CK(launch_decimate(P, nv, g0, h->dec_num, h->dec_den, j_lo, j_hi - j_lo + 1, h->ts + (size_t)d * h->ring,
                             h->ts_cnt + (size_t)d * h->ring, h->ring, cs));
          if (q == 0) RC(record(h, 1 + ST_DEC, cs, true));
        }
        CK(cudaEventRecord(ln.ev_chain[slot][q], cs));
        h->launches += 3;
      }
    }
  }
  if (h->want_voltages) h->v_len += nv;
  h->ts_hi = std::max(h->ts_hi, j_hi + 1);
  if (li == 0) h->outputs += nv;
  return POND_OK;
}

// Ingest n samples (n ch bytes) at device pointer d into every lane (work ordered on h->st
// and the side streams; callers that read results or release d join them).
int ingest_device(pond_t h, const int8_t* d, long long n) {
  const long long end = h->total_in + n;
  const long long ch = h->ch;                // bytes per sample at d and in the carry
  RC(fork_streams(h));
  for (size_t li = 0; li < h->lanes.size(); ++li) {
    Lane& ln = h->lanes[li];
    const Geom& g = ln.g;
    while (ln.seg_start + g.N <= end) {
      SegIn in;
      in.ch = ch;
      if (ln.seg_start < h->total_in) {
        in.a = ln.carry[ln.carry_cur] + (ln.seg_start - ln.carry_pos) * ch;
        in.a_len = (h->total_in - ln.seg_start) * ch;
        in.b = d;
        in.b_len = g.N * ch - in.a_len;
      } else {
        in.a = d + (ln.seg_start - h->total_in) * ch;
        in.a_len = g.N * ch;
        in.b = nullptr;
        in.b_len = 0;
      }
      RC(run_segment(h, (int)li, in, ln.seg_start / g.S, 1ll << 62));
      ln.seg_start += g.S;
    }
  }
  // Each lane's carry is double-buffered: the buffer rewritten below was last
  // read by the previous ingest's segments, so st waits for that ingest's
  // side-stream work (recorded then), not for this one's.
  const int par = h->ingest_par;
  for (int k = 1; k < NSLOT; ++k) {
    CK(cudaEventRecord(h->ev_side[par][k], h->sx[k]));
    CK(cudaStreamWaitEvent(h->st, h->ev_side[1 - par][k], 0));
  }
  h->ingest_par = 1 - par;
  for (size_t li = 0; li < h->lanes.size(); ++li) {
    Lane& ln = h->lanes[li];
    // keep [seg_start, end) for the lane's next segment
    int8_t* dst = ln.carry[1 - ln.carry_cur];
    // the carry is rewritten by a kernel, not a copy engine, so the copy engines
    // carry only the host pushes' pieces
    if (ln.seg_start < h->total_in) {
      const long long old = h->total_in - ln.seg_start;
      CK(launch_copy_bytes(dst, ln.carry[ln.carry_cur] + (ln.seg_start - ln.carry_pos) * ch, old * ch, h->st));
      if (n > 0) CK(launch_copy_bytes(dst + old * ch, d, n * ch, h->st));
      h->launches += 1 + (n > 0 && old > 0);
    } else if (end > ln.seg_start) {
      CK(launch_copy_bytes(dst, d + (ln.seg_start - h->total_in) * ch, (end - ln.seg_start) * ch, h->st));
      h->launches += 1;
    }
    ln.carry_cur = 1 - ln.carry_cur;
    ln.carry_pos = ln.seg_start;
  }
  h->total_in = end;
  update_complete(h);
  return POND_OK;
}

// POND_E_TIMEOUT when a bounded tensor-core MMA wait expired since the last check.
int check_tc(pond_t h) {
  if (!h->tc_err) return POND_OK;
  int e = 0;
  CK(cudaMemcpy(&e, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) {
    CK(cudaMemset(h->tc_err, 0, sizeof(int)));
    return fail(POND_E_TIMEOUT, "a tensor-core MMA completion wait expired");
  }
  return POND_OK;
}

void destroy_all(pond_t h) {
  if (!h) return;
  for (int k = 1; k < NSLOT; ++k)
    if (h->sx[k]) cudaStreamSynchronize(h->sx[k]);
  if (h->st) cudaStreamSynchronize(h->st);
  for (auto& ln : h->lanes) free_lane(&ln);
  for (auto& t : h->trials) {
    cudaFree(t.anc);
    cudaFree(t.ctab);
  }
  cudaFree(h->prof_sum);
  cudaFree(h->prof_hits);
  cudaFree(h->psum);
  cudaFree(h->phits);
  cudaFree(h->ts);
  cudaFree(h->ts_cnt);
  if (h->ts_pin) cudaFreeHost(h->ts_pin);
  for (int i = 0; i < NSTAGE; ++i) cudaFree(h->stage[i]);
  cudaFree(h->vbuf);
  cudaFree(h->wdft);
  cudaFree(h->tc_err);
  cudaFree(h->ic_ops);
  for (auto& se : h->ev_pending)
    for (int i = 0; i <= ST_COUNT; ++i)
      if (se.e[i]) cudaEventDestroy(se.e[i]);
  for (auto e : h->ev_pool) cudaEventDestroy(e);
  for (int i = 0; i < NSTAGE; ++i) {
    if (h->ev_copied[i]) cudaEventDestroy(h->ev_copied[i]);
    if (h->ev_used[i]) cudaEventDestroy(h->ev_used[i]);
  }
  if (h->ev_done) cudaEventDestroy(h->ev_done);
  if (h->ev_caller) cudaEventDestroy(h->ev_caller);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_fjoin) cudaEventDestroy(h->ev_fjoin);
  for (int k = 0; k < NSLOT; ++k) {
    if (h->ev_pready[k]) cudaEventDestroy(h->ev_pready[k]);
    if (h->ev_pfree[k]) cudaEventDestroy(h->ev_pfree[k]);
  }
  if (h->sf) cudaStreamDestroy(h->sf);
  if (h->st) cudaStreamDestroy(h->st);
  for (int k = 1; k < NSLOT; ++k) {
    if (h->ev_join[k]) cudaEventDestroy(h->ev_join[k]);
    for (int i = 0; i < 2; ++i)
      if (h->ev_side[i][k]) cudaEventDestroy(h->ev_side[i][k]);
    for (int i = 0; i < NSTAGE; ++i)
      if (h->ev_used_x[i][k]) cudaEventDestroy(h->ev_used_x[i][k]);
    if (h->sx[k]) cudaStreamDestroy(h->sx[k]);
  }
  if (h->cst) cudaStreamDestroy(h->cst);
  delete h;
}

// ---------------------------------------------------------------------------
// Autotuner: per FFT length, the device time of the shared forward passes
// (F1 + F2) and of one trial's inverse passes (I1 + I2 + decimation), measured
// with CUDA events over timed launches and cached per (nfft, nchan, device).
// ---------------------------------------------------------------------------

std::mutex g_tune_mu;
std::map<std::tuple<long long, int, int, int, int>, std::pair<double, double>> g_tune_cache;

int measure_lane(pond_t h, const pond_opts* o, long long nfft, double* t_fwd, double* t_inv) {
  const auto key = std::make_tuple(nfft, o->nchan, o->device, o->schedule, o->inv_split);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      *t_fwd = it->second.first;
      *t_inv = it->second.second;
      return POND_OK;
    }
  }
  Lane ln;
  RC(geometry(o, nfft, 0.0, &ln.g));
  ChirpAnchor* anc = nullptr;
  float* T = nullptr;
  int* C = nullptr;
  cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
  auto cleanup = [&]() {
    cudaStreamSynchronize(h->st);
    free_lane(&ln);
    cudaFree(anc);
    cudaFree(T);
    cudaFree(C);
    for (auto& x : e)
      if (x) cudaEventDestroy(x);
  };
  int rc = build_lane(h, &ln);
  if (rc) {
    cleanup();
    return rc;
  }
  const Geom& g = ln.g;
  const int clog = anchor_log(o, nfft, 0.0);
  const long long nanc = (g.L + (1ll << clog) - 1) >> clog;
  const long long nv = std::min<long long>(g.S_c, 1 << 16);
  cudaError_t ce = cudaMalloc(&anc, nanc * sizeof(ChirpAnchor));
  if (ce == cudaSuccess) ce = cudaMalloc(&T, (size_t)(nv / 8 + 1) * sizeof(float));
  if (ce == cudaSuccess) ce = cudaMalloc(&C, (size_t)(nv / 8 + 1) * sizeof(int));
  for (auto& x : e)
    if (ce == cudaSuccess) ce = cudaEventCreate(&x);
  if (ce == cudaSuccess) ce = cudaMemsetAsync(ln.carry[0], 0, g.N * h->ch, h->st);
  if (ce == cudaSuccess)
    ce = launch_tables(anc, nanc, clog, o->fs_hz / (double)nfft * 1e-6, std::fabs(o->bw_mhz) / 2, o->f0_mhz, 0.0,
                       h->sgn, h->st);
  const int reps = 3;
  SegIn in{ln.carry[0], g.N * h->ch, nullptr, 0, 0, h->ch};
  for (int it = 0; it <= reps && ce == cudaSuccess; ++it) {      // first pass warms up
    if (it == 1) ce = cudaEventRecord(e[0], h->st);
    if (ce == cudaSuccess) ce = launch_fwd_cols(g, in, ln.bufA[0], ln.stwR2, h->st);
    if (ce == cudaSuccess) ce = launch_fwd_rows(g, ln.bufA[0], ln.bufB[0], ln.tw3L, ln.tw2L, ln.stwR1, h->st);
  }
  if (ce == cudaSuccess) ce = cudaEventRecord(e[1], h->st);
  for (int it = 0; it <= reps && ce == cudaSuccess; ++it) {
    if (it == 1) ce = cudaEventRecord(e[2], h->st);
    if (ln.fused_multi) {   // the per-trial passes the plan will run
      if (ce == cudaSuccess) ce = launch_inv_rows_chirp(g, ln.bufB[0], ln.bufA[0], ln.tw3L, ln.stwJ, anc, clog, h->st);
      if (ce == cudaSuccess)
        ce = launch_ic(h, ln, ln.bufA[0], ln.P[0], ln.part[0], ln.cnt[0], nullptr, 0, 0, (int)g.n_past,
                       (int)(g.n_past + nv), h->st);
    } else {
      if (ce == cudaSuccess) ce = launch_inv_cols(g, ln.bufB[0], ln.bufA[0], anc, clog, ln.stwQ2, h->st);
      if (ce == cudaSuccess)
        ce = launch_inv_rows(g, ln.bufA[0], ln.P[0], nullptr, 0, 0, (int)g.n_past, (int)(g.n_past + nv), ln.tw3M,
                             ln.stwQ1, h->st);
    }
    if (ce == cudaSuccess) ce = launch_decimate(ln.P[0], nv, 0, 8, 1, 0, nv / 8, T, C, nv / 8 + 1, h->st);
  }
  if (ce == cudaSuccess) ce = cudaEventRecord(e[3], h->st);
  float ms_f = 0, ms_i = 0;
  if (ce == cudaSuccess) ce = cudaEventSynchronize(e[3]);
  if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms_f, e[0], e[1]);
  if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms_i, e[2], e[3]);
  cleanup();
  if (ce != cudaSuccess) return fail(POND_E_CUDA, "autotune: %s", cudaGetErrorString(ce));
  *t_fwd = ms_f / reps;
  *t_inv = ms_i / reps;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_cache[key] = {*t_fwd, *t_inv};
  return POND_OK;
}

// Split the DM-sorted trials into contiguous groups, each with one FFT length,
// minimising the predicted device time per real input sample:
//   cost(group) = (t_fwd(N) + n_trials t_inv(N)) / S(N, largest DM of the group).
int choose_groups(pond_t h, const pond_opts* o, const std::vector<double>& dms, const std::vector<int>& order,
                  const std::vector<long long>& cands, std::vector<long long>* nfft_of_trial) {
  const int n = (int)order.size();
  std::vector<double> tf(cands.size(), 0), ti(cands.size(), 0);
  std::vector<char> usable(cands.size(), 0);
  for (size_t c = 0; c < cands.size(); ++c) {
    Geom g0;
    const std::string keep = g_last_error;
    if (geometry(o, cands[c], 0.0, &g0)) {
      g_last_error = keep;
      continue;
    }
    RC(measure_lane(h, o, cands[c], &tf[c], &ti[c]));
    usable[c] = 1;
  }
  std::vector<double> best(n + 1, 1e300);
  std::vector<int> from(n + 1, -1), with(n + 1, -1);
  best[0] = 0;
  for (int j = 1; j <= n; ++j) {
    const double dmax = dms[order[j - 1]];
    for (size_t c = 0; c < cands.size(); ++c) {
      if (!usable[c]) continue;
      Geom g;
      const std::string keep = g_last_error;
      const int rc = geometry(o, cands[c], dmax, &g);
      g_last_error = keep;
      if (rc) continue;
      for (int i = 0; i < j; ++i) {
        if (best[i] >= 1e299) continue;
        const double cost = (tf[c] + (j - i) * ti[c]) / (double)g.S;
        if (best[i] + cost < best[j]) {
          best[j] = best[i] + cost;
          from[j] = i;
          with[j] = (int)c;
        }
      }
    }
  }
  if (best[n] >= 1e299) return fail(POND_E_NFFT, "no candidate nfft carries DM %g", dms[order[n - 1]]);
  nfft_of_trial->assign(dms.size(), 0);
  for (int j = n; j > 0; j = from[j])
    for (int k = from[j]; k < j; ++k) (*nfft_of_trial)[order[k]] = cands[with[j]];
  return POND_OK;
}

// ---------------------------------------------------------------------------
// Trials of a batched lane: per-trial launches, or kt trials per launch with
// the chirp from each trial's anchors or from one per-bin table
// ---------------------------------------------------------------------------

// The lane's DMs as whole multiples n_d of one step dDM (the table form): the
// step is the smallest positive gap between the sorted DMs (0 included), refined
// by least squares over the n_d; every DM must lie within 1e-13 of the largest
// DM from n_d dDM, so that the table's phase differs from Eq. 4's at the
// trial's own DM by under 1e-7 cycles across the band.
bool dm_steps(const std::vector<double>& dms, double* step, std::vector<unsigned>* n) {
  std::vector<double> v(dms);
  std::sort(v.begin(), v.end());
  const double dmax = v.back();
  if (!(dmax > 0) || v.front() < 0) return false;
  double gap = 0, prev = 0;
  for (double x : v) {
    const double d = x - prev;
    if (d > 1e-9 * dmax && (gap == 0 || d < gap)) gap = d;
    prev = x;
  }
  if (!(gap > 0)) return false;
  n->resize(dms.size());
  double sxn = 0, snn = 0;
  for (size_t i = 0; i < dms.size(); ++i) {
    const double q = std::nearbyint(dms[i] / gap);
    if (q < 0 || q > (double)(1 << 24)) return false;
    (*n)[i] = (unsigned)q;
    sxn += q * dms[i];
    snn += q * q;
  }
  const double st = sxn / snn;
  for (size_t i = 0; i < dms.size(); ++i)
    if (std::fabs(dms[i] - (*n)[i] * st) > 1e-13 * dmax) return false;
  *step = st;
  return true;
}

int alloc_multi(Lane* ln, int kt) {
  const Geom& g = ln->g;
  const int G = fused_groups(g);
  for (int k = 0; k < NSLOT; ++k) {
    cudaFree(ln->bufT[k]);
    cudaFree(ln->Pm[k]);
    cudaFree(ln->partm[k]);
    cudaFree(ln->cntm[k]);
    ln->bufT[k] = nullptr;
    ln->Pm[k] = ln->partm[k] = nullptr;
    ln->cntm[k] = nullptr;
  }
  for (int k = 0; k < NSLOT; ++k) {
    CK(cudaMalloc(&ln->bufT[k], (size_t)kt * g.L * sizeof(float2)));
    CK(cudaMalloc(&ln->Pm[k], (size_t)kt * g.M * sizeof(float)));
    if (G > 1) CK(cudaMalloc(&ln->partm[k], (size_t)kt * G * g.M * sizeof(float)));
    CK(cudaMalloc(&ln->cntm[k], (size_t)kt * FUSED_J * sizeof(int)));
    CK(cudaMemset(ln->cntm[k], 0, (size_t)kt * FUSED_J * sizeof(int)));
  }
  ln->kt = kt;
  return POND_OK;
}

// Device time per trial (us) of one block of min(kt, ntrials) trials of the
// lane in the given mode (row pass, column pass, decimation), on slot 0, by
// CUDA events over three launches after a warm-up.  The series rows it adds to
// are cleared by the caller afterwards.
int time_trials(pond_t h, Lane* ln, int mode, int kt, int split, double* us) {
  const Geom& g = ln->g;
  const int nq = std::min(kt, (int)ln->trials.size());
  const long long m_lo = g.n_past, m_hi = g.M - g.n_fut, g0 = m_lo, nv = m_hi - m_lo;
  const long long j_lo = (g0 * h->dec_den) / h->dec_num, j_hi = ((g0 + nv - 1) * h->dec_den) / h->dec_num;
  // the four-pass form at this split: its own Q1 / Q2 tables
  Geom gq = g;
  float2* tq = nullptr;
  const float2 *tq1 = nullptr, *tq2 = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaSuccess;
  if (mode == POND_TRIALS_FOUR_PASS) {
    gq.logQ1 = split;
    gq.logQ2 = g.logM - split;
    const int n1 = stage_tw_entries(1 << gq.logQ1), n2 = stage_tw_entries(1 << gq.logQ2);
    ce = cudaMalloc(&tq, (size_t)std::max(1, n1 + n2) * sizeof(float2));
    tq1 = tq;
    tq2 = tq + n1;
    if (ce == cudaSuccess) ce = launch_stage_tw(tq, 1 << gq.logQ1, h->st);
    if (ce == cudaSuccess) ce = launch_stage_tw(tq + n1, 1 << gq.logQ2, h->st);
  }
  if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  const int reps = 3;
  for (int it = 0; it <= reps && ce == cudaSuccess; ++it) {
    if (it == 1) ce = cudaEventRecord(e0, h->st);
    if (mode == POND_TRIALS_FOUR_PASS) {
      for (int q = 0; q < nq && ce == cudaSuccess; ++q) {
        const Trial& t = h->trials[ln->trials[q]];
        ce = launch_inv_cols(gq, ln->bufB[0], ln->bufA[0], t.anc, t.clog, tq2, h->st);
        if (ce == cudaSuccess)
          ce = launch_inv_rows(gq, ln->bufA[0], ln->P[0], nullptr, 0, 0, (int)m_lo, (int)m_hi, ln->tw3M, tq1, h->st);
        if (ce == cudaSuccess)
          ce = launch_decimate(ln->P[0], nv, g0, h->dec_num, h->dec_den, j_lo, j_hi - j_lo + 1,
                               h->ts + (size_t)ln->trials[q] * h->ring, h->ts_cnt + (size_t)ln->trials[q] * h->ring,
                               h->ring, h->st);
      }
    } else if (mode == POND_TRIALS_PER_TRIAL) {
      for (int q = 0; q < nq && ce == cudaSuccess; ++q) {
        const Trial& t = h->trials[ln->trials[q]];
        ce = launch_inv_rows_chirp(g, ln->bufB[0], ln->bufA[0], ln->tw3L, ln->stwJ, t.anc, t.clog, h->st);
        if (ce == cudaSuccess)
          ce = launch_ic(h, *ln, ln->bufA[0], ln->P[0], ln->part[0], ln->cnt[0], nullptr, 0, 0, (int)m_lo, (int)m_hi,
                         h->st);
        if (ce == cudaSuccess)
          ce = launch_decimate(ln->P[0], nv, g0, h->dec_num, h->dec_den, j_lo, j_hi - j_lo + 1,
                               h->ts + (size_t)ln->trials[q] * h->ring, h->ts_cnt + (size_t)ln->trials[q] * h->ring,
                               h->ring, h->st);
      }
    } else {
      const MultiChirp mc{ln->atab, ln->d_nmul, ln->d_anc, ln->d_clog};
      ce = launch_inv_rows_chirp_multi(g, ln->bufB[0], ln->bufT[0], nq, ln->tw3L, ln->stwJ, mc,
                                       mode == POND_TRIALS_MULTI_TABLE, h->st);
      if (ce == cudaSuccess)
        ce = launch_ic(h, *ln, ln->bufT[0], ln->Pm[0], ln->partm[0], ln->cntm[0], nullptr, 0, 0, (int)m_lo, (int)m_hi,
                       h->st, nq);
      if (ce == cudaSuccess && h->dec_num < 64 * h->dec_den)
        ce = launch_decimate_multi(ln->Pm[0], g.M, nv, g0, h->dec_num, h->dec_den, j_lo, j_hi - j_lo + 1, h->ts,
                                   h->ts_cnt, h->ring, ln->d_rows, nq, h->st);
    }
  }
  if (ce == cudaSuccess) ce = cudaEventRecord(e1, h->st);
  float ms = 0;
  if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
  if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (tq) {
    cudaStreamSynchronize(h->st);
    cudaFree(tq);
  }
  if (ce != cudaSuccess) return fail(POND_E_CUDA, "trial autotune: %s", cudaGetErrorString(ce));
  *us = 1e3 * ms / reps / nq;
  return POND_OK;
}

// Run the lane's four-pass inverse at split q: its Q1 / Q2 tables are built
// here unless q is the split the lane was built with.
int use_split(pond_t h, Lane* ln, int q) {
  Geom& g = ln->g;
  if (q == g.logQ1) return POND_OK;
  g.logQ1 = q;
  g.logQ2 = g.logM - q;
  const int n1 = stage_tw_entries(1 << g.logQ1), n2 = stage_tw_entries(1 << g.logQ2);
  cudaFree(ln->stwq);
  ln->stwq = nullptr;
  CK(cudaMalloc(&ln->stwq, (size_t)std::max(1, n1 + n2) * sizeof(float2)));
  ln->stwQ1 = ln->stwq;
  ln->stwQ2 = ln->stwq + n1;
  CK(launch_stage_tw(ln->stwq, 1 << g.logQ1, h->st));
  CK(launch_stage_tw(ln->stwq + n1, 1 << g.logQ2, h->st));
  return POND_OK;
}

// Inverse splits the tuner times: the lane's own split and the admissible ones
// nearest to it, at most four (only opts.inv_split when it is set).
std::vector<int> split_candidates(const pond_opts* o, const Geom& g) {
  if (o->inv_split) return {g.logQ1};
  const int lognch = ilog2ll(g.nchan);
  std::vector<int> v{g.logQ1};
  for (int d = 1; d <= 12 && v.size() < 4; ++d)
    for (int q : {g.logQ1 - d, g.logQ1 + d})
      if (v.size() < 4 && split_ok(g, lognch, q)) v.push_back(q);
  return v;
}

// A tuned lane: mode, trials per launch, split, and every candidate (mode, kt, split, us).
struct TrialTune {
  int mode = 0, kt = 1, split = 0;
  std::vector<int> cmode, ckt, csplit;
  std::vector<double> cus;
};
std::map<std::tuple<long long, int, int, int, bool, int, int, int>, TrialTune> g_trial_tune;

void free_multi(Lane* ln) {
  for (int k = 0; k < NSLOT; ++k) {
    cudaFree(ln->bufT[k]);
    cudaFree(ln->Pm[k]);
    cudaFree(ln->partm[k]);
    cudaFree(ln->cntm[k]);
    ln->bufT[k] = nullptr;
    ln->Pm[k] = ln->partm[k] = nullptr;
    ln->cntm[k] = nullptr;
  }
  ln->kt = 1;
}

// Put the lane into a tuned (or cached) form.
int apply_tune(pond_t h, Lane* ln, const TrialTune& t) {
  ln->mode = t.mode;
  ln->cand_mode = t.cmode;
  ln->cand_kt = t.ckt;
  ln->cand_split = t.csplit;
  ln->cand_us = t.cus;
  if (t.mode == POND_TRIALS_FOUR_PASS) RC(use_split(h, ln, t.split));
  if (t.mode == POND_TRIALS_PER_TRIAL || t.mode == POND_TRIALS_FOUR_PASS) {
    free_multi(ln);
    return POND_OK;
  }
  return t.kt != ln->kt || !ln->bufT[0] ? alloc_multi(ln, t.kt) : POND_OK;
}

// Choose how the lane runs its trials (after its trials' anchors exist and the
// series rings are allocated; the rings are cleared afterwards by the caller).
// Lanes with the three-pass geometry (M = 64 R2) run the per-trial row and
// column passes, the multi-trial forms or the four-pass form; the others run
// the four-pass form, at the split opts.inv_split, the default or the tuner's.
int setup_trials(pond_t h, const pond_opts* o, Lane* ln) {
  const Geom& g = ln->g;
  const int ntr = (int)ln->trials.size();
  const int req = o->trial_mode;
  ln->kt = 1;
  ln->mode = ln->fused_multi ? POND_TRIALS_PER_TRIAL : POND_TRIALS_FOUR_PASS;
  if (!h->multi) return POND_OK;
  if (req == POND_TRIALS_FOUR_PASS) ln->mode = POND_TRIALS_FOUR_PASS;
  const bool tune = req == POND_TRIALS_AUTO && o->autotune;
  // several trials per launch need the three-pass lane geometry and two or more trials
  const bool multi_ok = ln->fused_multi && ntr >= 2 && (req == POND_TRIALS_AUTO || req == POND_TRIALS_MULTI_ANCHOR ||
                                                       req == POND_TRIALS_MULTI_TABLE);
  if (multi_ok) {
    std::vector<int> rows(ntr), clogs(ntr);
    std::vector<const ChirpAnchor*> ancs(ntr);
    std::vector<double> dms(ntr);
    for (int q = 0; q < ntr; ++q) {
      const Trial& t = h->trials[ln->trials[q]];
      rows[q] = ln->trials[q];
      ancs[q] = t.anc;
      clogs[q] = t.clog;
      dms[q] = t.dm;
    }
    CK(cudaMalloc(&ln->d_rows, ntr * sizeof(int)));
    CK(cudaMalloc(&ln->d_clog, ntr * sizeof(int)));
    CK(cudaMalloc(&ln->d_anc, ntr * sizeof(ChirpAnchor*)));
    CK(cudaMemcpy(ln->d_rows, rows.data(), ntr * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ln->d_clog, clogs.data(), ntr * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ln->d_anc, ancs.data(), ntr * sizeof(ChirpAnchor*), cudaMemcpyHostToDevice));
    double step = 0;
    std::vector<unsigned> nm;
    if (dm_steps(dms, &step, &nm)) {
      ln->dm_step = step;
      CK(cudaMalloc(&ln->d_nmul, ntr * sizeof(unsigned)));
      CK(cudaMemcpy(ln->d_nmul, nm.data(), ntr * sizeof(unsigned), cudaMemcpyHostToDevice));
      CK(cudaMalloc(&ln->atab, (size_t)g.L * sizeof(unsigned)));
      const double alpha = K_DM * 1e6 * step / (o->f0_mhz * o->f0_mhz);
      CK(launch_chirp_table(ln->atab, g, o->fs_hz / (double)g.N * 1e-6, std::fabs(o->bw_mhz) / 2.0, o->f0_mhz, alpha,
                            h->sgn, h->st));
    }
  }
  const int best_multi = ln->dm_step > 0 ? POND_TRIALS_MULTI_TABLE : POND_TRIALS_MULTI_ANCHOR;
  const int kt_req = o->trials_per_launch ? std::min(o->trials_per_launch, ntr) : 0;
  if (!tune) {
    // the requested form (the table form only where the DMs allow it), else the table form where possible
    if (!multi_ok) return POND_OK;
    ln->mode = (req == POND_TRIALS_MULTI_ANCHOR) ? POND_TRIALS_MULTI_ANCHOR : best_multi;
    return alloc_multi(ln, kt_req ? kt_req : std::min(32, ntr));
  }
  // autotune: time every candidate on this lane, keep the fastest per trial
  struct Cand {
    int mode, kt, split;
  };
  std::vector<Cand> cands;
  std::vector<int> kts;
  if (ln->fused_multi) cands.push_back({POND_TRIALS_PER_TRIAL, 1, 0});
  if (multi_ok) {
    if (kt_req) kts.push_back(kt_req);
    else kts = {std::min(8, ntr), std::min(32, ntr)};
    kts.erase(std::unique(kts.begin(), kts.end()), kts.end());
    for (int kt : kts) {
      cands.push_back({POND_TRIALS_MULTI_ANCHOR, kt, 0});
      if (ln->dm_step > 0) cands.push_back({POND_TRIALS_MULTI_TABLE, kt, 0});
    }
  }
  for (int q : split_candidates(o, g)) cands.push_back({POND_TRIALS_FOUR_PASS, 1, q});
  const auto key = std::make_tuple(g.N, g.nchan, o->device, ntr, ln->dm_step > 0, kt_req,
                                   (int)(h->dec_num / h->dec_den), o->inv_split);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_trial_tune.find(key);
    if (it != g_trial_tune.end()) return apply_tune(h, ln, it->second);
  }
  if (!kts.empty()) RC(alloc_multi(ln, *std::max_element(kts.begin(), kts.end())));
  CK(cudaMemsetAsync(ln->bufB[0], 0, (size_t)g.L * sizeof(float2), h->st));
  TrialTune t;
  size_t best = 0;
  for (size_t c = 0; c < cands.size(); ++c) {
    double us = 0;
    RC(time_trials(h, ln, cands[c].mode, cands[c].kt, cands[c].split, &us));
    t.cmode.push_back(cands[c].mode);
    t.ckt.push_back(cands[c].kt);
    t.csplit.push_back(cands[c].split);
    t.cus.push_back(us);
    if (us < t.cus[best]) best = c;
  }
  t.mode = cands[best].mode;
  t.kt = cands[best].kt;
  t.split = cands[best].split;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_trial_tune[key] = t;
  }
  return apply_tune(h, ln, t);
}

int plan_impl(pond_t* out, const pond_opts* o) {
  RC(validate(o));
  // trials (caller's order) and their DMs
  const bool multi = o->ndm > 0;
  std::vector<double> dms;
  if (multi) dms.assign(o->dm_list, o->dm_list + o->ndm);
  else dms.push_back(o->dm);
  const double dm_max = *std::max_element(dms.begin(), dms.end());
  {  // host-side geometry checks before touching the device
    Geom g;
    RC(geometry(o, o->nfft, multi ? 0.0 : o->dm, &g));
    if (multi && !o->autotune) RC(geometry(o, o->nfft, dm_max, &g));
  }
  pond_t h = new pond_s();
  h->f0 = o->f0_mhz;
  h->bw = o->bw_mhz;
  h->fs = o->fs_hz;
  h->period = o->period_s;
  h->nbins = multi ? 0 : o->nbins;
  h->nchan = o->nchan;
  h->epoch_day = o->epoch_mjd_day;
  h->epoch_sec = o->epoch_mjd_sec;
  h->want_voltages = o->want_voltages;
  h->timing = o->timing;
  h->device = o->device;
  h->sgn = o->bw_mhz > 0 ? 1 : -1;
  h->multi = multi;
  h->schedule = o->schedule;
  h->ch = o->input_channels == 2 ? 2 : 1;
  h->dtc = 2.0 * o->nchan / o->fs_hz;
  h->inc = multi ? 0.0 : h->dtc / o->period_s;
  h->fold_rule.inc = h->inc;
  h->fold_rule.nc = o->phase_ncoef;
  h->fold_rule.dt = h->dtc;
  h->fold_rule.t_ref = o->phase_tref_s;
  for (int i = 0; i < o->phase_ncoef; ++i) h->fold_rule.c[i] = o->phase_coef[i];
  const double tdec = o->t_dec_s > 0 ? o->t_dec_s : 61.44e-6;
  h->t_dec_ns = (long long)std::llround(tdec * 1e9);
  auto bail = [&](int rc) {
    destroy_all(h);
    return rc;
  };
  if (h->t_dec_ns <= 0) return bail(fail(POND_E_ARG, "t_dec must be >= 1 ns"));
  {  // D = t_dec fs / (2 nchan) channel samples, exact rational num/den
    long long num = h->t_dec_ns, den = 1000000000ll * 2 * o->nchan;
    long long fsi = (long long)o->fs_hz;
    long long gq = gcd_ll(fsi, den);
    fsi /= gq;
    den /= gq;
    long long g2 = gcd_ll(num, den);
    num /= g2;
    den /= g2;
    if (num > (1ll << 40) / std::max(1ll, fsi)) return bail(fail(POND_E_ARG, "t_dec too long"));
    h->dec_num = num * fsi;
    h->dec_den = den;
  }
  {  // the common emitted range is set by the largest DM
    const double half = std::fabs(o->bw_mhz) / 2.0;
    const double fut = K_DM * dm_max * (std::pow(o->f0_mhz - half, -2) - std::pow(o->f0_mhz, -2));
    const double past = K_DM * dm_max * (std::pow(o->f0_mhz, -2) - std::pow(o->f0_mhz + half, -2));
    h->g_first = (long long)std::ceil(past / h->dtc);
    h->n_fut_max = (long long)std::ceil(fut / h->dtc);
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) return bail(fail(POND_E_CUDA, "no CUDA device"));
  if (o->device < 0 || o->device >= ndev) return bail(fail(POND_E_ARG, "device %d out of range", o->device));
#define CKD(call)                                                                                   \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess)                                                                          \
      return bail(fail(e_ == cudaErrorMemoryAllocation ? POND_E_OOM : POND_E_CUDA, "%s: %s", #call, \
                       cudaGetErrorString(e_)));                                                    \
  } while (0)
#define RCD(call)              \
  do {                         \
    int rc_ = (call);          \
    if (rc_) return bail(rc_); \
  } while (0)
  CKD(cudaSetDevice(o->device));
  int sms = 0;
  CKD(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, o->device));
  CKD(set_kernel_attributes());
  if (o->precision != POND_FP32) {
    h->tc_terms = o->precision == POND_SPLIT_BF16_5T ? 5 : 3;
    CKD(set_kernel_attributes_tc());
    std::vector<uint16_t> w(2 * TC_W_BYTES / 2);
    build_w16_parts(w.data());
    CKD(cudaMalloc(&h->wdft, 2 * TC_W_BYTES));
    CKD(cudaMalloc(&h->tc_err, sizeof(int)));
    CKD(cudaMemcpy(h->wdft, w.data(), 2 * TC_W_BYTES, cudaMemcpyHostToDevice));
    CKD(cudaMemset(h->tc_err, 0, sizeof(int)));
    std::vector<unsigned char> icops(ic_tc_ops_bytes());
    build_ic_tc_ops(icops.data());
    CKD(cudaMalloc(&h->ic_ops, icops.size()));
    CKD(cudaMemcpy(h->ic_ops, icops.data(), icops.size(), cudaMemcpyHostToDevice));
  }
  CKD(cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking));
  CKD(cudaStreamCreateWithFlags(&h->cst, cudaStreamNonBlocking));
  for (int k = 1; k < NSLOT; ++k) {
    CKD(cudaStreamCreateWithFlags(&h->sx[k], cudaStreamNonBlocking));
    CKD(cudaEventCreateWithFlags(&h->ev_join[k], cudaEventDisableTiming));
    for (int i = 0; i < 2; ++i) CKD(cudaEventCreateWithFlags(&h->ev_side[i][k], cudaEventDisableTiming));
    for (int i = 0; i < NSTAGE; ++i) CKD(cudaEventCreateWithFlags(&h->ev_used_x[i][k], cudaEventDisableTiming));
  }
  CKD(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
  CKD(cudaStreamCreateWithFlags(&h->sf, cudaStreamNonBlocking));
  CKD(cudaEventCreateWithFlags(&h->ev_fjoin, cudaEventDisableTiming));
  for (int k = 0; k < NSLOT; ++k) {
    CKD(cudaEventCreateWithFlags(&h->ev_pready[k], cudaEventDisableTiming));
    CKD(cudaEventCreateWithFlags(&h->ev_pfree[k], cudaEventDisableTiming));
  }
  CKD(cudaEventCreateWithFlags(&h->ev_done, cudaEventDisableTiming));
  CKD(cudaEventCreateWithFlags(&h->ev_caller, cudaEventDisableTiming));
  for (int i = 0; i < NSTAGE; ++i) {
    CKD(cudaEventCreateWithFlags(&h->ev_copied[i], cudaEventDisableTiming));
    CKD(cudaEventCreateWithFlags(&h->ev_used[i], cudaEventDisableTiming));
  }
  // FFT length of every trial
  std::vector<long long> nfft_of(dms.size(), o->nfft);
  if (multi && o->autotune) {
    std::vector<long long> cands;
    for (int i = 0; i < 4; ++i)
      if (o->nfft_choices[i] > 0) cands.push_back(o->nfft_choices[i]);
    if (cands.empty()) cands.push_back(o->nfft);
    std::vector<int> order(dms.size());
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return dms[a] < dms[b]; });
    RCD(choose_groups(h, o, dms, order, cands, &nfft_of));
  }
  // one lane per FFT length, in increasing length; trials keep the caller's order
  std::vector<long long> lens(nfft_of);
  std::sort(lens.begin(), lens.end());
  lens.erase(std::unique(lens.begin(), lens.end()), lens.end());
  h->trials.resize(dms.size());
  h->lanes.resize(lens.size());
  for (size_t li = 0; li < lens.size(); ++li) {
    double lmax = 0;
    for (size_t d = 0; d < dms.size(); ++d)
      if (nfft_of[d] == lens[li]) lmax = std::max(lmax, dms[d]);
    h->lanes[li].dm_max = lmax;
    RCD(geometry(o, lens[li], lmax, &h->lanes[li].g));
    h->lanes[li].g.sms = sms;
    RCD(build_lane(h, &h->lanes[li]));
  }
  for (size_t d = 0; d < dms.size(); ++d) {
    Trial& t = h->trials[d];
    t.dm = dms[d];
    t.lane = (int)(std::lower_bound(lens.begin(), lens.end(), nfft_of[d]) - lens.begin());
    h->lanes[t.lane].trials.push_back((int)d);
    RCD(build_trial(h, o, &t));
  }
  for (auto& ln : h->lanes)
    for (int k = 0; k < NSLOT; ++k) {
      ln.ev_chain[k].assign(ln.trials.size(), nullptr);
      for (auto& e : ln.ev_chain[k]) CKD(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
  // outputs
  const int ntr = (int)dms.size();
  h->ring = multi ? TS_RING_MULTI : TS_RING_SINGLE;
  CKD(cudaMalloc(&h->ts, (size_t)ntr * h->ring * sizeof(float)));
  CKD(cudaMalloc(&h->ts_cnt, (size_t)ntr * h->ring * sizeof(int)));
  CKD(cudaMemsetAsync(h->ts, 0, (size_t)ntr * h->ring * sizeof(float), h->st));
  CKD(cudaMemsetAsync(h->ts_cnt, 0, (size_t)ntr * h->ring * sizeof(int), h->st));
  h->ts_host.assign(ntr, {});
  for (auto& ln : h->lanes) RCD(setup_trials(h, o, &ln));
  if (multi) {   // the trial autotuner's launches added to the series rings
    CKD(cudaMemsetAsync(h->ts, 0, (size_t)ntr * h->ring * sizeof(float), h->st));
    CKD(cudaMemsetAsync(h->ts_cnt, 0, (size_t)ntr * h->ring * sizeof(int), h->st));
  }
  if (!multi) {
    CKD(cudaMalloc(&h->prof_sum, h->nbins * sizeof(double)));
    CKD(cudaMalloc(&h->prof_hits, h->nbins * sizeof(long long)));
    CKD(cudaMalloc(&h->psum, (size_t)MAX_FOLD_PARTS * h->nbins * sizeof(double)));
    CKD(cudaMalloc(&h->phits, (size_t)MAX_FOLD_PARTS * h->nbins * sizeof(long long)));
    CKD(cudaMemsetAsync(h->prof_sum, 0, h->nbins * sizeof(double), h->st));
    CKD(cudaMemsetAsync(h->prof_hits, 0, h->nbins * sizeof(long long), h->st));
    CKD(cudaMemsetAsync(h->psum, 0, (size_t)MAX_FOLD_PARTS * h->nbins * sizeof(double), h->st));
    CKD(cudaMemsetAsync(h->phits, 0, (size_t)MAX_FOLD_PARTS * h->nbins * sizeof(long long), h->st));
  }
  if (h->want_voltages) {
    h->v_cap = std::max<long long>(4 * h->lanes[0].g.S_c, 1 << 16);
    CKD(cudaMalloc(&h->vbuf, (size_t)h->nchan * h->v_cap * sizeof(float2)));
    h->v_host.resize(h->nchan);
  }
  CKD(cudaStreamSynchronize(h->st));
#undef CKD
#undef RCD
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
  if (n % h->ch) return fail(POND_E_ARG, "push of %zu bytes splits an N / S sample pair", n);
  CK(cudaSetDevice(h->device));
  cudaStream_t cs = (cudaStream_t)cuda_stream;
  RC(caller_wait(h, cs));
  RC(ingest_device(h, d_x, (long long)(n / h->ch)));
  RC(join_streams(h));   // every segment that read d_x precedes the release
  return caller_release(h, cs);
}

int pond_push(pond_t h, const int8_t* x, size_t n) {
  if (!h) return fail(POND_E_ARG, "null handle");
  if (h->flushed) return fail(POND_E_STATE, "push after flush");
  if (n == 0) return POND_OK;
  if (!x) return fail(POND_E_ARG, "null data");
  if (n % h->ch) return fail(POND_E_ARG, "push of %zu bytes splits an N / S sample pair", n);
  CK(cudaSetDevice(h->device));
  if (!h->stage[0]) {
    for (int i = 0; i < NSTAGE; ++i) {
      CK(cudaMalloc(&h->stage[i], STAGE_BYTES));
      CK(cudaEventRecord(h->ev_used[i], h->st));
      for (int k = 1; k < NSLOT; ++k) CK(cudaEventRecord(h->ev_used_x[i][k], h->sx[k]));
    }
  }
  cudaEvent_t last = nullptr;
  const auto t_start = std::chrono::steady_clock::now();
  // Pinned host memory is addressable from the device: a copy kernel on a few
  // CTAs moves each piece into its staging buffer.  Copy-engine transfers that
  // overlap the passes were seen to stall now and then for tens of ms (the
  // same copies alone do not); the kernel copy, at a small cost in SMs, does not.
  const int8_t* xdev = nullptr;
  {
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, x) == cudaSuccess && attr.type == cudaMemoryTypeHost && attr.devicePointer)
      xdev = static_cast<const int8_t*>(attr.devicePointer);
    else
      cudaGetLastError();
  }
  for (size_t off = 0; off < n;) {
    // a short first piece of a stream lets the passes start while the rest is copied
    const long long cap = (h->total_in == 0 && off == 0) ? FIRST_STAGE_BYTES : STAGE_BYTES;
    const long long len = std::min<long long>(cap, (long long)(n - off));
    const int i = h->stage_next;
    h->stage_next = (h->stage_next + 1) % NSTAGE;
    CK(cudaStreamWaitEvent(h->cst, h->ev_used[i], 0));
    for (int k = 1; k < NSLOT; ++k) CK(cudaStreamWaitEvent(h->cst, h->ev_used_x[i][k], 0));
    if (xdev) {
      CK(launch_copy_host(h->stage[i], xdev + off, len, 8, h->cst));
      h->launches += 1;
    } else {
      CK(cudaMemcpyAsync(h->stage[i], x + off, len, cudaMemcpyHostToDevice, h->cst));
    }
    CK(cudaEventRecord(h->ev_copied[i], h->cst));
    CK(cudaStreamWaitEvent(h->st, h->ev_copied[i], 0));
    RC(ingest_device(h, h->stage[i], len / h->ch));
    CK(cudaEventRecord(h->ev_used[i], h->st));
    for (int k = 1; k < NSLOT; ++k) CK(cudaEventRecord(h->ev_used_x[i][k], h->sx[k]));
    last = h->ev_copied[i];
    off += (size_t)len;
  }
  // the caller's buffer is free once the copies have landed
  const auto t_enq = std::chrono::steady_clock::now();
  if (last) CK(cudaEventSynchronize(last));
  const auto t_end = std::chrono::steady_clock::now();
  h->push_enqueue_ms = std::chrono::duration<double, std::milli>(t_enq - t_start).count();
  h->push_wait_ms = std::chrono::duration<double, std::milli>(t_end - t_enq).count();
  return POND_OK;
}

int pond_flush(pond_t h) {
  if (!h) return fail(POND_E_ARG, "null handle");
  if (h->flushed) return POND_OK;
  CK(cudaSetDevice(h->device));
  const long long total_c = h->total_in / (2ll * h->nchan);
  const long long g_end = total_c - h->n_fut_max;
  RC(fork_streams(h));
  for (size_t li = 0; li < h->lanes.size(); ++li) {
    Lane& ln = h->lanes[li];
    const Geom& g = ln.g;
    while ((ln.seg_start / g.S) * g.S_c + g.n_past < g_end) {
      SegIn in;
      in.ch = h->ch;
      in.a = ln.carry[ln.carry_cur] + (ln.seg_start - ln.carry_pos) * h->ch;
      in.a_len = std::max(0ll, h->total_in - ln.seg_start) * h->ch;
      in.b = nullptr;
      in.b_len = 0;
      RC(run_segment(h, (int)li, in, ln.seg_start / g.S, g_end));
      ln.seg_start += g.S;
    }
  }
  RC(join_streams(h));
  h->flushed = true;
  if (h->ts_first >= 0) h->ts_complete = h->ts_hi;
  CK(cudaStreamSynchronize(h->st));
  return check_tc(h);
}

int pond_sync(pond_t h) {
  if (!h) return fail(POND_E_ARG, "null handle");
  CK(cudaSetDevice(h->device));
  RC(join_streams(h));
  CK(cudaStreamSynchronize(h->st));
  return check_tc(h);
}

int pond_reset(pond_t h) {
  if (!h) return fail(POND_E_ARG, "null handle");
  CK(cudaSetDevice(h->device));
  RC(collect_timing(h));
  RC(join_streams(h));
  CK(cudaStreamSynchronize(h->st));
  const int ntr = (int)h->trials.size();
  if (!h->multi) {
    CK(cudaMemsetAsync(h->prof_sum, 0, h->nbins * sizeof(double), h->st));
    CK(cudaMemsetAsync(h->prof_hits, 0, h->nbins * sizeof(long long), h->st));
    CK(cudaMemsetAsync(h->psum, 0, (size_t)MAX_FOLD_PARTS * h->nbins * sizeof(double), h->st));
    CK(cudaMemsetAsync(h->phits, 0, (size_t)MAX_FOLD_PARTS * h->nbins * sizeof(long long), h->st));
  }
  CK(cudaMemsetAsync(h->ts, 0, (size_t)ntr * h->ring * sizeof(float), h->st));
  CK(cudaMemsetAsync(h->ts_cnt, 0, (size_t)ntr * h->ring * sizeof(int), h->st));
  CK(cudaStreamSynchronize(h->st));
  for (auto& ln : h->lanes) {
    ln.seg_start = ln.carry_pos = ln.segments = 0;
    ln.carry_cur = 0;
  }
  h->total_in = 0;
  h->flushed = false;
  h->outputs = 0;
  h->launches = 0;
  h->ts_first = -1;
  h->ts_drained = h->ts_hi = h->ts_complete = 0;
  for (auto& v : h->ts_host) v.clear();
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
  if (h->multi) return fail(POND_E_STATE, "a batched plan does not fold");
  CK(cudaSetDevice(h->device));
  RC(join_streams(h));
  CK(launch_fold_snapshot(h->psum, h->phits, h->nbins, h->prof_sum, h->prof_hits, h->st));
  if (sum) CK(cudaMemcpyAsync(sum, h->prof_sum, h->nbins * sizeof(double), cudaMemcpyDeviceToHost, h->st));
  if (hits) CK(cudaMemcpyAsync(hits, h->prof_hits, h->nbins * sizeof(long long), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  if (meta) {
    meta->epoch_mjd_day = h->epoch_day;
    meta->epoch_mjd_sec = h->epoch_sec;
    meta->period_s = h->period;
    meta->dm = h->trials[0].dm;
    meta->dtc_s = h->dtc;
    meta->first_g = h->g_first;
    meta->nsamples = h->outputs;
    meta->nbins = h->nbins;
  }
  return POND_OK;
}

int pond_timeseries(pond_t h, float* out, int32_t* counts, size_t cap, size_t* n_out, int64_t* first_index) {
  if (!h || !n_out || !first_index || (cap > 0 && !out)) return fail(POND_E_ARG, "null argument");
  CK(cudaSetDevice(h->device));
  *n_out = 0;
  *first_index = h->ts_host[0].empty() ? std::max(h->ts_drained, 0ll) : h->ts_host_first;
  if (h->ts_first < 0) return POND_OK;
  if (h->ts_host[0].empty() && h->ts_complete > h->ts_drained) {
    // nothing held on the host: drain the device ring straight into the caller's rows
    RC(join_streams(h));
    CK(cudaStreamSynchronize(h->st));
    const long long n = std::min<long long>((long long)cap, h->ts_complete - h->ts_drained);
    *first_index = h->ts_drained;
    int32_t* cnt = counts;
    std::vector<int32_t> scratch;
    if (!cnt) {
      scratch.resize((size_t)n);
      cnt = scratch.data();
    }
    RC(drain_ts(h, n, [&](int d) { return out + (size_t)d * cap; }, cnt));
    *n_out = (size_t)n;
    return POND_OK;
  }
  RC(spill_ts(h));
  const size_t n = std::min(cap, h->ts_host[0].size());
  if (n) {
    for (size_t d = 0; d < h->trials.size(); ++d) {
      memcpy(out + d * cap, h->ts_host[d].data(), n * sizeof(float));
      h->ts_host[d].erase(h->ts_host[d].begin(), h->ts_host[d].begin() + n);
    }
    if (counts) memcpy(counts, h->ts_host_cnt.data(), n * sizeof(int32_t));
    *first_index = h->ts_host_first;
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
  RC(spill_voltages(h));
  *n_out = 0;
  *first_g = h->v_host_first < 0 ? h->g_first : h->v_host_first;
  if (h->v_host_first < 0) return POND_OK;
  const size_t avail = h->v_host[0].size() / 2;
  const size_t n = std::min(cap, avail);
  for (int c = 0; c < h->nchan; ++c) {
    auto& vec = h->v_host[c];
    memcpy(out_c + (size_t)c * cap * 2, vec.data(), n * 2 * sizeof(float));
    vec.erase(vec.begin(), vec.begin() + 2 * n);
  }
  *n_out = n;
  h->v_host_first += (long long)n;
  return POND_OK;
}

int pond_trials(pond_t h, double* dm, int64_t* nfft, int32_t cap, int32_t* ntrials) {
  if (!h || !ntrials || cap < 0) return fail(POND_E_ARG, "null argument");
  *ntrials = (int32_t)h->trials.size();
  for (int32_t d = 0; d < std::min(cap, *ntrials); ++d) {
    if (dm) dm[d] = h->trials[d].dm;
    if (nfft) nfft[d] = h->lanes[h->trials[d].lane].g.N;
  }
  return POND_OK;
}

// Boxcar candidates over the undrained series block; with net, each is scored
// by the classifier on its patch of the same block.
int pond_tuning(pond_t h, pond_lane_info* out, int32_t cap, int32_t* nlanes) {
  if (!h || !nlanes || (cap > 0 && !out)) return fail(POND_E_ARG, "null argument");
  *nlanes = (int32_t)h->lanes.size();
  for (int i = 0; i < cap && i < (int)h->lanes.size(); ++i) {
    const Lane& ln = h->lanes[i];
    pond_lane_info& r = out[i];
    memset(&r, 0, sizeof r);
    r.nfft = ln.g.N;
    r.ntrials = (int32_t)ln.trials.size();
    r.mode = ln.mode;
    r.trials_per_launch = ln.kt;
    r.inv_split = ln.g.logQ1;
    r.dm_step = ln.dm_step;
    r.ncand = (int32_t)std::min<size_t>(ln.cand_us.size(), POND_TUNE_MAXCAND);
    for (int c = 0; c < r.ncand; ++c) {
      r.cand_mode[c] = ln.cand_mode[c];
      r.cand_kt[c] = ln.cand_kt[c];
      r.cand_split[c] = ln.cand_split[c];
      r.cand_us[c] = ln.cand_us[c];
    }
  }
  return POND_OK;
}

static int candidates_impl(pond_t h, pond_cnn_t net, double threshold, pond_cand* out, size_t cap,
                           size_t* n_found) {
  if (!h || !n_found || (cap > 0 && !out)) return fail(POND_E_ARG, "null argument");
  CK(cudaSetDevice(h->device));
  *n_found = 0;
  if (h->ts_first < 0) return POND_OK;
  RC(join_streams(h));
  CK(cudaStreamSynchronize(h->st));
  const long long j0 = h->ts_drained, n = h->ts_complete - h->ts_drained;
  if (n <= 0) return POND_OK;
  if (n > h->ring) return fail(POND_E_OVERRUN, "more undrained series samples than the device ring holds");
  const int ntr = (int)h->trials.size();
  float* blk = nullptr;
  CK(cudaMalloc(&blk, (size_t)ntr * n * sizeof(float)));
  // gather [j0, j0 + n) of every trial from the rings (at most two runs each)
  long long done = 0;
  cudaError_t e = cudaSuccess;
  while (done < n && e == cudaSuccess) {
    const long long slot = (j0 + done) % h->ring;
    const long long run = std::min(n - done, h->ring - slot);
    e = cudaMemcpy2DAsync(blk + done, n * sizeof(float), h->ts + slot, h->ring * sizeof(float), run * sizeof(float),
                          ntr, cudaMemcpyDeviceToDevice, h->st);
    done += run;
  }
  if (e != cudaSuccess) {
    cudaFree(blk);
    return fail(POND_E_CUDA, "gather series: %s", cudaGetErrorString(e));
  }
  int rc = run_boxcar(blk, ntr, n, n, threshold, out, cap, n_found, h->st);
  const size_t m = std::min(*n_found, cap);
  if (net && m > 0 && (rc == POND_OK || rc == POND_E_OVERRUN)) {
    const int maxb = cnn_max_batch(net);
    std::vector<int32_t> corners(2 * m);
    for (size_t i = 0; i < m; ++i) {
      corners[2 * i] = std::max(0, std::min(out[i].trial - 16, std::max(ntr - 32, 0)));
      corners[2 * i + 1] = (int32_t)(out[i].index - 128);
    }
    int32_t* d_corners = nullptr;
    void* d_patch = nullptr;
    float* d_prob = nullptr;
    const size_t patch_bytes = 32 * 256 * 2;
    e = cudaMalloc(&d_corners, corners.size() * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&d_patch, (size_t)maxb * patch_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&d_prob, m * 4 * sizeof(float));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_corners, corners.data(), corners.size() * sizeof(int32_t), cudaMemcpyHostToDevice, h->st);
    int rs = e == cudaSuccess ? POND_OK : fail(POND_E_CUDA, "score scratch: %s", cudaGetErrorString(e));
    for (size_t b = 0; b < m && rs == POND_OK; b += (size_t)maxb) {
      const int nb = (int)std::min<size_t>((size_t)maxb, m - b);
      rs = pond_patches(blk, ntr, n, n, d_corners + 2 * b, nb, d_patch, h->st);
      if (rs == POND_OK) rs = pond_cnn_forward(net, d_patch, nb, d_prob + 4 * b, h->st);
    }
    std::vector<float> prob(m * 4);
    if (rs == POND_OK) {
      e = cudaMemcpyAsync(prob.data(), d_prob, m * 4 * sizeof(float), cudaMemcpyDeviceToHost, h->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
      if (e != cudaSuccess) rs = fail(POND_E_CUDA, "scores: %s", cudaGetErrorString(e));
    }
    cudaFree(d_corners);
    cudaFree(d_patch);
    cudaFree(d_prob);
    if (rs != POND_OK) {
      cudaFree(blk);
      return rs;
    }
    for (size_t i = 0; i < m; ++i) out[i].score = prob[4 * i];
  }
  cudaFree(blk);
  for (size_t i = 0; i < m; ++i) {
    out[i].index += j0;
    out[i].dm = h->trials[out[i].trial].dm;
  }
  return rc;
}

int pond_candidates(pond_t h, double threshold, pond_cand* out, size_t cap, size_t* n_found) {
  return candidates_impl(h, nullptr, threshold, out, cap, n_found);
}

int pond_candidates_scored(pond_t h, pond_cnn_t net, double threshold, pond_cand* out, size_t cap,
                           size_t* n_found) {
  if (!net) return fail(POND_E_ARG, "pond_candidates_scored: null network");
  return candidates_impl(h, net, threshold, out, cap, n_found);
}

int pond_check_bounded_wait(double limit_s, int32_t device, double* waited_s) {
  if (!(limit_s > 0) || limit_s > 10.0 || !waited_s) return fail(POND_E_ARG, "limit must be in (0, 10] s");
  CK(cudaSetDevice(device));
  int* d_status = nullptr;
  unsigned long long* d_waited = nullptr;
  CK(cudaMalloc(&d_status, sizeof(int)));
  cudaError_t e = cudaMalloc(&d_waited, sizeof(unsigned long long));
  if (e == cudaSuccess) e = launch_wait_probe((unsigned long long)(limit_s * 1e9), d_status, d_waited);
  int status = 0;
  unsigned long long waited = 0;
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&waited, d_waited, sizeof(waited), cudaMemcpyDeviceToHost);
  cudaFree(d_status);
  cudaFree(d_waited);
  if (e != cudaSuccess) return fail(POND_E_CUDA, "bounded-wait check: %s", cudaGetErrorString(e));
  *waited_s = (double)waited * 1e-9;
  if (status) return fail(POND_E_TIMEOUT, "the bounded wait gave up after %.3f s, as it must", *waited_s);
  return POND_OK;
}

int pond_stats(pond_t h, pond_stats_t* s) {
  if (!h || !s) return fail(POND_E_ARG, "null argument");
  CK(cudaSetDevice(h->device));
  RC(collect_timing(h));
  CK(cudaStreamSynchronize(h->st));
  memset(s, 0, sizeof *s);
  const Geom& g = h->lanes[0].g;
  s->samples_in = h->total_in;
  s->segments = 0;
  for (auto& ln : h->lanes) s->segments += ln.segments;
  s->outputs = h->outputs;
  s->n_past = g.n_past;
  s->n_fut = g.n_fut;
  s->seg_step = g.S;
  s->nfft = (int32_t)g.N;
  s->nchan = g.nchan;
  s->kernel_launches = (int32_t)std::min<long long>(h->launches, 0x7fffffff);
  s->flushed = h->flushed;
  const double spec = (double)g.L * sizeof(float2);
  const double nv = (double)g.S_c;
  s->pass_bytes[ST_F1] = (double)g.N * h->ch + spec;  // int8 in (pairs for AIP input)
  s->pass_bytes[ST_F2] = 2 * spec;
  s->pass_bytes[ST_F2F] = 2 * spec;
  s->pass_bytes[ST_IR] = 2 * spec;
  s->pass_bytes[ST_I1] = 2 * spec;
  s->pass_bytes[ST_I2] = spec + nv * sizeof(float);
  s->pass_bytes[ST_IC] = spec + nv * sizeof(float);
  s->pass_bytes[ST_FOLD] = nv * sizeof(float);
  s->pass_bytes[ST_DEC] = nv * sizeof(float);
  // algorithmic FP32 work: 5 n log2 n per length-n FFT factor over all L bins
  const double L = (double)g.L;
  const int logJ = g.logM - g.logR2;   // first inverse factor of the three-pass schedule
  const double detect = 4.0 * g.nchan * nv;
  s->algo_flops[ST_F1] = 5 * L * g.logR2 + (h->ch > 1 ? (double)g.N : 0.0);
  s->algo_flops[ST_F2] = 5 * L * g.logR1 + 10 * L;
  s->algo_flops[ST_F2F] = 5 * L * g.logR1 + 10 * L + 6 * L + 5 * L * logJ;
  s->algo_flops[ST_IR] = 6 * L + 5 * L * logJ;
  s->algo_flops[ST_I1] = 6 * L + 5 * L * g.logQ2;
  s->algo_flops[ST_I2] = 5 * L * g.logQ1 + detect;
  s->algo_flops[ST_IC] = 5 * L * g.logR2 + detect;
  s->algo_flops[ST_FOLD] = nv;
  s->algo_flops[ST_DEC] = nv;
  s->push_enqueue_ms = h->push_enqueue_ms;
  s->push_wait_ms = h->push_wait_ms;
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
