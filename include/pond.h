/*
 * pond.h -- C ABI of the GB300 phase-coherent dedispersion engine.
 *
 * The engine implements the phase-coherent dedispersion (PCD) mode of PONDER
 * (Naidu, Joshi, Manoharan & Krishnakumar, "PONDER - A real time software
 * backend for pulsar and IPS observations at the Ooty Radio Telescope",
 * Sec. 3.7 and Fig. "gpuflow"): a raw real-sampled 8-bit voltage stream is cut
 * into overlap-save segments, Fourier transformed, multiplied by the inverse of
 * the interstellar-medium transfer function H of Eq. 4, inverse transformed
 * into sub-channels, detected (|v|^2, summed over sub-channels), folded at the
 * pulsar period (the fold of Sec. 3.4) and decimated to a time series.
 * Around it: batched DM trials with an FFT-length autotuner, a boxcar
 * single-pulse detector and a small CNN classifier (pond_candidates*,
 * pond_cnn_*), the incoherent AID / CID modes of Sec. 3.4 and the
 * scintillation mode of Sec. 3.5 (pond_incoh_*), and folding with a phase
 * model into pulse stacks (pond_fold_stack).
 *
 * Conventions shared by every entry point:
 *  - Units: frequencies in MHz, the sampling rate fs in real samples per second
 *    (fs must equal 2 |bw| 1e6: real Nyquist sampling, Sec. 3.2), DM in
 *    pc cm^-3, times in seconds.
 *  - Dispersion constant K = 1/2.41e-4 s MHz^2 (Eq. 1's constant); the phase of
 *    H(f0+f) is 2 pi K 1e6 DM f^2 / (f0^2 (f0+f)) radians, f in MHz.
 *    bw > 0 is an upper sideband (baseband b <-> sky f0 - |bw|/2 + b); bw < 0 is
 *    inverted (sky f0 + |bw|/2 - b), where the baseband spectrum is conjugated
 *    so the inverse filter is H itself rather than conj(H).
 *  - Channel samples: sub-channel c (c = 0..nchan-1) covers spectrum bins
 *    c*M .. c*M+M-1 of the N/2 kept bins (M = nfft/(2 nchan)); its complex
 *    voltage is sampled every dtc = 2 nchan / fs seconds.  The global channel
 *    sample index g counts from the first stream sample; output g refers to
 *    arrival at the band centre f0.  The first n_past and the last n_fut
 *    channel samples of a stream have incomplete support and are never emitted.
 *  - Return codes: POND_OK (0) or a negative POND_E_* code.  A message for the
 *    last error of the calling thread is available from pond_last_error().
 *  - Ownership: the caller owns every pointer it passes; the library keeps no
 *    caller pointer after a call returns (device pushes: see pond_push_device).
 *    A handle owns all device memory, streams and events it creates.
 *  - Threading: a handle may be used by one thread at a time.
 *  - Determinism: outputs do not depend on how the stream is split into pushes,
 *    and repeated runs give bit-identical outputs (no floating-point atomics).
 */
#ifndef POND_H
#define POND_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define POND_OK 0
#define POND_E_ARG (-1)           /* invalid argument (band, DM, period, sizes, null pointer) */
#define POND_E_NFFT (-2)          /* nfft not a power of two, outside the supported range,
                                     or not longer than the overlap (no valid output; Sec. 3.7:
                                     the filter must exceed the dispersion smear) */
#define POND_E_NCHAN (-3)         /* nchan not a power of two dividing nfft/2, or too many */
#define POND_E_OOM (-4)           /* device or pinned-host allocation failed */
#define POND_E_CUDA (-5)          /* a CUDA runtime call failed */
#define POND_E_STATE (-6)         /* call not allowed in this state (e.g. push after flush) */
#define POND_E_OVERRUN (-7)       /* an output buffer would overflow */
#define POND_E_TIMEOUT (-8)       /* a bounded device wait expired */
#define POND_E_UNIMPLEMENTED (-9) /* option not supported by this build */

/* Arithmetic of the FFT stages. */
#define POND_FP32 0           /* FP32 butterflies (CUDA cores) */
#define POND_SPLIT_BF16 1     /* radix-16 stages as 16-point DFT-matrix products on the
                                 tensor cores: data split into hi + lo BF16, W16 into
                                 hi + mid + lo, three product terms (x_hi w_hi + x_hi w_mid
                                 + x_lo w_hi) accumulated in FP32 */
#define POND_SPLIT_BF16_5T 2  /* as POND_SPLIT_BF16 with five terms (adds x_hi w_lo and
                                 x_lo w_mid): only the data split rounds to BF16 */

/* Pass schedule of a segment (Sec. 3.7 path, same outputs either way). */
#define POND_SCHEDULE_AUTO 0       /* single-trial FP32 plans whose sub-channel length M is
                                      64 times the forward column length R2 >= 16 (e.g. nfft
                                      2^24 with 64 sub-channels) run three passes: the forward
                                      row pass also applies Eq. 4 and the first length-64
                                      factor of each sub-channel's inverse DFT, and one
                                      column pass finishes the inverse, detects and sums
                                      the sub-channels; every other plan runs four */
#define POND_SCHEDULE_FOUR_PASS 1  /* always the four-pass schedule (forward columns,
                                      forward rows, inverse columns with Eq. 4, inverse
                                      rows with detection) */

typedef struct pond_s* pond_t;

/* Full plan description for pond_plan_ex.  Zero-initialise, then set fields. */
typedef struct {
  double f0_mhz;        /* band centre (Sec. 3.7: f0 of Eq. 4) */
  double bw_mhz;        /* bandwidth; negative = inverted sideband */
  double fs_hz;         /* real samples per second, = 2 |bw| 1e6, a whole number */
  double dm;            /* dispersion measure, >= 0 */
  int64_t nfft;         /* real samples per overlap-save segment, power of two */
  int32_t nchan;        /* detected sub-channels, power of two dividing nfft/2 */
  int32_t nbins;        /* fold bins, 1..4096 */
  double period_s;      /* folding period, > 0 */
  double t_dec_s;       /* time-series resolution; rounded to whole ns; 0 -> 61.44e-6 */
  int32_t epoch_mjd_day;/* time of the first stream sample: MJD day ... */
  double epoch_mjd_sec; /* ... and seconds into that day (reported in pond_meta) */
  int32_t precision;    /* POND_FP32, POND_SPLIT_BF16 or POND_SPLIT_BF16_5T */
  int32_t want_voltages;/* nonzero: keep dedispersed voltages for pond_voltages (tests) */
  int32_t timing;       /* nonzero: time each GPU stage with CUDA events (pond_stats); the
                           segments then run one after another on one stream (without it,
                           consecutive segments run on two streams and overlap) */
  int32_t device;       /* CUDA device ordinal */
  /* Batched DM trials: ndm > 0 makes a batched plan over dm_list[0..ndm) (dm,
   * period and nbins are then ignored and nothing is folded).  Trials that use
   * the same FFT length share one overlap-save segmentation, set by their largest
   * DM, and one forward transform per segment; each trial applies its own chirp
   * and is detected, summed over sub-channels and decimated to its own series.
   * All trials emit the channel samples of the largest DM in the list. */
  int32_t ndm;
  const double* dm_list;
  int64_t nfft_choices[4]; /* FFT lengths the autotuner may use (0 = unused slot) */
  int32_t autotune;     /* nonzero (batched plans): group the DM-sorted trials and give
                           each group one of nfft_choices, minimising the device time per
                           input sample predicted from timed launches of each length
                           (cached per nfft, nchan and device); zero: every trial uses nfft */
  int32_t schedule;     /* POND_SCHEDULE_AUTO or POND_SCHEDULE_FOUR_PASS (below) */
  int32_t input_channels; /* 0 or 1: one int8 sample per byte; 2: the two halves' int8
                             samples interleaved (N0 S0 N1 S1 ...) and added in phase,
                             x[m] = N[m] + S[m] (PONDER's AIP; -256..254): pushes then
                             take whole pairs (an even byte count, POND_E_ARG otherwise)
                             and stats count pairs */
  int32_t trial_mode;   /* batched plans: how the trials of a lane run their per-trial passes
                           (POND_TRIALS_*); 0 = chosen by the autotuner when autotune is set,
                           else the multi-trial table form where the lane's DMs allow it */
  int32_t trials_per_launch; /* batched plans with a multi-trial mode: trials per launch
                                (1 .. 128); 0 = chosen as for trial_mode (default 32) */
  int32_t chirp;        /* single-DM three-pass plans: where the forward row pass takes Eq. 4's
                           inverse filter from (POND_CHIRP_*) */
  int32_t inv_split;    /* log2 Q1 of the four-pass inverse, M = Q1 Q2 (M = nfft / (2 nchan)): I1
                           transforms columns of Q2 = M / Q1 bins of each sub-channel, I2 rows of
                           Q1 (the tile shape of the per-sub-channel inverse).  Used where the plan
                           runs the four-pass inverse: single-DM plans on the four-pass schedule
                           and batched lanes running POND_TRIALS_FOUR_PASS.  0 = the default split
                           (batched plans with autotune: the tuner times the admissible splits).
                           Admissible: 2 <= q <= 12, q <= 13 - log2 nchan, q <= log2 R2 (the
                           forward column length) and 2 <= log2 M - q <= 12, for every FFT length
                           the plan uses; else POND_E_ARG (with nfft_choices, lengths where the
                           split is not admissible are not candidates) */
  int32_t phase_ncoef;  /* single-DM plans: 0 = fold at the constant period_s; 1 .. 8 = fold with
                           the polynomial phase model below instead (Sec. 3.4: the fold period
                           comes from the TEMPO2 predictors): phi(g) = sum_i phase_coef[i] tau^i
                           cycles, tau = g dt_c - phase_tref_s seconds from the first stream
                           sample (dt_c = 2 nchan / fs), by Horner's rule with every FP64 multiply
                           and add rounded on its own; bin = min(floor((phi - floor(phi)) nbins),
                           nbins - 1).  A spin-down model (P, Pdot, epoch t_e) is {phi_0, 1/P,
                           -Pdot / (2 P^2)} about t_e.  period_s is still required (> 0) and is
                           what pond_meta reports.  POND_E_ARG: more than 8 coefficients,
                           non-finite values, or a batched plan */
  double phase_tref_s;
  double phase_coef[8];
} pond_opts;

/* Chirp source of a single-DM plan's fused forward row pass. */
#define POND_CHIRP_AUTO 0     /* this build's default: POND_CHIRP_TABLE (measured faster in the
                                 two-stream pipeline once its rows are prefetched into L2) */
#define POND_CHIRP_ANCHORS 1  /* evaluated per bin from FP64-built anchors (exact Q0.64 phase
                                 polynomial, FP32 sine and cosine): no per-bin memory read, as the
                                 paper's convolution kernel computes the chirp per thread */
#define POND_CHIRP_TABLE 2    /* read per bin from an FP32 (cos, -sin) table built once per plan in
                                 FP64 (8 bytes per bin, nfft * 4 bytes of device memory) */

/* Per-trial passes of a batched lane (one FFT length).  Every trial of the lane
 * shares the lane's forward spectrum; its own passes are the chirp (Eq. 4) with
 * the first inverse factor (row pass), the rest of the sub-channel inverse with
 * detection (column pass) and the decimation. */
#define POND_TRIALS_AUTO 0
#define POND_TRIALS_PER_TRIAL 1    /* three launches per trial, chirp from the trial's anchors */
#define POND_TRIALS_MULTI_ANCHOR 2 /* one launch of each pass over trials_per_launch trials,
                                      chirp from each trial's anchors */
#define POND_TRIALS_MULTI_TABLE 3  /* as POND_TRIALS_MULTI_ANCHOR, chirp from one per-bin
                                      table: the lane's DMs are whole multiples n_d of a step
                                      dDM (e.g. a uniform grid from 0), the table holds the
                                      phase of dDM mod 1 in Q0.32 and trial d's phase is
                                      n_d times it mod 2^32 (exact integer product) */
#define POND_TRIALS_FOUR_PASS 4    /* three launches per trial: I1 (the trial's chirp applied as the
                                      shared spectrum's columns are loaded, inverse columns of Q2),
                                      I2 (inverse rows of Q1, detection, sum over sub-channels) and
                                      the decimation; the split M = Q1 Q2 is opts.inv_split, the
                                      default or the tuner's.  Lanes without the three-pass geometry
                                      (M = 64 R2) always run this form */

/* Fold metadata returned with a profile snapshot. */
typedef struct {
  int32_t epoch_mjd_day;  /* epoch of phase 0 = time of the first stream sample */
  double epoch_mjd_sec;
  double period_s;
  double dm;
  double dtc_s;           /* channel sample time, 2 nchan / fs */
  int64_t first_g;        /* first emitted channel sample (= n_past) */
  int64_t nsamples;       /* channel samples folded so far */
  int32_t nbins;
} pond_meta;

/* A single-pulse candidate of the boxcar detector. */
typedef struct {
  int32_t trial;    /* DM trial (row of the series block) */
  int32_t width;    /* boxcar width w* in series samples (1, 2, 4, ..., 64) */
  int64_t index;    /* series sample where the boxcar starts */
  double snr;       /* S/N at (trial, index, width) */
  double dm;        /* DM of the trial (pond_candidates; 0 from pond_boxcar) */
  float score;      /* classifier score, -1 when not scored */
  int32_t reserved;
} pond_cand;

/* Counters and per-stage GPU time (ms; stage times only with opts.timing). */
#define POND_NSTAGE 9
typedef struct {
  int64_t samples_in;       /* int8 samples accepted */
  int64_t segments;         /* segments processed */
  int64_t outputs;          /* channel samples emitted (detected, folded, decimated) */
  int64_t n_past, n_fut;    /* overlap discarded at each segment edge, channel samples */
  int64_t seg_step;         /* real samples between segment starts */
  int32_t nfft, nchan;
  int32_t kernel_launches;  /* kernels launched since the plan or the last pond_reset */
  int32_t flushed;
  double stage_ms[POND_NSTAGE];   /* accumulated GPU time per stage */
  int64_t stage_launches[POND_NSTAGE];
  double pass_bytes[POND_NSTAGE]; /* DRAM bytes one launch of each stage moves at its own
                                     minimum (its input once and its output once); the
                                     method's own minimum is the int8 input, 1 byte per
                                     sample read, plus the small outputs */
  const char* stage_name[POND_NSTAGE];
  double algo_flops[POND_NSTAGE]; /* algorithmic FP32 operations per launch of each stage:
                                     5 n log2 n per length-n complex FFT factor, 10 per bin
                                     for the real-input split, 6 per bin for the chirp
                                     multiply (Eq. 4), 4 per detected channel sample
                                     (|v|^2 and the sub-channel sum), 1 per sample for the
                                     in-phase sum of two halves, fold and decimation */
  double push_enqueue_ms;   /* host time of the last pond_push spent enqueueing copies and passes */
  double push_wait_ms;      /* host time of the last pond_push spent waiting for its last copy */
} pond_stats_t;

/*
 * pond_plan / pond_plan_ex: create a handle for one stream.
 *   out     : receives the handle (set to NULL on error).
 *   The plan derives the overlap-save geometry: n_past = ceil(K DM (f0^-2 -
 *   f_hi^-2) / dtc), n_fut = ceil(K DM (f_lo^-2 - f0^-2) / dtc) channel
 *   samples (Sec. 3.7: the impulse response must span the smear), the
 *   segment step S_c = M - n_past - n_fut channel samples (S = 2 nchan S_c real
 *   samples), and builds the FFT twiddle and chirp tables on the device in FP64.
 *   Supported: 2^5 <= nfft <= 2^25; nchan <= 2048 with M = nfft/(2 nchan) >= 16.
 *   With precision POND_SPLIT_BF16 / POND_SPLIT_BF16_5T every radix-16 stage of
 *   the four FFT passes multiplies 16-point blocks by the DFT matrix on the
 *   tensor cores (tcgen05, FP32 accumulators); radix-2/4/8 stages, twiddles, the
 *   chirp (FP64 phase argument) and detection stay as in POND_FP32.
 *   Errors: POND_E_ARG (including an unknown precision), POND_E_NFFT,
 *   POND_E_NCHAN, POND_E_OOM, POND_E_CUDA.
 * pond_plan uses t_dec = 61.44 us, epoch 0, FP32, device 0.
 */
int pond_plan(pond_t* out, double f0_mhz, double bw_mhz, double fs_hz, double dm,
              int64_t nfft, int32_t nchan, int32_t nbins, double period_s);
int pond_plan_ex(pond_t* out, const pond_opts* opts);

/*
 * pond_push: append n int8 samples from HOST memory x (any n >= 0).  This is
 *   the input of the paper's GPU flow (Sec. 3.7, Fig. "gpuflow": the digitised
 *   voltages held on the host are sent to the device's global memory; Sec. 3.1:
 *   the ADC delivers 8-bit real samples of each half of the band).  The data
 *   move to the device in pieces of 128 MiB through two staging buffers while
 *   the passes run: page-locked (pinned, device-mapped) memory by a copy kernel
 *   on 8 CTAs that reads it over the host link, pageable memory by the copy
 *   engines.  The data are copied to the device before the call returns (pinned memory copies
 *   asynchronously, pageable memory through the driver's staging), so x may be
 *   reused at once; processing of complete segments continues asynchronously.
 *   Errors: POND_E_ARG (x NULL with n > 0), POND_E_STATE (after pond_flush),
 *   POND_E_CUDA.
 */
int pond_push(pond_t h, const int8_t* x, size_t n);

/*
 * pond_push_device: append n int8 samples already in DEVICE memory d_x (the
 *   same input as pond_push, Sec. 3.7, for a caller whose samples are already
 *   in global memory, skipping the host-to-device copy of the flow).  All
 *   work is enqueued on cuda_stream (a cudaStream_t; NULL = the handle's own
 *   stream, which then waits for the legacy default stream), in stream order,
 *   and reads d_x directly for segments that lie inside it.  d_x must stay
 *   valid and unmodified until the work enqueued on cuda_stream has finished;
 *   the library itself does not touch d_x after that work completes.
 *   Errors: as pond_push.
 */
int pond_push_device(pond_t h, const int8_t* d_x, size_t n, void* cuda_stream);

/*
 * pond_flush: end of stream (Sec. 3.7: the overlap-save segmentation keeps
 *   only outputs whose filter support lies inside the data, so the last
 *   segment is completed here).  Processes the zero-padded tail and emits every
 *   output whose support lies inside the stream (g < floor(n_total/(2 nchan))
 *   - n_fut), then waits for the device.  Further pushes return POND_E_STATE.
 *   Errors: POND_E_CUDA; POND_E_TIMEOUT when a tensor-core stage's bounded wait
 *   for its MMAs expired (the outputs are then invalid).
 */
int pond_flush(pond_t h);

/*
 * pond_sync: wait until all work enqueued for the handle has finished.
 *   Errors: as pond_flush.
 */
int pond_sync(pond_t h);

/*
 * pond_reset: start a new stream with the same plan.  Waits for the device,
 *   then clears the profile, the time series, the kept voltages, the carried
 *   samples and the counters; the plan's tables and buffers are kept.
 */
int pond_reset(pond_t h);

/*
 * pond_profile: snapshot of the folded profile (Sec. 3.7: the last thread of
 *   the GPU flow folds the dedispersed series to the required number of bins;
 *   the fold thread of Sec. 3.4 folds at the period from the timing model, here
 *   a constant period with the epoch at the first stream sample).
 *   Non-destructive; waits for the device; POND_E_STATE for a batched plan,
 *   which does not fold.  sum[b] (FP64) is the sum of detected power P[g] over the channel
 *   samples folded into bin b = min(floor(frac(g dtc / P) nbins), nbins-1)
 *   (phase in FP64, epoch = first stream sample), hits[b] their count; the
 *   mean profile is sum/hits.  sum and hits hold nbins entries; either may be
 *   NULL.  meta may be NULL.  Errors: POND_E_ARG, POND_E_CUDA.
 */
int pond_profile(pond_t h, double* sum, int64_t* hits, pond_meta* meta);

/*
 * pond_trials: the DM and the FFT length of each trial (in the order of
 *   dm_list; a single-DM plan has one trial).  dm and nfft (nullable) hold cap
 *   entries; *ntrials receives the number of trials.
 */
int pond_trials(pond_t h, double* dm, int64_t* nfft, int32_t cap, int32_t* ntrials);

/*
 * pond_tuning: how each lane of a batched plan runs its trials (the
 *   autotuner's choices).  Lanes in increasing FFT length; out holds cap
 *   entries and *nlanes receives the number of lanes.  With autotune, each
 *   lane's candidates were timed on the lane's own buffers with CUDA events
 *   and the fastest per trial is the one used: in lanes with the three-pass
 *   geometry the per-trial launches and the multi-trial forms (8 or 32 trials
 *   per launch, anchors or table), in every lane the four-pass form at up to
 *   four admissible inverse splits (the default and its nearest neighbours;
 *   only opts.inv_split when it is set).  The choice is cached per (nfft,
 *   nchan, device, trial count, inv_split).  A single-DM plan has one lane:
 *   mode POND_TRIALS_PER_TRIAL, or POND_TRIALS_FOUR_PASS on the four-pass
 *   schedule.
 */
#define POND_TUNE_MAXCAND 12
typedef struct {
  int64_t nfft;
  int32_t ntrials;
  int32_t mode;               /* POND_TRIALS_PER_TRIAL, _MULTI_ANCHOR, _MULTI_TABLE or _FOUR_PASS */
  int32_t trials_per_launch;
  int32_t ncand;              /* candidates timed (0 without autotune) */
  int32_t inv_split;          /* log2 Q1 of the lane's four-pass inverse (used by mode _FOUR_PASS) */
  int32_t reserved;
  double dm_step;             /* the table form's dDM (0 when the DMs allow no table) */
  int32_t cand_mode[POND_TUNE_MAXCAND];
  int32_t cand_kt[POND_TUNE_MAXCAND];
  int32_t cand_split[POND_TUNE_MAXCAND];   /* log2 Q1 of a _FOUR_PASS candidate, else 0 */
  double cand_us[POND_TUNE_MAXCAND];   /* device time per trial and segment, us */
} pond_lane_info;
int pond_tuning(pond_t h, pond_lane_info* out, int32_t cap, int32_t* nlanes);

/*
 * pond_timeseries: drain completed samples of the decimated time series
 *   (Sec. 3.7: the dedispersed series is the output of the flow; Sec. 3.4:
 *   detected power is added to reach the desired time resolution).
 *   Sample j sums P[g] over the emitted g with floor(g / D) = j, where
 *   D = t_dec fs / (2 nchan) channel samples (an exact rational; with 4 us
 *   channel samples and t_dec = 61.44 us, bins hold 15 or 16 samples).
 *   counts[j] (nullable) is the number of channel samples summed; the first
 *   and last samples of a stream may be partial.  Copies at most cap samples
 *   into out; *n_out receives the number copied and *first_index the j of
 *   out[0] (both required).  A batched plan writes trial d's samples at
 *   out[d * cap + i] (out holds ndm * cap floats); counts are common to all trials.  Samples are complete once every g they cover has
 *   been processed; after pond_flush all remaining samples are complete.
 *   When out (or counts) is page-locked host memory (cudaMallocHost,
 *   cudaHostRegister) the device's rows are copied into it directly; other
 *   host memory receives them through the handle's pinned row buffer.
 */
int pond_timeseries(pond_t h, float* out, int32_t* counts, size_t cap, size_t* n_out,
                    int64_t* first_index);

/*
 * pond_voltages: drain dedispersed sub-channel voltages v_c[g] (complex, FP32
 *   re/im pairs) of the emitted channel samples: the output of the inverse FFT
 *   after multiplication by the inverse of H (Sec. 3.7, Eq. 4), before the
 *   power detection of Sec. 3.4; only with opts.want_voltages (tests).
 *   out_c is laid out [nchan][cap][2]; at most cap samples per channel are
 *   copied; *n_out receives the number per channel, *first_g the g of the first.
 *   Errors: POND_E_STATE when the plan was made without want_voltages.
 */
int pond_voltages(pond_t h, float* out_c, size_t cap, size_t* n_out, int64_t* first_g);

/*
 * pond_boxcar: boxcar S/N single-pulse search over a block of dedispersed
 *   series (automatic transient detection is the paper's plan in Sec. 5).
 *   d_series: DEVICE float [ndm][stride], n samples per row (stride >= n).
 *   Per row d: mu = median, sigma = 1.4826 x median absolute deviation (exact
 *   order statistics; an even count takes the FP64 mean of the middle two);
 *   S_w(t) = (sum_{i<w} T[t+i] - w mu) / (sigma sqrt(w)) for w = 1, 2, ..., 64
 *   with the sum in FP64 in index order; s(t) = max_w S_w(t) with its smallest
 *   maximising width w*; (d, t) is a candidate when s >= threshold and no
 *   point within 2 rows and w* samples has a larger s (equal s: the earlier
 *   point in (row, sample) order wins).  A row with sigma = 0 has none.
 *   Candidates go to HOST out[cap], sorted by (trial, index); *n_found gets
 *   their number.  Allocates device scratch (8 + 1 bytes per series sample).
 *   Work runs on cuda_stream and the call waits for it.
 *   Errors: POND_E_ARG, POND_E_OVERRUN (more candidates than cap; *n_found is
 *   the number found), POND_E_OOM, POND_E_CUDA.
 */
int pond_boxcar(const float* d_series, int32_t ndm, int64_t n, int64_t stride, double threshold,
                pond_cand* out, size_t cap, size_t* n_found, void* cuda_stream);

/*
 * pond_candidates: pond_boxcar over the handle's completed series samples that
 *   have not been drained yet (all trials of a batched plan), with index = the
 *   series sample index j and dm = the trial's DM.  Call it before
 *   pond_timeseries drains the samples.  Sec. 5 names automatic detection of
 *   transients as the paper's plan; the detector is this library's.  Besides
 *   the handle and the output array it takes the S/N threshold (the boxcar's
 *   detection level, 6 in the learned form), so callers choose it per call.
 */
int pond_candidates(pond_t h, double threshold, pond_cand* out, size_t cap, size_t* n_found);

/*
 * Single-pulse candidate classifier (automatic transient detection is the
 * paper's plan in Sec. 5; the network is this library's).  Input: patches of
 * 32 DM trials x 256 series samples, BF16 [batch][32][256] in device memory
 * (see pond_patches).  Network: 3 x [Conv1d(32 -> 32, kernel 7, zero padding
 * 3) + ReLU], 2:1 max-pool after the first two, global average over time,
 * Linear(32 -> 4), softmax over {dispersed pulse, broadband RFI, narrowband
 * RFI, noise}.  Parameters (POND_CNN_NPARAM FP32 values, flat): for each conv
 * layer w[co][ci][k] then b[co]; then fc w[4][32], fc b[4].  BF16 weights and
 * activations, FP32 accumulation and master weights; training minimises the
 * batch-mean cross-entropy with Adam (beta1 0.9, beta2 0.999, eps 1e-8).
 * Weight gradients are reduced over the batch in sample order (deterministic).
 * A network belongs to one device and one thread at a time.
 */
#define POND_CNN_NPARAM 21732
typedef struct pond_cnn_s* pond_cnn_t;
/* create with host initial parameters; scratch for batches up to max_batch */
int pond_cnn_create(pond_cnn_t* out, const float* init_params, int32_t max_batch, int32_t device);
/* replace the parameters (host) and reset the Adam state */
int pond_cnn_set_params(pond_cnn_t net, const float* params);
/* copy the FP32 master parameters to host memory */
int pond_cnn_params(pond_cnn_t net, float* out);
/* class probabilities of a batch: d_prob (device) [batch][4] */
int pond_cnn_forward(pond_cnn_t net, const void* d_x, int32_t batch, float* d_prob, void* cuda_stream);
/* gradient of the batch-mean cross-entropy (host [POND_CNN_NPARAM], nullable) and
 * the loss (host, nullable), without updating; labels are device int32 [batch] */
int pond_cnn_gradient(pond_cnn_t net, const void* d_x, const int32_t* d_labels, int32_t batch,
                      float* grad_out, float* loss_out, void* cuda_stream);
/* one Adam step on a batch; loss_out (host, nullable) receives the loss before it */
int pond_cnn_train_step(pond_cnn_t net, const void* d_x, const int32_t* d_labels, int32_t batch,
                        float lr, float* loss_out, void* cuda_stream);
int pond_cnn_destroy(pond_cnn_t net);

/*
 * pond_patches: cut classifier patches from a series block [ndm][stride]
 *   (DEVICE float, n samples per row).  Patch p covers rows d0..d0+31 and
 *   samples t0..t0+255 with (d0, t0) = d_corners[2p], d_corners[2p+1] (device
 *   int32); rows and samples outside the block repeat the nearest edge.  Each
 *   patch is shifted to zero mean and scaled to unit standard deviation (FP32;
 *   a constant patch keeps scale 1) and stored as BF16 [npatch][32][256].
 */
int pond_patches(const float* d_series, int32_t ndm, int64_t n, int64_t stride, const int32_t* d_corners,
                 int32_t npatch, void* d_out, void* cuda_stream);

/*
 * pond_candidates_scored: pond_candidates, then each candidate's patch
 *   (trials trial-16 .. trial+15, clamped into the block, and series samples
 *   index-128 .. index+127 of the same undrained block, cut as by
 *   pond_patches) is classified by net on the handle's device and stream;
 *   score = the network's probability of the dispersed-pulse class.  net must
 *   live on the handle's device.  Allocates device scratch for the block, the
 *   patches (16 KiB each) and the probabilities; batches are at most the
 *   network's max_batch.  Errors: as pond_candidates; POND_E_ARG for a null
 *   net.
 */
int pond_candidates_scored(pond_t h, pond_cnn_t net, double threshold, pond_cand* out, size_t cap,
                           size_t* n_found);

/*
 * pond_check_bounded_wait: self-check of the bounded device wait the
 *   tensor-core stages use for their MMA completions.  One CTA on `device`
 *   waits on a barrier that nothing ever arrives on, polling it against the
 *   GPU's global timer with a limit of limit_s seconds (0 < limit_s <= 10);
 *   *waited_s receives how long it waited.  Returns POND_E_TIMEOUT when the
 *   wait gave up (the expected result: the kernel ended by itself and the
 *   context stays usable), POND_OK if the barrier somehow completed,
 *   POND_E_ARG or POND_E_CUDA otherwise.
 */
int pond_check_bounded_wait(double limit_s, int32_t device, double* waited_s);

/*
 * pond_probe_fp32_fma: measure the FP32 arithmetic ceiling of the current
 *   device.  The FFT butterflies of Sec. 3.7's forward and inverse transforms
 *   are FP32 multiply-adds, so this is the roofline that bounds the path at
 *   its algorithmic minimum of DRAM traffic.  Enqueues one kernel on
 *   cuda_stream (NULL = legacy default stream): `blocks` CTAs of 512 threads,
 *   each thread running 8 independent FMA chains for iters x 16 steps, and
 *   writes one float per thread to d_out (DEVICE, blocks x 512 floats, caller
 *   owned).  *flops (host) receives the FP32 operations enqueued (2 per FMA);
 *   time the launch with events on cuda_stream.  Returns at once.
 *   Errors: POND_E_ARG (null pointer, blocks or iters < 1), POND_E_CUDA.
 */
int pond_probe_fp32_fma(float* d_out, int32_t blocks, int32_t iters, void* cuda_stream, double* flops);

/* pond_stats: counters and per-stage GPU times (waits for the device).  The
 * stage times give the paper's measure of real-time capability, the compute
 * to observed ratio (Sec. 3.4: processing time over digitisation time, which
 * must stay below 1), as stage time over samples_in / fs. */
int pond_stats(pond_t h, pond_stats_t* s);

/*
 * pond_fold_noalloc: fold n detected power samples d_power[0..n) (device,
 *   FP32), which are the channel samples g0 .. g0+n-1, into a caller-owned
 *   profile, ADDING to d_sum[nbins] (device, FP64) and d_hits[nbins] (device,
 *   int64); zero them before the first call.  The bin of g is the engine's:
 *   min(floor(frac(g * (dtc_s / period_s)) * nbins), nbins - 1) in FP64, so
 *   with dtc_s = 2 nchan / fs the result matches pond_profile bin for bin.
 *   The paper has no counterpart: this entry point exists for callers that
 *   cannot allocate device memory (a real-time thread that must not stall on
 *   cudaMalloc/cudaFree, which can synchronise the device, or a host
 *   application whose memory manager owns all device allocations).  It
 *   allocates nothing: its scratch (per-CTA partial histograms) is one fixed
 *   3.6 MiB device array that every GPU loading the library holds until the
 *   process exits, so nbins is limited to POND_NOALLOC_MAX_NBINS.  The work
 *   is enqueued on cuda_stream (a cudaStream_t of the current device, NULL =
 *   legacy default stream).  The first call on a device looks up the array's
 *   device address; make that first call before any stream capture.  That
 *   address is cached per device for the life of the process: after a
 *   cudaDeviceReset it is stale, so do not call this entry point again in
 *   that process.  All calls share the one array: calls that overlap on the
 *   GPU (other streams, other threads) race and must be serialised by the
 *   caller.  Each call overwrites the partial rows it reads, so nothing in
 *   the array needs clearing between calls.
 *   Accumulation: a call never overwrites d_sum / d_hits; it adds its n
 *   samples to them, so a profile can be built over many calls.
 *   Limit per call: a CTA counts its hits in int32 over about n / 304
 *   samples, so n may not exceed POND_NOALLOC_MAX_SAMPLES (2^39, about
 *   5.5e11, 4.8 hours of 32 MS/s channel samples); split longer series over
 *   several calls.
 *   Errors: POND_E_ARG (nbins > POND_NOALLOC_MAX_NBINS or < 1, n < 0,
 *   n > POND_NOALLOC_MAX_SAMPLES, g0 < 0, dtc_s or period_s <= 0, null
 *   pointer with n > 0), POND_E_CUDA.
 */
#define POND_NOALLOC_MAX_NBINS 1024
#define POND_NOALLOC_MAX_SAMPLES (1LL << 39)
int pond_fold_noalloc(const float* d_power, int64_t n, int64_t g0, double dtc_s, double period_s,
                      int32_t nbins, double* d_sum, int64_t* d_hits, void* cuda_stream);

/*
 * Fold with a polynomial phase model into a pulse stack (the fold of Sec. 3.4
 * with the period of a timing model, as PONDER takes it from TEMPO2 predictors;
 * the single-pulse stack of Sec. 4).  Series sample i is sample g = g0 + i of
 * spacing dt_s from the first stream sample; its phase is
 *   phi = sum_{k < ncoef} coef[k] tau^k,  tau = g dt_s - t_ref_s  (cycles),
 * evaluated by Horner's rule with every multiply and add rounded on its own in
 * FP64 (a spin-down model: coef = {phase0, 1/P, -Pdot/(2 P^2)}).  Rotation
 * q = floor(phi), bin b = min(floor((phi - q) nbins), nbins - 1): with coef
 * {0, 1/P} the bins are the constant-period fold's when g dt / P rounds as g
 * (dt / P) does.  Rows: POND_STACK_ROTATION, one per rotation from the first
 * sample's (row = q - first_rotation); POND_STACK_SUBINT, one per n_sub samples
 * (row = i / n_sub).  Cell (row, b) receives the FP64 sum of its samples, added
 * in sample order, and their count.
 */
#define POND_STACK_ROTATION 0
#define POND_STACK_SUBINT 1

/* pond_stack_rows: the number of rows pond_fold_stack fills for these arguments
 * and the first sample's rotation (host arithmetic only).  Errors: POND_E_ARG
 * (n or g0 < 0, dt_s <= 0, ncoef outside 1..8, nbins outside 1..4096, bad mode,
 * n_sub < 1 for SUBINT, a non-finite coefficient, null pointer). */
int pond_stack_rows(int64_t n, int64_t g0, double dt_s, const double* coef, int32_t ncoef, double t_ref_s,
                    int32_t nbins, int32_t mode, int64_t n_sub, int64_t* rows, int64_t* first_rotation);

/* pond_fold_stack: fold d_series[0..n) (device, FP32) into the caller-owned
 * stack d_sum[rows][nbins] (device, FP64) and d_hits[rows][nbins] (device,
 * int64), every cell written (rows as pond_stack_rows returns them, at most
 * rows_cap); *rows and *first_rotation as from pond_stack_rows.  Work is
 * enqueued on cuda_stream (NULL = legacy default stream); the call waits for a
 * check that the phase model runs forwards over the whole series (a
 * non-decreasing (rotation, bin) key, which the stack relies on).  Calls that
 * overlap on the GPU share that check's flag and must be serialised.  Errors:
 * as pond_stack_rows, POND_E_OVERRUN (rows > rows_cap; nothing written),
 * POND_E_ARG (the phase model runs backwards; null device pointer with n > 0),
 * POND_E_CUDA. */
int pond_fold_stack(const float* d_series, int64_t n, int64_t g0, double dt_s, const double* coef, int32_t ncoef,
                    double t_ref_s, int32_t nbins, int32_t mode, int64_t n_sub, double* d_sum, int64_t* d_hits,
                    int64_t rows_cap, int64_t* rows, int64_t* first_rotation, void* cuda_stream);

/* pond_strerror: static text for a return code.  pond_last_error: message of the
 * calling thread's last failure (empty if none). */
const char* pond_strerror(int code);
const char* pond_last_error(void);

/* pond_destroy: wait for the device, release everything the handle owns
 * (the end of an observation; the paper has no passage for it).
 * NULL is accepted. */
int pond_destroy(pond_t h);

/*
 * Incoherent dedispersion modes (PONDER Sec. 3.4, sub-modes AID of Sec. 3.4.1
 * and CID of Sec. 3.4.2): an FFT filterbank over the same band, detected,
 * integrated, shifted per channel by the dispersive delay of Eq. 3, summed over
 * channels and folded.  One call processes one whole device buffer.
 *
 *  - Filterbank: the stream is cut into consecutive blocks of 2 nchan real
 *    samples (no overlap, no window); X[k] = sum_n x[n] exp(-2 pi i k n /
 *    (2 nchan)), k = 0 .. nchan-1 (DC kept, Nyquist dropped).  Channel k sits
 *    at the sky frequency f_k = f0 - |bw|/2 + k |bw|/nchan (bw > 0) or
 *    f0 + |bw|/2 - k |bw|/nchan (bw < 0).
 *  - Detection: AID takes |X[k]|^2 of the single stream (input_channels 1) or
 *    of the two halves added in phase, x = N + S (input_channels 2, bytes
 *    N0 S0 N1 S1 ...); CID takes the cross-power Re(X_N[k] conj(X_S[k])) of
 *    the two halves (input_channels 2).
 *  - Integration: output sample t (t_s = 2 nchan nint / fs seconds) sums the
 *    spectra t nint .. t nint + nint - 1, in that order; T = floor(samples /
 *    (2 nchan nint)) output samples, trailing input is not used.
 *  - Dedispersion: channel k is read d_k samples later, d_k = floor(K DM
 *    (f_k^-2 - f0^-2) / t_s + 1/2) in FP64 (K as for the coherent mode,
 *    delays referred to the band centre); D[t] = sum_k F[t + d_k][k] for
 *    t = t_first .. t_first + n - 1 with t_first = max(0, -min d) and
 *    n = max(0, T - max(0, max d) - t_first).
 *  - Fold: D[t] goes to bin min(floor(frac(t * (t_s / period)) * nbins),
 *    nbins - 1), FP64 phase, epoch at the first input sample.
 * Results are FP32 (filterbank, series) and FP64 / int64 (profile); repeated
 * runs give bit-identical results.
 */
#define POND_INCOH_AID 0   /* adding (in phase) and incoherent dedispersion */
#define POND_INCOH_CID 1   /* correlation and incoherent dedispersion */
typedef struct pond_incoh_s* pond_incoh_t;
typedef struct {
  double f0_mhz, bw_mhz, fs_hz;  /* the band, as for pond_plan (fs = 2 |bw| 1e6) */
  double dm;                     /* >= 0 */
  double period_s;               /* fold period, > 0 */
  int32_t nchan;                 /* filterbank channels: power of two, 64 .. 2048 */
  int32_t nint;                  /* spectra per output sample: power of two, 1 .. 65536 */
  int32_t mode;                  /* POND_INCOH_AID or POND_INCOH_CID */
  int32_t input_channels;        /* AID: 1 or 2; CID: 2 */
  int32_t nbins;                 /* fold bins, 1 .. 4096 */
  int32_t device;                /* CUDA device ordinal */
  int32_t ips_len;               /* 0, or the chunk length L of the fluctuation spectrum
                                    (power of two, 64 .. 4096): see pond_incoh_ips */
  int32_t reserved[5];           /* zero */
} pond_incoh_opts;

/* Counts and device times of the last run (times from CUDA events around each
 * stage, on the run's stream). */
typedef struct {
  int64_t T;             /* filterbank samples */
  int64_t t_first;       /* first dedispersed sample */
  int64_t n_out;         /* dedispersed samples */
  int64_t ips_chunks;    /* complete chunks in the fluctuation spectrum (0 without ips_len) */
  int32_t d_min, d_max;  /* channel delays, output samples */
  double ts;             /* output sample time, s */
  double ms_filterbank, ms_dedisperse, ms_fold, ms_ips;
  double algo_bytes_filterbank;  /* input bytes read + filterbank bytes written */
  double algo_bytes_dedisperse;  /* filterbank bytes read + series bytes written */
  int32_t launches;      /* kernel launches of the run */
  int32_t reserved[3];
} pond_incoh_info;

/* pond_incoh_create: validate opts and allocate the tables.  Errors:
 * POND_E_ARG (band, DM, period, nbins, mode / input_channels, reserved not
 * zero, nint), POND_E_NCHAN (nchan), POND_E_OOM, POND_E_CUDA. */
int pond_incoh_create(pond_incoh_t* out, const pond_incoh_opts* opts);

/* pond_incoh_run: enqueue the whole mode on cuda_stream (a cudaStream_t of the
 * handle's device, NULL = legacy default stream) over nbytes bytes of int8 at
 * d_x (device memory, 16-byte aligned, caller-owned and unchanged until the
 * run completes).  Replaces the previous run's results.  Grows the handle's
 * device buffers (cudaMalloc, which may synchronise) when the input is longer
 * than any before.  Errors: POND_E_ARG (null or misaligned d_x with nbytes >
 * 0, nbytes not a multiple of input_channels), POND_E_OOM, POND_E_CUDA. */
int pond_incoh_run(pond_incoh_t h, const int8_t* d_x, size_t nbytes, void* cuda_stream);

/* pond_incoh_info_get: counts and stage times of the last run (waits for it). */
int pond_incoh_info_get(pond_incoh_t h, pond_incoh_info* info);

/* pond_incoh_filterbank: copy the last run's integrated filterbank to host
 * out[T][nchan] (time-major: one spectrum of nchan channels per output sample,
 * FP32); *T receives the sample count.  Errors: POND_E_OVERRUN if cap (floats)
 * < T nchan (nothing copied, *T still set), POND_E_ARG. */
int pond_incoh_filterbank(pond_incoh_t h, float* out, size_t cap, int64_t* T);

/* pond_incoh_series: copy the dedispersed series to host out[n_out];
 * *n_out and *t_first receive its length and first sample index.  Errors:
 * POND_E_OVERRUN (cap < n_out, nothing copied), POND_E_ARG. */
int pond_incoh_series(pond_incoh_t h, float* out, size_t cap, int64_t* n_out, int64_t* t_first);

/* pond_incoh_profile: copy the folded profile of the last run to host sum[nbins]
 * (FP64) and hits[nbins] (int64). */
int pond_incoh_profile(pond_incoh_t h, double* sum, int64_t* hits);

/* pond_incoh_ips: the fluctuation spectrum of the interplanetary scintillation
 * mode (PONDER Sec. 3.5), computed by every run of a handle created with
 * ips_len = L > 0: the series D is cut into its J = floor(n_out / L) complete
 * chunks of L samples and out[f] = sum_j |sum_u D[j L + u] exp(-2 pi i f u / L)|^2
 * for f = 0 .. L/2 (L/2 + 1 FP64 values; no window, no mean removed; zero when
 * J = 0); *chunks receives J.  With mode CID and dm 0 every channel delay is
 * zero and D is the band-collapsed cross-power series of Sec. 3.5 (its further
 * integration is nint).  Errors: POND_E_STATE (ips_len was 0), POND_E_ARG. */
int pond_incoh_ips(pond_incoh_t h, double* out, int64_t* chunks);

/* pond_incoh_delays: copy the channel delays d_k (output samples) to out[nchan]. */
int pond_incoh_delays(pond_incoh_t h, int32_t* out);

/* pond_incoh_destroy: wait for the device and release the handle (NULL accepted). */
int pond_incoh_destroy(pond_incoh_t h);

#ifdef __cplusplus
}
#endif
#endif /* POND_H */
