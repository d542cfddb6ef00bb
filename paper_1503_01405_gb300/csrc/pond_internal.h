// Internal types shared by the kernels and the C-ABI layer.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "../../include/pond.h"

namespace pond {

constexpr int CHIRP_LOG_MAX = 15;            // at most 2^15 bins per chirp anchor
constexpr int MAX_NBINS = 4096;              // fold bins (per-warp FP64 histograms in smem)
constexpr int MAX_FOLD_PARTS = 304;          // fold CTAs per segment (2 per SM)

// Taylor coefficients of the dedispersion phase phi (cycles) about an anchor
// bin: phi(k_a + d) = phi0 + phi1 d + phi2 d^2 + phi3 d^3.  The first three
// terms are evaluated exactly mod 1 in 64-bit fixed point (d is an integer),
// so only the small cubic term is rounded in FP32.
struct __align__(16) ChirpAnchor {
  unsigned long long p1;   // phi1 mod 1, Q0.64
  unsigned long long p2;   // phi2 mod 1, Q0.64
  unsigned p0;             // phi0 mod 1, Q0.32
  float p3;                // phi3
  unsigned pad[2];
};

// Chirps of the trials of one batched launch.  Table form (the lane's DMs are
// whole multiples n_d of one step dDM): atab[k] = frac(sgn dDM c(f_k)) in Q0.32,
// built once per lane in FP64, and trial d's phase at bin k is n_d atab[k]
// mod 2^32, an exact integer product (its error is n_d times the table's
// rounding, below 2^-33 cycles per step).  Anchor form: each trial's own
// anchor table (chirp_from).
struct MultiChirp {
  const unsigned* atab;            // table form: [L], bin k2 + R2 k1 at k2 R1 + k1
  const unsigned* nmul;            // table form: per trial of the launch, n_d
  const ChirpAnchor* const* anc;   // anchor form: per trial of the launch
  const int* clog;                 // anchor form: per trial of the launch
};

// Two-level twiddle table for exponents e < n: w^e = hi[e >> 12] * lo[e & 4095].
constexpr int TW2_LOG = 12;
constexpr int TW2_LO = 1 << TW2_LOG;
struct Tw2 {
  const float2* lo;
  const float2* hi;
};

// A segment's int8 input as up to two runs: samples [0, a_len) from a,
// [a_len, a_len + b_len) from b, zeros beyond.
// One segment's input: bytes [0, a_len) of run a, then [0, b_len) of run b, then
// zeros.  Real sample m is byte m (ch = 1) or the sum of bytes 2m, 2m + 1 (ch = 2:
// the two halves' interleaved int8 samples, added in phase); a_len is a whole
// number of samples.
struct SegIn {
  const int8_t* a;
  long long a_len;
  const int8_t* b;
  long long b_len;
  int vec8;   // ch 1, both runs 8-byte aligned with a_len % 8 == 0: F1 may load 8 bytes at a time
  int ch = 1;
  int pair4 = 0;  // ch 2, both runs 4-byte aligned with a_len, b_len % 4 == 0: F1 may load
                  // one complex sample's two N / S pairs (4 bytes) at a time
};

constexpr int TC_W_BYTES = 3 * 32 * 32 * 2;   // W16 hi, mid, lo parts of one direction

// Tensor-core stage arguments: the W16 parts of one transform direction
// (hi, mid, lo BF16 in the operand layout, 6 KiB), the product terms (3 or 5)
// and the plan's error flag (set when a bounded MMA wait expires).
struct TcArgs {
  const uint4* w;
  int terms;
  int* err;
};

// Geometry of a plan: segment and pass decomposition.
struct Geom {
  long long N, L, M;     // real samples per segment, spectrum bins kept, samples per sub-channel
  int nchan;
  int logL, logM;
  int logR1, logR2;      // forward: L = R1 * R2 (F2 rows of R1, F1 columns of R2)
  int logQ1, logQ2;      // inverse: M = Q1 * Q2 (I2 rows of Q1, I1 columns of Q2)
  long long n_past, n_fut, S_c, S;
  int sms;               // streaming multiprocessors of the device
  int tc_terms = 0;      // 0: FP32 stages; 3 or 5: split-BF16 tensor-core radix-16 stages
  TcArgs tc_fwd{}, tc_inv{};
};

cudaError_t set_kernel_attributes();
// Largest batch a classifier accepts (its scratch size).
int cnn_max_batch(pond_cnn_t net);
cudaError_t set_kernel_attributes_tc();
// One CTA waiting on a barrier nothing arrives on (bounded by limit_ns); status 1 = gave up.
cudaError_t launch_wait_probe(unsigned long long limit_ns, int* status, unsigned long long* waited);
// W16 parts for the tensor-core stages, host-built: [fwd, inv][hi, mid, lo] in
// the K-major operand layout (2 x 6 KiB).
void build_w16_parts(uint16_t* out);
int run_boxcar(const float* d_series, int ndm, long long n, long long stride, double thr, pond_cand* host_out,
               size_t cap, size_t* n_found, cudaStream_t st);
// Record msg as the calling thread's last error (pond_last_error) and return code.
int set_error(int code, const char* msg);
cudaError_t launch_tables(ChirpAnchor* anc, long long nanc, int clog, double du, double half,
                          double f0, double alpha, int sgn, cudaStream_t st);
cudaError_t launch_tw2(float2* lo, float2* hi, int logn, int sign, cudaStream_t st);
// Three-level table (768 entries) of w^e, w = exp(sign 2 pi i / 2^logn), e < 2^24.
cudaError_t launch_tw3(float2* out, int logn, int sign, cudaStream_t st);
cudaError_t launch_stage_tw(float2* out, int R, cudaStream_t st);
int stage_tw_entries(int R);
cudaError_t launch_fwd_cols(const Geom& g, SegIn in, float2* out, const float2* tw, cudaStream_t st);
cudaError_t launch_fwd_rows(const Geom& g, const float2* in, float2* out, const float2* tw3L, Tw2 tw2L, const float2* tw,
                            cudaStream_t st);
cudaError_t launch_inv_cols(const Geom& g, const float2* in, float2* out, const ChirpAnchor* anc,
                            int clog, const float2* tw, cudaStream_t st);
cudaError_t launch_inv_rows(const Geom& g, const float2* buf, float* P, float2* vout, long long vstride,
                            long long vofs, int m_lo, int m_hi, const float2* tw3M, const float2* tw,
                               cudaStream_t st);
// Fused schedule (F1, F2f, Ic) for single-trial FP32 plans whose geometry has
// J = M / R2 = FUSED_J; fused_groups = sub-channel groups per m1 in Ic.
constexpr int FUSED_J = 64;
bool fused_geometry(const Geom& g);
int fused_groups(const Geom& g);
// ctab non-null: the chirp from that per-bin table (launch_chirp_c64), else from the anchors
cudaError_t launch_fwd_rows_inv(const Geom& g, const float2* in, float2* out, const float2* tw3L, Tw2 tw2L,
                                const float2* tw, const float2* twJ, const ChirpAnchor* anc, int clog,
                                const float2* ctab, cudaStream_t st);
cudaError_t launch_chirp_c64(float2* tab, const Geom& g, double du, double half, double f0, double alpha, int sgn,
                             cudaStream_t st);
cudaError_t launch_inv_rows_chirp(const Geom& g, const float2* in, float2* out, const float2* tw3L, const float2* twJ,
                                  const ChirpAnchor* anc, int clog, cudaStream_t st);
// ntr > 1: one launch over ntr trials, trial t reading in + t L and writing
// P + t M, part + t G M, cnt + t FUSED_J (G = fused_groups)
cudaError_t launch_inv_cols_det(const Geom& g, const float2* in, float* P, float* part, int* cnt, float2* vout,
                                long long vstride, long long vofs, int m_lo, int m_hi, const float2* tw,
                                cudaStream_t st, int ntr = 1);
// Batched lanes: Ir over ntr trials in one launch (trial t writes out + t L),
// the chirp from the lane's Q0.32 table (table = true) or each trial's anchors
cudaError_t launch_inv_rows_chirp_multi(const Geom& g, const float2* in, float2* out, int ntr, const float2* tw3L,
                                        const float2* twJ, MultiChirp mc, bool table, cudaStream_t st);
// Tensor-core column pass (split-BF16, three terms) for R2 = 2048 and at least
// four sub-channels: same outputs and arguments as launch_inv_cols_det, plus
// its operand block (build_ic_tc_ops, ic_tc_ops_bytes() bytes on the device)
// and the plan's MMA-wait error flag.
bool ic_tc_geometry(const Geom& g);
cudaError_t launch_inv_cols_det_tc(const Geom& g, const float2* in, float* P, float* part, int* cnt, float2* vout,
                                   long long vstride, long long vofs, int m_lo, int m_hi, const uint4* ops, int* err,
                                   cudaStream_t st, int ntr = 1);
void build_ic_tc_ops(unsigned char* out);
int ic_tc_ops_bytes();
// Device-to-device byte copy as a kernel (the carry rewrite between pushes).
cudaError_t launch_copy_bytes(int8_t* dst, const int8_t* src, long long n, cudaStream_t st);
// Host-to-device copy from mapped pinned memory by `blocks` CTAs (the copy engines are not used).
cudaError_t launch_copy_host(int8_t* dst, const int8_t* src, long long n, int blocks, cudaStream_t st);
cudaError_t launch_chirp_table(unsigned* tab, const Geom& g, double du, double half, double f0, double alpha, int sgn,
                               cudaStream_t st);
cudaError_t launch_decimate_multi(const float* P, long long pstride, long long n, long long g0, long long num,
                                  long long den, long long j_lo, long long nj, float* T, int* C, long long ring,
                                  const int* rows, int ntr, cudaStream_t st);
size_t fold_smem_bytes(int nbins);
int fold_parts(long long n, long long* chunk);
cudaError_t launch_fold(const float* P, long long n, long long g0, double inc, int nbins, double* psum,
                        int* phits, double* prof_sum, long long* prof_hits, cudaStream_t st);
// The fold's phase rule: nc = 0 folds at the constant period (phase g inc);
// 1 <= nc <= 8 evaluates the polynomial phi = sum_i c[i] tau^i, tau = g dt - t_ref
// (Horner's rule, every FP64 operation rounded on its own).
struct FoldPhase {
  double inc = 0;
  int nc = 0;
  double dt = 0, t_ref = 0;
  double c[8] = {};
};
// Fold + decimation of one segment (single-DM plans): the fold adds to
// per-CTA partial rows [MAX_FOLD_PARTS][nbins] that accumulate over the
// stream; launch_fold_snapshot merges them into the profile (replacing it).
cudaError_t launch_fold_dec(const float* P, long long n, long long g0, const FoldPhase& ph, int nbins, long long num,
                            long long den, long long j_lo, long long nj, float* T, int* C, long long ring,
                            double* psum, long long* phits, cudaStream_t st);
cudaError_t launch_fold_snapshot(const double* psum, const long long* phits, int nbins, double* prof_sum,
                                 long long* prof_hits, cudaStream_t st);
cudaError_t launch_decimate(const float* P, long long n, long long g0, long long num, long long den,
                            long long j_lo, long long nj, float* T, int* C, long long ring, cudaStream_t st);

}  // namespace pond
