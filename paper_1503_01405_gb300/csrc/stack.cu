// Fold with a polynomial phase model into a pulse stack (PONDER Sec. 3.4: the
// fold uses the period predicted by TEMPO2; Sec. 4: a stack of single pulses,
// one row per rotation).
//
// phi(g) = sum_i c_i tau^i, tau = g dt - t_ref, by Horner's rule with every
// multiply and add rounded on its own (explicit _rn intrinsics, no contraction;
// the host evaluates the same expression with products kept unfused), so that
// rotation q = floor(phi) and bin b = min(floor((phi - q) nbins), nbins - 1)
// are decided exactly as a plain FP64 evaluation decides them.
//
// The key K(g) = q nbins + b never decreases along the series for a phase
// model that runs forwards (checked first, by k_stack_check), so the samples of
// one (rotation, bin) pair form one contiguous run.  One thread per stack cell
// (row, bin) finds the runs of its rotations by binary search on K and adds
// their samples in sample order in FP64: no atomics, no partials to merge, and
// the sums are those of a sequential loop over the series.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <string>

#include "../../include/pond.h"
#include "pond_internal.h"

namespace {

constexpr int MAX_COEF = 8;
constexpr int CELL_THREADS = 256;

struct PhaseModel {
  double c[MAX_COEF];
  int nc;
  double dt, t_ref;
  long long g0;
  int nbins;
};

struct Key {
  long long q;   // rotation
  int b;         // bin
};

__device__ __forceinline__ Key key_at(const PhaseModel& m, long long i) {
  const double tau = __dsub_rn(__dmul_rn((double)(m.g0 + i), m.dt), m.t_ref);
  double x = m.c[m.nc - 1];
  for (int k = m.nc - 2; k >= 0; --k) x = __dadd_rn(__dmul_rn(x, tau), m.c[k]);
  const double q = floor(x);
  const int b = (int)__dmul_rn(__dsub_rn(x, q), (double)m.nbins);
  return Key{(long long)q, b < m.nbins - 1 ? b : m.nbins - 1};
}

__device__ __forceinline__ long long key_value(const PhaseModel& m, long long i) {
  const Key k = key_at(m, i);
  return k.q * m.nbins + k.b;
}

// Lowest i in [lo, hi] with K(g0 + i) >= K (hi when there is none).
__device__ long long first_at_or_after(const PhaseModel& m, long long lo, long long hi, long long K) {
  while (lo < hi) {
    const long long mid = lo + ((hi - lo) >> 1);
    if (key_value(m, mid) >= K) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

__device__ int g_backwards;   // set when K decreases somewhere along the series

__global__ void k_stack_check(PhaseModel m, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i + 1 < n;
       i += (long long)gridDim.x * blockDim.x)
    if (key_value(m, i + 1) < key_value(m, i)) g_backwards = 1;
}

// Cell (row, b): ROTATION rows are rotations q_first + row; SUBINT rows are the
// samples [row n_sub, min(n, (row + 1) n_sub)) with every rotation they touch.
__global__ void __launch_bounds__(CELL_THREADS) k_stack_cells(const float* __restrict__ y, long long n, PhaseModel m,
                                                              int mode, long long n_sub, long long q_first,
                                                              long long rows, double* __restrict__ S,
                                                              long long* __restrict__ H) {
  const long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (cell >= rows * m.nbins) return;
  const long long row = cell / m.nbins;
  const int b = (int)(cell - row * m.nbins);
  long long lo = 0, hi = n, qa, qb;
  if (mode == POND_STACK_ROTATION) {
    qa = qb = q_first + row;
  } else {
    lo = row * n_sub;
    hi = min(n, lo + n_sub);
    qa = key_at(m, lo).q;
    qb = key_at(m, hi - 1).q;
  }
  double s = 0.0;
  long long h = 0;
  for (long long q = qa; q <= qb; ++q) {
    const long long K = q * m.nbins + b;
    const long long a = first_at_or_after(m, lo, hi, K);
    const long long e = first_at_or_after(m, a, hi, K + 1);
    for (long long i = a; i < e; ++i) s = __dadd_rn(s, (double)__ldg(y + i));
    if (e > a) h += e - a;
  }
  S[cell] = s;
  H[cell] = h;
}

double rounded(double x) {
  volatile double v = x;
  return v;
}

// The host's evaluation of the same rotation, for the row count.
long long host_rotation(const PhaseModel& m, long long i) {
  const double tau = rounded((double)(m.g0 + i) * m.dt) - m.t_ref;
  double x = m.c[m.nc - 1];
  for (int k = m.nc - 2; k >= 0; --k) x = rounded(x * tau) + m.c[k];
  return (long long)std::floor(x);
}

int stack_args(int64_t n, int64_t g0, double dt_s, const double* coef, int32_t ncoef, double t_ref_s, int32_t nbins,
               int32_t mode, int64_t n_sub, PhaseModel* m, int64_t* rows, int64_t* first_rotation) {
  if (!rows || !first_rotation || (!coef && ncoef > 0))
    return pond::set_error(POND_E_ARG, "pond_fold_stack: null pointer");
  if (n < 0 || g0 < 0 || !(dt_s > 0) || !std::isfinite(dt_s) || !std::isfinite(t_ref_s) || ncoef < 1 ||
      ncoef > MAX_COEF || nbins < 1 || nbins > pond::MAX_NBINS ||
      !(mode == POND_STACK_ROTATION || (mode == POND_STACK_SUBINT && n_sub >= 1)))
    return pond::set_error(POND_E_ARG,
                           "pond_fold_stack: need n, g0 >= 0, dt > 0, 1..8 coefficients, nbins 1..4096, "
                           "mode ROTATION or SUBINT with n_sub >= 1");
  for (int k = 0; k < ncoef; ++k)
    if (!std::isfinite(coef[k])) return pond::set_error(POND_E_ARG, "pond_fold_stack: coefficient not finite");
  *m = PhaseModel{};
  for (int k = 0; k < ncoef; ++k) m->c[k] = coef[k];
  m->nc = ncoef;
  m->dt = dt_s;
  m->t_ref = t_ref_s;
  m->g0 = g0;
  m->nbins = nbins;
  if (n == 0) {
    *rows = 0;
    *first_rotation = 0;
    return POND_OK;
  }
  const long long q0 = host_rotation(*m, 0);
  *first_rotation = q0;
  *rows = mode == POND_STACK_ROTATION ? std::max(0ll, host_rotation(*m, n - 1) - q0 + 1) : (n + n_sub - 1) / n_sub;
  return POND_OK;
}

}  // namespace

extern "C" int pond_stack_rows(int64_t n, int64_t g0, double dt_s, const double* coef, int32_t ncoef, double t_ref_s,
                               int32_t nbins, int32_t mode, int64_t n_sub, int64_t* rows, int64_t* first_rotation) {
  PhaseModel m;
  return stack_args(n, g0, dt_s, coef, ncoef, t_ref_s, nbins, mode, n_sub, &m, rows, first_rotation);
}

extern "C" int pond_fold_stack(const float* d_series, int64_t n, int64_t g0, double dt_s, const double* coef,
                               int32_t ncoef, double t_ref_s, int32_t nbins, int32_t mode, int64_t n_sub,
                               double* d_sum, int64_t* d_hits, int64_t rows_cap, int64_t* rows,
                               int64_t* first_rotation, void* cuda_stream) {
  PhaseModel m;
  int rc = stack_args(n, g0, dt_s, coef, ncoef, t_ref_s, nbins, mode, n_sub, &m, rows, first_rotation);
  if (rc) return rc;
  if (*rows > rows_cap) {
    char msg[160];
    snprintf(msg, sizeof msg, "pond_fold_stack: %lld rows needed, room for %lld", (long long)*rows,
             (long long)rows_cap);
    return pond::set_error(POND_E_OVERRUN, msg);
  }
  if (n == 0) return POND_OK;
  if (!d_series || !d_sum || !d_hits) return pond::set_error(POND_E_ARG, "pond_fold_stack: null device pointer");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const int zero = 0;
  int back = 0;
  cudaError_t e = cudaMemcpyToSymbolAsync(g_backwards, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    const long long blocks = std::min<long long>((n + 255) / 256, 4096);
    k_stack_check<<<(unsigned)blocks, 256, 0, st>>>(m, n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyFromSymbolAsync(&back, g_backwards, sizeof(int), 0, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess)
    return pond::set_error(POND_E_CUDA, (std::string("pond_fold_stack: ") + cudaGetErrorString(e)).c_str());
  if (back) return pond::set_error(POND_E_ARG, "pond_fold_stack: the phase model runs backwards over the series");
  const long long cells = *rows * (long long)nbins;
  if (cells > 0) {
    k_stack_cells<<<(unsigned)((cells + CELL_THREADS - 1) / CELL_THREADS), CELL_THREADS, 0, st>>>(
        d_series, n, m, mode, n_sub, *first_rotation, *rows, d_sum, reinterpret_cast<long long*>(d_hits));
    e = cudaGetLastError();
    if (e != cudaSuccess)
      return pond::set_error(POND_E_CUDA, (std::string("pond_fold_stack: ") + cudaGetErrorString(e)).c_str());
  }
  return POND_OK;
}
