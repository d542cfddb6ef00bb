// pond_fold_noalloc: the fold with its scratch memory in a fixed device array.
//
// The engine's fold keeps per-CTA partial histograms in buffers that
// pond_plan allocates.  Some callers cannot allocate device memory at all:
// a real-time acquisition thread that must never stall (cudaMalloc and
// cudaFree may synchronise the whole device and take unbounded time), or a
// host application whose own memory manager owns every device allocation and
// forbids libraries from making their own.  This entry point serves them: it
// allocates nothing.  Its scratch is the file-scope array below, reserved in
// the memory of every GPU that loads the library and held until the process
// exits.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/pond.h"
#include "pond_internal.h"

namespace {

constexpr int kMaxDevices = 64;
constexpr size_t kParts = (size_t)pond::MAX_FOLD_PARTS;
// Per-CTA fold partials for up to POND_NOALLOC_MAX_NBINS bins: FP64 sums, then int32 hits.
constexpr size_t kSumBytes = kParts * POND_NOALLOC_MAX_NBINS * sizeof(double);
constexpr size_t kHitBytes = kParts * POND_NOALLOC_MAX_NBINS * sizeof(int);
constexpr size_t kScratchBytes = kSumBytes + kHitBytes;   // 3.6 MiB

static __device__ __align__(256) unsigned char g_fold_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char* g_scratch_addr[kMaxDevices];   // device address per device, once looked up

// Set-up, once per device with that device current: the device address of the
// scratch array (in host code the array's name is only a host-side stand-in,
// so the kernels get this address) and the fold kernel's shared-memory limit.
int scratch_for(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = pond::set_kernel_attributes();
    if (e != cudaSuccess)
      return pond::set_error(POND_E_CUDA, (std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e)).c_str());
    e = cudaGetSymbolAddress(&p, g_fold_scratch);
    if (e != cudaSuccess)
      return pond::set_error(POND_E_CUDA, (std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_addr[dev];
  return POND_OK;
}

}  // namespace

extern "C" int pond_fold_noalloc(const float* d_power, int64_t n, int64_t g0, double dtc_s, double period_s,
                                 int32_t nbins, double* d_sum, int64_t* d_hits, void* cuda_stream) {
  if (n < 0 || g0 < 0 || nbins < 1 || !(dtc_s > 0) || !(period_s > 0))
    return pond::set_error(POND_E_ARG, "pond_fold_noalloc: need n >= 0, g0 >= 0, nbins >= 1, dtc > 0, period > 0");
  if (nbins > POND_NOALLOC_MAX_NBINS) {
    char msg[128];
    snprintf(msg, sizeof msg, "pond_fold_noalloc: nbins %d exceeds the limit of %d", nbins, POND_NOALLOC_MAX_NBINS);
    return pond::set_error(POND_E_ARG, msg);
  }
  // per-CTA hits are int32 over ceil(n / kParts) samples (rounded up to 128)
  static_assert(POND_NOALLOC_MAX_SAMPLES / kParts + 128 < (1LL << 31), "per-CTA hit count must fit in int32");
  if (n > POND_NOALLOC_MAX_SAMPLES)
    return pond::set_error(POND_E_ARG, "pond_fold_noalloc: n exceeds the per-call limit POND_NOALLOC_MAX_SAMPLES");
  if (n == 0) return POND_OK;
  if (!d_power || !d_sum || !d_hits) return pond::set_error(POND_E_ARG, "pond_fold_noalloc: null pointer");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return pond::set_error(POND_E_CUDA, "pond_fold_noalloc: no usable current device");
  unsigned char* base = nullptr;
  int rc = scratch_for(dev, &base);
  if (rc) return rc;
  double* psum = reinterpret_cast<double*>(base);
  int* phits = reinterpret_cast<int*>(base + kSumBytes);
  const double inc = dtc_s / period_s;
  e = pond::launch_fold(d_power, n, g0, inc, nbins, psum, phits, d_sum, reinterpret_cast<long long*>(d_hits),
                        static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess)
    return pond::set_error(POND_E_CUDA, (std::string("pond_fold_noalloc: ") + cudaGetErrorString(e)).c_str());
  return POND_OK;
}
