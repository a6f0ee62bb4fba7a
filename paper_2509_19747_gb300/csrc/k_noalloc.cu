// Allocation-free entry point: the float64-accurate Gaussian-kernel product
// w = (K + mu I) v with all of its scratch in a fixed, file-scope device
// array instead of a caller-provided workspace.
//
// Who needs it: code that cannot call cudaMalloc (or have anyone allocate on
// its behalf) at the point of use -- for example a plugin running inside a
// host framework that owns every byte of device memory through its own
// pool, a latency-critical serving loop that forbids allocator calls on its
// hot path, or a process whose device memory is already fully committed.
// Such callers still own their inputs and outputs; this entry point only
// removes the need for a workspace.
//
// Costs and rules of the static array:
//   * kNoAllocScratchBytes (32 MiB) of device memory are reserved on every
//     GPU that loads the library, for as long as the library stays loaded;
//   * every call shares it, so calls that overlap on the GPU (from several
//     streams or host threads at once) race and corrupt each other's
//     results; serialise them;
//   * every scratch element a call reads is written earlier in the same
//     call, so nothing has to start at zero and the last call's leftovers
//     are harmless;
//   * host code cannot use the array's name as a device address: every
//     call made outside stream capture looks the address up with
//     cudaGetSymbolAddress (current device) and remembers it per device; a
//     call made while its stream is being captured uses the remembered
//     address, so make the first call on each device before any capture
//     (that first call also loads the module into the device's context).
#include <cmath>
#include <mutex>

#include "rr_common.cuh"
#include "rr_krylov.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = 32u << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {nullptr};

// device address of the static scratch for the current device.  Outside
// stream capture the address is looked up on every call (cheap), so a
// context re-created after cudaDeviceReset is seen; during capture the
// address remembered from the last uncaptured call on this device is used.
rr_status scratch_address(int dev, bool capturing, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return RR_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_addr_mu);
  if (!capturing) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return RR_ERR_CUDA;
    }
    g_addr[dev] = p;
  }
  if (!g_addr[dev]) return RR_ERR_CUDA;     // first call on this device under capture
  *out = g_addr[dev];
  return RR_OK;
}

inline size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

extern "C" rr_status randrand_kernel_matvec_noalloc(const float* points, int64_t n, int32_t dim,
                                                    double bandwidth, double mu, const double* v,
                                                    double* w, int32_t m, int64_t ld,
                                                    void* stream) {
  using namespace rr;
  if (!points || !v || !w || n < 1 || n > (int64_t)INT32_MAX || dim < 1 || dim > 16 ||
      m < 1 || m > 8 || ld < n || !(bandwidth > 0.0) || !std::isfinite(bandwidth) ||
      !(mu >= 0.0) || !std::isfinite(mu))
    return RR_ERR_INVALID_ARG;
  int mp = 1;
  while (mp < m) mp <<= 1;
  // layout: V and W interleaved (n x mp doubles each), |p|^2 (n float2), partials
  const size_t vec = a256((size_t)n * mp * sizeof(double));
  const size_t pnb = a256((size_t)n * sizeof(float2));
  const size_t part1 = (size_t)n * mp * sizeof(double);
  const size_t fixed = 2 * vec + pnb;
  if (fixed + part1 > kNoAllocScratchBytes) return RR_ERR_WORKSPACE;  // n, m beyond the array
  int nsplit = kernel_mv_nsplit(n);
  while (nsplit > 1 && fixed + (size_t)nsplit * part1 > kNoAllocScratchBytes) --nsplit;
  // an error left pending by earlier, unrelated work is not ours to clear or
  // to report as a failed launch of this call
  if (cudaPeekAtLastError() != cudaSuccess) return RR_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = -1, sdev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return RR_ERR_CUDA;
  if (cudaStreamGetDevice(st, &sdev) != cudaSuccess) {
    cudaGetLastError();
    return RR_ERR_INVALID_ARG;                // not a stream handle of this process
  }
  if (sdev != dev) return RR_ERR_INVALID_ARG;  // the stream belongs to another device
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
    cudaGetLastError();
    return RR_ERR_CUDA;
  }
  void* base = nullptr;
  RR_TRY(scratch_address(dev, cap != cudaStreamCaptureStatusNone, &base));
  unsigned char* b = (unsigned char*)base;
  double* Vi = (double*)b;
  double* Wi = (double*)(b + vec);
  float2* pn = (float2*)(b + 2 * vec);
  double* part = (double*)(b + fixed);
  gather_cols(v, ld, m, n, mp, Vi, st);
  if (cudaGetLastError() != cudaSuccess) return RR_ERR_CUDA;
  kernel_mv_df_raw(points, n, dim, bandwidth, mu, Vi, Wi, mp, pn, part, nsplit, st);
  if (cudaGetLastError() != cudaSuccess) return RR_ERR_CUDA;
  scatter_cols(Wi, n, mp, m, w, ld, st);
  if (cudaGetLastError() != cudaSuccess) return RR_ERR_CUDA;
  return RR_OK;
}
