// Residual norms for callers that cannot allocate device memory.
//
// chase_residuals needs a context, and chase_create allocates the context's
// workspace with cudaMalloc. Some callers cannot do that: code that runs inside
// another framework's memory budget (a caching allocator or pool that owns the
// device memory and must not be bypassed), and code that must not trigger the
// device-wide synchronisation cudaMalloc/cudaFree can imply. This entry point
// computes the same residual norms with the same kernels but takes its scratch
// (the per-tile partial sums) from a fixed array in the library's own device
// memory, so it allocates nothing.
#include <cstdio>
#include <mutex>

#include "common.cuh"

namespace chase {
namespace {

// Scratch of the residual kernel: one partial sum per 64-row tile and column,
// i.e. ceil(N / 64) * ncols doubles. 4 MiB, held on every GPU that loads the
// library until the process exits.
constexpr size_t kScratchDoubles = (size_t)4 << 17;  // 524288 doubles = 4 MiB
static __device__ __align__(256) double g_resid_scratch[kScratchDoubles];

std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_resid_scratch on the current device. In host code the
// symbol is only a host-side stand-in, so its device address is looked up once
// per device, with that device current, and cached. The cache assumes the
// device's primary context (the one the CUDA runtime and torch use) for the
// life of the process: after cudaDeviceReset the module is loaded again at
// another address and the cached pointer would be stale.
int scratch_address(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CHASE_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_resid_scratch);
    if (e != cudaSuccess || !p) {
      fprintf(stderr, "[chase] cudaGetSymbolAddress(residual scratch) failed: %s\n",
              cudaGetErrorString(e));
      return CHASE_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return CHASE_OK;
}

}  // namespace
}  // namespace chase

using namespace chase;

extern "C" int chase_residuals_noalloc(const chase_c128* A, int64_t lda, const chase_c128* V,
                                       int64_t ldv, const double* ritz, int64_t N, int64_t ncols,
                                       double* resid, void* stream) {
  if (!A || !V || !ritz || !resid || N < 1 || ncols < 0 || lda < N || ldv < N)
    return CHASE_ERR_INVALID_ARG;
  if (ncols == 0) return CHASE_OK;
  const int64_t tiles = zgemm_row_tiles(N);
  if ((size_t)tiles * (size_t)ncols > kScratchDoubles) {
    fprintf(stderr,
            "[chase] chase_residuals_noalloc: ceil(N/64) * ncols = %lld exceeds the fixed "
            "scratch of %zu doubles (N = %lld, ncols = %lld)\n",
            (long long)(tiles * ncols), kScratchDoubles, (long long)N, (long long)ncols);
    return CHASE_ERR_INVALID_ARG;
  }
  double* scratch = nullptr;
  const int rc = scratch_address(&scratch);
  if (rc != CHASE_OK) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  Epilogue ep{};
  ep.mode = EPI_RESID;
  ep.X = reinterpret_cast<const double2*>(V);
  ep.ldx = ldv;
  ep.theta = ritz;
  ep.partial = scratch;  // every partial the reduction reads is written first below
  if (zgemm_nn(s, N, ncols, N, reinterpret_cast<const double2*>(A), lda,
               reinterpret_cast<const double2*>(V), ldv, ep) != cudaSuccess)
    return CHASE_ERR_CUDA;
  if (resid_reduce(s, scratch, tiles, ncols, resid) != cudaSuccess) return CHASE_ERR_CUDA;
  return CHASE_OK;
}
