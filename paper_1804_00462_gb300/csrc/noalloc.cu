// sorsvd_run_noalloc: sorsvd_run with its scratch space in a fixed device
// array owned by the library, for callers that cannot allocate device memory
// at call time - for example code embedded in a host application that hands
// out all device memory from its own fixed pool and forbids other
// allocations, or latency-critical loops where cudaMalloc (which may
// synchronise the device) is not acceptable.  The caller still provides A
// and the outputs U, S, V.
//
// The scratch array is a file-scope __device__ array of kNoallocBytes; every
// GPU that loads this library holds it until the process exits.  Its device
// address is looked up once per device (cudaGetSymbolAddress, with that
// device current) by the first call made on that device, so that first call
// should come before any stream capture.  All calls share the one array and
// it keeps the last call's contents: sorsvd_run clears the status word it
// starts from and writes every other buffer before reading it, and calls
// that overlap on the GPU race on the array.  The cached address belongs to
// the device's primary context: do not use this entry point after a
// cudaDeviceReset or from another context in the same process.
//
// sorsvd_noalloc_get_status reads the device status word at the start of
// the array (Cholesky breakdown, Jacobi not converged, bounded-wait
// timeout), the counterpart of sorsvd_get_status for a caller workspace.
#include "internal.cuh"

#include <mutex>

namespace sorsvd {
namespace {

constexpr size_t kNoallocBytes = (size_t)SORSVD_NOALLOC_MAX_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};

// device address of the scratch array on the current device (set up once)
int noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SORSVD_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return SORSVD_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SORSVD_ERR_CUDA;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return SORSVD_OK;
}

}  // namespace
}  // namespace sorsvd

extern "C" int sorsvd_run_noalloc(const void* A, int64_t m, int64_t n, int64_t lda, int k, int p, int q,
                                  uint64_t seed, int dtype, unsigned flags, void* U, int64_t ldu, void* S, void* V,
                                  int64_t ldv, void* stream) {
  const size_t need = sorsvd_workspace_size(m, n, k, p, dtype, flags);
  if (need == 0 || need > sorsvd::kNoallocBytes) {
    // sorsvd_run checks the arguments before it touches a workspace or the
    // GPU: an invalid argument keeps its own code, a valid problem that does
    // not fit the scratch array is reported as beyond the documented limit
    const int r = sorsvd_run(A, m, n, lda, k, p, q, seed, dtype, flags, U, ldu, S, V, ldv, nullptr, 0, stream);
    return r == SORSVD_ERR_WORKSPACE ? SORSVD_ERR_UNSUPPORTED : r;
  }
  void* ws = nullptr;
  if (int r = sorsvd::noalloc_scratch(&ws)) return r;
  return sorsvd_run(A, m, n, lda, k, p, q, seed, dtype, flags, U, ldu, S, V, ldv, ws, sorsvd::kNoallocBytes,
                    stream);
}

extern "C" int sorsvd_noalloc_get_status(int* device_status, int* info, void* stream) {
  void* ws = nullptr;
  if (int r = sorsvd::noalloc_scratch(&ws)) return r;
  return sorsvd_get_status(ws, device_status, info, stream);
}
