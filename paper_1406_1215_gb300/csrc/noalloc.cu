// noalloc.cu -- cl_scan_noalloc: the count -> offset exclusive scan of cl_scan
// for callers that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not an option -- inside a
// host callback or a real-time loop where cudaMalloc's implicit device
// synchronisation is not acceptable, inside a plug-in whose host framework
// owns every device allocation and hands out no scratch, or under a fixed
// memory budget where a fresh allocation could fail.  Such a caller still
// provides the input counts and the output offsets; the scratch the scan
// needs (one int64 partial sum per 2048-count tile) comes from the array
// below, which lives in the library image of every GPU that loads it until
// the process exits (1 MiB + 8 bytes per device).
//
// Host code must not pass `g_noalloc_partials` itself to a kernel: on the
// host that name is only a stand-in for the device symbol.  Each call looks up
// the array's device address with cudaGetSymbolAddress on the current device
// and passes that address to the kernels.  The lookup is repeated on every
// call rather than cached: after a cudaDeviceReset the library's device code
// is loaded again and the array may sit at another address, so a cached
// pointer could point into freed memory.  Once the device code is loaded the
// lookup is cheap next to a kernel launch.
#include <cuda_runtime.h>

#include "cl_internal.cuh"

namespace {

constexpr long long NOALLOC_MAX_COUNTS = 1ll << 28;  // 268,435,456 counts
constexpr long long NOALLOC_MAX_TILES = NOALLOC_MAX_COUNTS / cl::SCAN_TILE_HOST;

// The shared scratch: tile partials of the three-phase scan.
static __device__ __align__(256) long long g_noalloc_partials[NOALLOC_MAX_TILES + 1];

// Device address of the scratch on the current device.  The first call on a
// device also loads the library's device code there (lazy module loading).
cl_status noalloc_scratch(long long** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) return CL_ERR_CUDA;
  *out = (long long*)p;
  return CL_OK;
}

}  // namespace

extern "C" cl_status cl_scan_noalloc(const int32_t* d_counts, int64_t n, int64_t* d_offsets, cl_stream_t stream) {
  if (n < 0 || !d_offsets || (n > 0 && !d_counts)) return CL_ERR_INVALID_ARG;
  if (n > NOALLOC_MAX_COUNTS) return CL_ERR_RANGE;
  long long* part = nullptr;
  cl_status st = noalloc_scratch(&part);
  if (st != CL_OK) return st;
  // every partial the scan reads is written first by its reduce phase: nothing to clear
  cl::launch_count_scan(d_counts, n, (long long*)d_offsets, part, (cudaStream_t)stream);
  return cudaGetLastError() == cudaSuccess ? CL_OK : CL_ERR_CUDA;
}
