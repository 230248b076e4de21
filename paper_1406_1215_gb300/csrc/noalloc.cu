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
// host that name is only a stand-in for the device symbol.  Its device
// address is fetched once per device with cudaGetSymbolAddress while that
// device is current, and that address is what the kernels receive.
#include <cuda_runtime.h>

#include <mutex>

#include "cl_internal.cuh"

namespace {

constexpr long long NOALLOC_MAX_COUNTS = 1ll << 28;  // 268,435,456 counts
constexpr long long NOALLOC_MAX_TILES = NOALLOC_MAX_COUNTS / cl::SCAN_TILE_HOST;

// The shared scratch: tile partials of the three-phase scan.
static __device__ __align__(256) long long g_noalloc_partials[NOALLOC_MAX_TILES + 1];

constexpr int MAX_DEVICES = 128;
std::mutex g_mu;
long long* g_dev_ptr[MAX_DEVICES] = {};

// Device address of the scratch on the current device (set up on first use).
cl_status noalloc_scratch(long long** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return CL_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) return CL_ERR_CUDA;
    g_dev_ptr[dev] = (long long*)p;
  }
  *out = g_dev_ptr[dev];
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
