// diag.cu -- diagnostic entry points: each applies one device primitive of the
// sampler to arrays, so that tests can compare it element by element with an
// independent implementation (cuRAND's Philox, the CPU oracle's skip).
#include <cuda_runtime.h>
#include <curand_kernel.h>

#include "cl_internal.cuh"
#include "clmath.cuh"
#include "philox.cuh"

namespace cl {

__global__ void diag_philox_kernel(const uint32_t* __restrict__ ctr, long long n, uint32_t k0, uint32_t k1,
                                   uint32_t* __restrict__ out) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  u32x4 c{ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]};
  u32x4 r = philox4x32_10(c, k0, k1);
  out[4 * i] = r.x;
  out[4 * i + 1] = r.y;
  out[4 * i + 2] = r.z;
  out[4 * i + 3] = r.w;
}

// cuRAND's device Philox4x32-10, called (not copied) as an independent reference.
__global__ void diag_philox_curand_kernel(const uint32_t* __restrict__ ctr, long long n, uint32_t k0, uint32_t k1,
                                          uint32_t* __restrict__ out) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
  uint4 r = curand_Philox4x32_10(c, make_uint2(k0, k1));
  out[4 * i] = r.x;
  out[4 * i + 1] = r.y;
  out[4 * i + 2] = r.z;
  out[4 * i + 3] = r.w;
}

__global__ void diag_neglog_kernel(const unsigned long long* __restrict__ A, const unsigned long long* __restrict__ B,
                                   long long n, float* __restrict__ oft, double* __restrict__ odd) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (!(A[i] >= 1 && A[i] < B[i] && B[i] <= (1ull << 55))) {  // outside the routine's domain
    oft[2 * i] = oft[2 * i + 1] = __int_as_float(0x7fc00000);
    odd[2 * i] = odd[2 * i + 1] = __longlong_as_double(0x7ff8000000000000ll);
    return;
  }
  // the float-float forms the sampler uses: -ln r (B = 2^53) or -ln(1 - Q/S)
  // -ln r as the sampler forms it from the Philox word pair (odd A: A = 2k + 1)
  const unsigned long long k = A[i] >> 1;
  ff f = B[i] == (1ull << 53)
             ? ((A[i] & 1ull) ? ff_neglog_r53_w((unsigned)((k & 0xFFFFFull) << 12), (unsigned)(k >> 20))
                              : ff_neglog_r53(A[i]))
             : ff_neglog1m(B[i] - A[i], B[i], lp_const(B[i]));
  dd d = dd_neglog_ratio(A[i], B[i]);
  oft[2 * i] = f.hi;
  oft[2 * i + 1] = f.lo;
  odd[2 * i] = d.hi;
  odd[2 * i + 1] = d.lo;
}

// The same two-tier decision the sampler makes for one skip.
__global__ void diag_skip_kernel(const unsigned long long* __restrict__ a, const unsigned long long* __restrict__ Q,
                                 const unsigned long long* __restrict__ S, const long long* __restrict__ R,
                                 long long n, long long* __restrict__ delta, int* __restrict__ tier) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (!(Q[i] > 0 && Q[i] < S[i] && S[i] < (1ull << 53) && a[i] < (1ull << 52) && R[i] >= 1)) {
    delta[i] = -2;  // outside the domain of the skip
    tier[i] = -1;
    return;
  }
  unsigned long long Ar = 2ull * a[i] + 1ull;
  ff Lr = ff_neglog_r53(Ar);
  ff Lp = ff_neglog1m(Q[i], S[i], lp_const(S[i]));
  // the sampler's decision (32-bit below 2^31, as in sample_kernel)
  long long d = R[i] < (1ll << 31) ? (long long)floor_decide_ff32(ff_div(Lr, Lp), (int)R[i])
                                   : floor_decide_ff(ff_div(Lr, Lp), R[i]);
  int tr = 0;
  if (d == SKIP_UNDECIDED) {
    bool tie;
    d = skip_fallback_dd(Ar, S[i] - Q[i], S[i], R[i], &tie);
    tr = tie ? 2 : 1;
  }
  delta[i] = d;
  tier[i] = tr;
}

// -ln(1 - Q/S) for doubles 0 < Q < S as the sampler evaluates it for double weights
// (float-float from the doubles).
__global__ void diag_neglog1m_f64_kernel(const double* __restrict__ Q, const double* __restrict__ S, long long n,
                                         float* __restrict__ out) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (!(Q[i] > 0.0 && Q[i] < S[i] && S[i] < 1e300)) {
    out[2 * i] = out[2 * i + 1] = __int_as_float(0x7fc00000);
    return;
  }
  const ff r = ff_neglog1m_d(Q[i], S[i], lp_const_d_dev(S[i]));
  out[2 * i] = r.hi;
  out[2 * i + 1] = r.lo;
}

// Philox4x32-10 throughput: every thread runs `iters` blocks, each keyed by
// the previous block's output (no work can be hoisted or skipped), and folds
// them into one word.  The rate bounds the sampler from above: one block per
// loop iteration of Algorithm 1.
__global__ void __launch_bounds__(256) diag_philox_rate_kernel(long long iters, uint32_t k0, uint32_t k1,
                                                                unsigned long long* __restrict__ sink) {
  const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
  u32x4 c{tid, 0u, tid * 2654435761u, 0u};
  uint32_t acc = 0;
  for (long long i = 0; i < iters; ++i) {
    const u32x4 r = philox4x32_10(c, k0, k1);
    acc ^= r.x ^ r.y ^ r.z ^ r.w;
    c = u32x4{(uint32_t)i + 1u, r.y, c.z, r.w};
  }
  if (acc == 0x9E3779B9u) atomicAdd(sink, 1ull);  // keeps the chain live
}

}  // namespace cl

using namespace cl;

extern "C" cl_status cl_diag_philox_rate(int64_t iters, uint64_t seed, uint64_t* d_sink, double* blocks_per_s,
                                         cl_stream_t stream) {
  if (iters <= 0 || !d_sink || !blocks_per_s) return CL_ERR_INVALID_ARG;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CL_ERR_CUDA;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, diag_philox_rate_kernel, 256, 0);
  const int grid = sms * (per_sm > 0 ? per_sm : 1);
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return CL_ERR_CUDA;
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return CL_ERR_CUDA;
  }
  diag_philox_rate_kernel<<<grid, 256, 0, s>>>(iters / 8 > 0 ? iters / 8 : 1, (uint32_t)seed, (uint32_t)(seed >> 32),
                                               (unsigned long long*)d_sink);  // warm-up
  cudaEventRecord(a, s);
  diag_philox_rate_kernel<<<grid, 256, 0, s>>>(iters, (uint32_t)seed, (uint32_t)(seed >> 32),
                                               (unsigned long long*)d_sink);
  cudaEventRecord(b, s);
  cl_status st = cudaEventSynchronize(b) == cudaSuccess ? CL_OK : CL_ERR_CUDA;
  float ms = 0;
  if (st == CL_OK && cudaEventElapsedTime(&ms, a, b) != cudaSuccess) st = CL_ERR_CUDA;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (st == CL_OK) *blocks_per_s = (double)grid * 256.0 * (double)iters / (ms * 1e-3);
  return st;
}

static cl_status diag_done() { return cudaGetLastError() == cudaSuccess ? CL_OK : CL_ERR_CUDA; }

extern "C" cl_status cl_diag_philox(const uint32_t* d_ctr, int64_t count, uint64_t seed, uint32_t* d_out,
                                    cl_stream_t stream) {
  if (count < 0 || (count > 0 && (!d_ctr || !d_out))) return CL_ERR_INVALID_ARG;
  if (count == 0) return CL_OK;
  diag_philox_kernel<<<(unsigned)((count + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      d_ctr, count, (uint32_t)seed, (uint32_t)(seed >> 32), d_out);
  return diag_done();
}

extern "C" cl_status cl_diag_philox_curand(const uint32_t* d_ctr, int64_t count, uint64_t seed, uint32_t* d_out,
                                           cl_stream_t stream) {
  if (count < 0 || (count > 0 && (!d_ctr || !d_out))) return CL_ERR_INVALID_ARG;
  if (count == 0) return CL_OK;
  diag_philox_curand_kernel<<<(unsigned)((count + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      d_ctr, count, (uint32_t)seed, (uint32_t)(seed >> 32), d_out);
  return diag_done();
}

extern "C" cl_status cl_diag_neglog(const uint64_t* d_A, const uint64_t* d_B, int64_t count, float* d_ff, double* d_dd,
                                    cl_stream_t stream) {
  if (count < 0 || (count > 0 && (!d_A || !d_B || !d_ff || !d_dd))) return CL_ERR_INVALID_ARG;
  if (count == 0) return CL_OK;
  diag_neglog_kernel<<<(unsigned)((count + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      (const unsigned long long*)d_A, (const unsigned long long*)d_B, count, d_ff, d_dd);
  return diag_done();
}

extern "C" cl_status cl_diag_skip(const uint64_t* d_a, const uint64_t* d_Q, const uint64_t* d_S, const int64_t* d_R,
                                  int64_t count, int64_t* d_delta, int32_t* d_tier, cl_stream_t stream) {
  if (count < 0 || (count > 0 && (!d_a || !d_Q || !d_S || !d_R || !d_delta || !d_tier))) return CL_ERR_INVALID_ARG;
  if (count == 0) return CL_OK;
  diag_skip_kernel<<<(unsigned)((count + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      (const unsigned long long*)d_a, (const unsigned long long*)d_Q, (const unsigned long long*)d_S,
      (const long long*)d_R, count, (long long*)d_delta, d_tier);
  return diag_done();
}

extern "C" cl_status cl_diag_neglog1m_f64(const double* d_Q, const double* d_S, int64_t count, float* d_ff,
                                          cl_stream_t stream) {
  if (count < 0 || (count > 0 && (!d_Q || !d_S || !d_ff))) return CL_ERR_INVALID_ARG;
  if (count == 0) return CL_OK;
  diag_neglog1m_f64_kernel<<<(unsigned)((count + 255) / 256), 256, 0, (cudaStream_t)stream>>>(d_Q, d_S, count, d_ff);
  return diag_done();
}
