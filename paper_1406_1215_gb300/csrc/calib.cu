// calib.cu -- capped expected degrees, their adjoint, and weight calibration.
//
// Section 3: with no capped pair the expected degree of node i is
// w_i - w_i^2/S.  With the cap min(1, .) of Algorithm 1 it is
//   E_u = sum_{v != u} min(1, w_u w_v / S),   S = sum_k w_k.
// For w sorted non-increasing the capped partners of u (fl(w_u w_v) >= S) are
// a prefix [0, t_u), so with R_k = sum_{v >= k} w_v
//   E_u = (t_u - [u < t_u]) + (w_u / S) A_u,   A_u = R_{t_u} - [u >= t_u] w_u.
// The gradient of L = sum_u gE_u E_u (S depends on w):
//   dL/dw_k = [gE_k A_k + B_k - K] / S,  B_k = G_{t_k} - [k >= t_k] gE_k w_k,
//   G_j = sum_{u >= j} gE_u w_u,  K = sum_u gE_u (w_u / S) A_u.
// Sums are carried in double-double (Dekker's sum); the per-node terms are
// rounded once to double.  R and G are needed only at the thresholds t_u <= t_0,
// so they come from one reduction over all nodes and a prefix over the first t_0.  FP64 is slow on this GPU (1/75 of
// FP32) and sets these kernels' time, so they spend as few FP64 operations as
// they can: division by S is a product with a double-double 1/S formed once per
// call, and t_u is found by a galloping search that ends at once for the nodes
// with no capped partner (almost all of them).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "cl_internal.cuh"
#include "clmath.cuh"

namespace cl {
namespace {

constexpr int CT = 256;            // threads per block
constexpr int CI = 16;             // items per thread in a scan tile (16 against 8: 0.114 against 0.125 s per calibration)
constexpr int CTILE = CT * CI;

__device__ __forceinline__ dd dd_shfl_up(dd v, int o) {
  return dd{__shfl_up_sync(FULL_MASK, v.hi, o), __shfl_up_sync(FULL_MASK, v.lo, o)};
}
__device__ __forceinline__ dd dd_shfl_xor(dd v, int o) {
  return dd{__shfl_xor_sync(FULL_MASK, v.hi, o), __shfl_xor_sync(FULL_MASK, v.lo, o)};
}

__device__ __forceinline__ dd dd_block_reduce(dd v) {
  __shared__ double rh[32], rl[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = dd_add_dekker(v, dd_shfl_xor(v, o));
  if (lane == 0) {
    rh[wid] = v.hi;
    rl[wid] = v.lo;
  }
  __syncthreads();
  dd t{0.0, 0.0};
  if (wid == 0) {
    if (lane < nw) t = dd{rh[lane], rl[lane]};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = dd_add_dekker(t, dd_shfl_xor(t, o));
  }
  __syncthreads();
  return t;  // valid in warp 0
}

// exclusive block scan of dd values (one per thread); total in *tot
__device__ __forceinline__ dd dd_block_excl(dd v, dd* tot) {
  __shared__ double sh[32], sl[32];
  __shared__ double th, tl;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  dd inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    dd y = dd_shfl_up(inc, o);
    if (lane >= o) inc = dd_add_dekker(inc, y);
  }
  if (lane == 31) {
    sh[wid] = inc.hi;
    sl[wid] = inc.lo;
  }
  __syncthreads();
  if (wid == 0) {
    dd t = lane < nw ? dd{sh[lane], sl[lane]} : dd{0.0, 0.0};
    dd ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      dd y = dd_shfl_up(ti, o);
      if (lane >= o) ti = dd_add_dekker(ti, y);
    }
    dd ex = dd_add_dekker(ti, dd{-t.hi, -t.lo});
    if (lane < nw) {
      sh[lane] = ex.hi;
      sl[lane] = ex.lo;
    }
    if (lane == nw - 1) {
      th = ti.hi;
      tl = ti.lo;
    }
  }
  __syncthreads();
  dd res = dd_add_dekker(dd{sh[wid], sl[wid]}, dd_add_dekker(inc, dd{-v.hi, -v.lo}));
  *tot = dd{th, tl};
  __syncthreads();
  return res;
}

// x_i of a tail sum: w_i, or the exact product gE_i w_i
__device__ __forceinline__ dd term(const double* a, const double* b, long long i) {
  return b ? dd_two_prod(a[i], b[i]) : dd{a[i], 0.0};
}

// Exclusive scan, in place, of nt double-double tile sums (one block, 1024 at a time).
__global__ void suffix_partials_kernel(double* __restrict__ part, long long nt, const long long* __restrict__ mp) {
  if (mp) {  // only the tiles up to the one holding index m are read afterwards
    const long long tm = *mp / CTILE + 1;
    nt = tm < nt ? tm : nt;
  }
  __shared__ double ch, cl_;
  if (threadIdx.x == 0) ch = cl_ = 0.0;
  __syncthreads();
  for (long long base = 0; base < nt; base += blockDim.x) {
    long long i = base + threadIdx.x;
    dd v = i < nt ? dd{part[2 * i], part[2 * i + 1]} : dd{0.0, 0.0};
    dd carry{ch, cl_};
    dd tot;
    dd ex = dd_add_dekker(dd_block_excl(v, &tot), carry);
    if (i < nt) {
      part[2 * i] = ex.hi;
      part[2 * i + 1] = ex.lo;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      dd c = dd_add_dekker(carry, tot);
      ch = c.hi;
      cl_ = c.lo;
    }
    __syncthreads();
  }
}

// Tail sums X_k = sum_{i >= k} x_i are needed only at the thresholds t_u, and
// t_u <= t_0 for every u (w_0 is the largest weight), so they are formed as
// X_k = total - sum_{i < k} x_i for k <= m = t_0 alone: one reduction over all n
// values and a prefix over the first m, instead of a scan over all n.  The
// subtraction is the accurate double-double sum (the two terms may nearly cancel).
// Tile sums of x_i over [0, n), or over [0, min(*mp, n)) when mp is given (tiles
// past it write zero).
__global__ void __launch_bounds__(CT) tile_sum_kernel(const double* __restrict__ a, const double* __restrict__ b,
                                                      long long n, const long long* __restrict__ mp,
                                                      double* __restrict__ part) {
  const long long m = mp ? (*mp < n ? *mp : n) : n;
  const long long i0 = blockIdx.x * (long long)CTILE;
  dd acc{0.0, 0.0};
  if (i0 < m) {
    for (int k = 0; k < CI; ++k) {
      const long long i = i0 + (long long)k * CT + threadIdx.x;
      if (i < m) acc = dd_add_dekker(acc, term(a, b, i));
    }
  }
  const dd t = dd_block_reduce(acc);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = t.hi;
    part[2 * blockIdx.x + 1] = t.lo;
  }
}

// The double-double total of nt tile sums (one block) into tot[0..1].
__global__ void total_kernel(const double* __restrict__ part, long long nt, double* __restrict__ tot) {
  dd acc{0.0, 0.0};
  for (long long i = threadIdx.x; i < nt; i += blockDim.x) acc = dd_add_dekker(acc, dd{part[2 * i], part[2 * i + 1]});
  const dd t = dd_block_reduce(acc);
  if (threadIdx.x == 0) {
    tot[0] = t.hi;
    tot[1] = t.lo;
  }
}

// X_k = tot - sum_{i < k} x_i for k = 0 .. m (part: the exclusive prefix of the tile sums).
__global__ void __launch_bounds__(CT) tail_scan_kernel(const double* __restrict__ a, const double* __restrict__ b,
                                                       long long n, const long long* __restrict__ mp,
                                                       const double* __restrict__ part, const double* __restrict__ tot,
                                                       double* __restrict__ X) {
  const long long m = *mp < n ? *mp : n;
  if (blockIdx.x * (long long)CTILE > m) return;  // the whole block: no index <= m here
  const long long k0 = blockIdx.x * (long long)CTILE + (long long)threadIdx.x * CI;
  dd v[CI];
  dd loc{0.0, 0.0};
#pragma unroll
  for (int k = 0; k < CI; ++k) {
    v[k] = (k0 + k < m) ? term(a, b, k0 + k) : dd{0.0, 0.0};
    loc = dd_add_dekker(loc, v[k]);
  }
  dd t;
  dd run = dd_add_dekker(dd_block_excl(loc, &t), dd{part[2 * blockIdx.x], part[2 * blockIdx.x + 1]});
  const dd T{tot[0], tot[1]};
#pragma unroll
  for (int k = 0; k < CI; ++k) {
    const long long idx = k0 + k;
    if (idx <= m) {
      const dd x = idx == n ? dd{0.0, 0.0} : dd_add(T, dd{-run.hi, -run.lo});
      X[2 * idx] = x.hi;
      X[2 * idx + 1] = x.lo;
    }
    run = dd_add_dekker(run, v[k]);
  }
}

// t_u = #{v : fl(w_u w_v) >= S}: the capped partners form a prefix of the sorted w.
// Galloping from v = 0 (w_0 is the largest weight, so fl(w_u w_0) < S means no
// capped partner), then bisection: about 2 log2(t_u) products.
__device__ __forceinline__ long long cap_threshold(const double* w, long long n, double wu, double S) {
  if (!(wu * w[0] >= S)) return 0;
  long long k = 1;  // w[k / 2] is a capped partner
  while (k < n && wu * w[k] >= S) k *= 2;
  long long lo = k / 2 + 1, hi = k < n ? k : n;  // the first non-partner lies in [lo, hi]
  while (lo < hi) {
    long long mid = (lo + hi) >> 1;
    if (wu * w[mid] >= S)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// m = t_0, the largest threshold (the heaviest node's)
__global__ void t0_kernel(const double* __restrict__ w, long long n, const double* __restrict__ sc,
                          long long* __restrict__ t0) {
  *t0 = cap_threshold(w, n, w[0], sc[0]);
}

// forward: E_u, and per node t_u and A_u / S (the uncapped part's derivative dE_u/dw_u at fixed S)
__global__ void __launch_bounds__(CT) expdeg_kernel(const double* __restrict__ w, long long n,
                                                    const double* __restrict__ sc,
                                                    const double* __restrict__ R, double* __restrict__ E,
                                                    long long* __restrict__ tcap, double* __restrict__ Ahi,
                                                    double* __restrict__ Alo) {
  long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (u >= n) return;
  const double S = sc[0];
  const dd iS{sc[1], sc[2]};
  double wu = w[u];
  long long t = cap_threshold(w, n, wu, S);
  dd A{R[2 * t], R[2 * t + 1]};
  if (u >= t) A = dd_add_dekker(A, dd{-wu, 0.0});
  dd part = dd_mul(dd_mul_d(A, wu), iS);  // (w_u / S) A_u
  double capped = (double)(t - (u < t ? 1 : 0));
  dd e = dd_add_dekker(part, dd{capped, 0.0});
  if (E) E[u] = e.hi + e.lo;
  if (tcap) tcap[u] = t;
  if (Ahi) {
    Ahi[u] = A.hi;
    Alo[u] = A.lo;
  }
}

// K = sum_u gE_u (w_u / S) A_u (block partial sums, dd)
// tile sums of gE_u w_u A_u (for K) and of gE_u w_u (the total of G), in one pass
__global__ void __launch_bounds__(CT) adj_K_kernel(const double* __restrict__ w, const double* __restrict__ gE,
                                                   long long n, const double* __restrict__ Ahi,
                                                   const double* __restrict__ Alo, double* __restrict__ part,
                                                   double* __restrict__ partG) {
  long long i0 = blockIdx.x * (long long)CTILE;
  dd acc{0.0, 0.0}, accG{0.0, 0.0};
  for (int k = 0; k < CI; ++k) {
    long long u = i0 + (long long)k * CT + threadIdx.x;
    if (u < n) {
      dd A{Ahi[u], Alo[u]};
      const double wu = w[u], gu = gE[u];
      acc = dd_add_dekker(acc, dd_mul_d(dd_mul_d(A, wu), gu));
      accG = dd_add_dekker(accG, dd_two_prod(gu, wu));
    }
  }
  dd t = dd_block_reduce(acc);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = t.hi;
    part[2 * blockIdx.x + 1] = t.lo;
  }
  t = dd_block_reduce(accG);
  if (threadIdx.x == 0) {
    partG[2 * blockIdx.x] = t.hi;
    partG[2 * blockIdx.x + 1] = t.lo;
  }
}

__global__ void sum_partials_kernel(const double* __restrict__ part, long long nt, const double* __restrict__ sc,
                                    double* __restrict__ out) {
  const dd iS{sc[1], sc[2]};
  dd acc{0.0, 0.0};
  for (long long i = threadIdx.x; i < nt; i += blockDim.x) acc = dd_add_dekker(acc, dd{part[2 * i], part[2 * i + 1]});
  dd t = dd_block_reduce(acc);
  if (threadIdx.x == 0) {
    dd K = dd_mul(t, iS);
    out[0] = K.hi;
    out[1] = K.lo;
  }
}

__global__ void __launch_bounds__(CT) adj_grad_kernel(const double* __restrict__ w, const double* __restrict__ gE,
                                                      long long n, const double* __restrict__ sc,
                                                      const long long* __restrict__ tcap,
                                                      const double* __restrict__ Ahi, const double* __restrict__ Alo,
                                                      const double* __restrict__ G, const double* __restrict__ Kp,
                                                      double* __restrict__ gw) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k >= n) return;
  const dd iS{sc[1], sc[2]};
  long long t = tcap[k];
  dd A{Ahi[k], Alo[k]};
  dd B{G[2 * t], G[2 * t + 1]};
  if (k >= t) {
    dd gw_k = dd_two_prod(gE[k], w[k]);
    B = dd_add_dekker(B, dd{-gw_k.hi, -gw_k.lo});
  }
  dd num = dd_add_dekker(dd_add_dekker(dd_mul_d(A, gE[k]), B), dd{-Kp[0], -Kp[1]});
  dd r = dd_mul(num, iS);
  gw[k] = r.hi + r.lo;
}

// S = sum w in double-double, rounded once (block partials, then one block)
__global__ void __launch_bounds__(CT) sum_reduce_kernel(const double* __restrict__ w, long long n,
                                                        double* __restrict__ part) {
  long long i0 = blockIdx.x * (long long)CTILE;
  dd acc{0.0, 0.0};
  for (int k = 0; k < CI; ++k) {
    long long i = i0 + (long long)k * CT + threadIdx.x;
    if (i < n) acc = dd_add_dekker(acc, dd{w[i], 0.0});
  }
  dd t = dd_block_reduce(acc);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = t.hi;
    part[2 * blockIdx.x + 1] = t.lo;
  }
}

__global__ void sum_final_kernel(const double* __restrict__ part, long long nt, double* __restrict__ out) {
  dd acc{0.0, 0.0};
  for (long long i = threadIdx.x; i < nt; i += blockDim.x) acc = dd_add_dekker(acc, dd{part[2 * i], part[2 * i + 1]});
  dd t = dd_block_reduce(acc);
  if (threadIdx.x == 0) out[0] = t.hi + t.lo;
}

// one calibration step, per node: max relative error of E against the target,
// then the preconditioned gradient step w - g / H, H = 2 J^2 / d, J = A / S
__global__ void __launch_bounds__(CT) relerr_kernel(const double* __restrict__ E, const double* __restrict__ d,
                                                    long long n, unsigned long long* __restrict__ maxbits,
                                                    double* __restrict__ gE) {
  long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double r = 0.0;
  if (u < n) {
    const double diff = E[u] - d[u], id = 1.0 / d[u];
    r = fabs(diff) * id;
    gE[u] = 2.0 * diff * id;  // dL/dE for L = sum (E - d)^2 / d
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(FULL_MASK, r, o));
  if ((threadIdx.x & 31) == 0 && r > 0.0) atomicMax(maxbits, (unsigned long long)__double_as_longlong(r));
}

__global__ void __launch_bounds__(CT) step_kernel(double* __restrict__ w, const double* __restrict__ d,
                                                  const double* __restrict__ g, const double* __restrict__ Ahi,
                                                  long long n, const double* __restrict__ sc) {
  long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (u >= n) return;
  double J = Ahi[u] * sc[1];
  J = J > 1e-300 ? J : 1e-300;
  double H = 2.0 * J * J / d[u];
  double wn = w[u] - g[u] / H;
  double floor_ = 1e-9 * d[u];
  w[u] = wn > floor_ ? wn : floor_;
}

// keep w non-increasing: w_u <- min_{v <= u} w_v (a running minimum, one block per tile + carry)
__global__ void __launch_bounds__(CT) runmin_tile_kernel(const double* __restrict__ w, long long n,
                                                         double* __restrict__ part) {
  long long i0 = blockIdx.x * (long long)CTILE;
  double m = INFINITY;
  for (int k = 0; k < CI; ++k) {
    long long i = i0 + (long long)k * CT + threadIdx.x;
    if (i < n) m = fmin(m, w[i]);
  }
  __shared__ double sm[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(FULL_MASK, m, o));
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = INFINITY;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t = fmin(t, sm[k]);
    part[blockIdx.x] = t;
  }
}

// exclusive running minimum of the tile minima (one block, 1024 values per round)
__global__ void runmin_partials_kernel(double* __restrict__ part, long long nt) {
  __shared__ double sm[1024];
  __shared__ double carry;
  if (threadIdx.x == 0) carry = INFINITY;
  __syncthreads();
  for (long long base = 0; base < nt; base += blockDim.x) {
    const long long i = base + threadIdx.x;
    const double v = i < nt ? part[i] : INFINITY;
    sm[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
      const double y = threadIdx.x >= (unsigned)o ? sm[threadIdx.x - o] : INFINITY;
      __syncthreads();
      sm[threadIdx.x] = fmin(sm[threadIdx.x], y);
      __syncthreads();
    }
    const double c = carry;
    const double ex = fmin(c, threadIdx.x > 0 ? sm[threadIdx.x - 1] : INFINITY);
    __syncthreads();
    if (i < nt) part[i] = ex;
    if (threadIdx.x == blockDim.x - 1) carry = fmin(c, sm[threadIdx.x]);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(CT) runmin_apply_kernel(double* __restrict__ w, long long n,
                                                          const double* __restrict__ part) {
  long long i0 = blockIdx.x * (long long)CTILE + (long long)threadIdx.x * CI;
  double v[CI];
  double loc = INFINITY;
#pragma unroll
  for (int k = 0; k < CI; ++k) {
    v[k] = i0 + k < n ? w[i0 + k] : INFINITY;
    loc = fmin(loc, v[k]);
  }
  // exclusive running minimum across the block's threads
  __shared__ double sm[CT];
  sm[threadIdx.x] = loc;
  __syncthreads();
  for (int o = 1; o < CT; o <<= 1) {
    double y = threadIdx.x >= (unsigned)o ? sm[threadIdx.x - o] : INFINITY;
    __syncthreads();
    sm[threadIdx.x] = fmin(sm[threadIdx.x], y);
    __syncthreads();
  }
  double run = threadIdx.x > 0 ? sm[threadIdx.x - 1] : INFINITY;
  run = fmin(run, part[blockIdx.x]);
#pragma unroll
  for (int k = 0; k < CI; ++k) {
    run = fmin(run, v[k]);
    if (i0 + k < n) w[i0 + k] = run;
  }
}

// The call's S and its double-double reciprocal, sc = {S, 1/S hi, 1/S lo}: from a
// given S, or from the forward pass's double-double sum of w (rounded once).
__device__ __forceinline__ void put_scal(double S, double* sc) {
  const double h = 1.0 / S;
  sc[0] = S;
  sc[1] = h;
  sc[2] = fma(-h, S, 1.0) / S;
}
__global__ void scal_set_kernel(double S, double* __restrict__ sc) { put_scal(S, sc); }
__global__ void scal_from_total_kernel(const double* __restrict__ tot, double* __restrict__ sc) {
  put_scal(tot[0] + tot[1], sc);
}

struct CalWs {
  double* R;      // 2 (n + 1)
  double* G;      // 2 (n + 1)
  long long* t;   // n
  double* Ahi;    // n
  double* Alo;    // n
  double* part;   // 2 tiles
  double* part2;  // 2 tiles
  double* scal;   // 16: S, 1/S (2), -, K (2), sum w (2), sum gE w (2)
  long long* t0;  // the largest threshold
  unsigned long long* maxbits;
  double* E;      // n (calibration)
  double* gE;     // n (calibration)
  double* g;      // n (calibration)
  size_t bytes;
};

size_t al(size_t x) { return (x + 255) / 256 * 256; }

CalWs cal_layout(void* base, long long n, bool calib) {
  char* b = (char*)base;
  size_t off = 0;
  CalWs L;
  auto take = [&](size_t bytes) -> void* {
    void* p = b ? (void*)(b + off) : nullptr;
    off += al(bytes);
    return p;
  };
  long long nt = (n + CTILE - 1) / CTILE + 1;
  L.R = (double*)take(sizeof(double) * 2 * (n + 1));
  L.G = (double*)take(sizeof(double) * 2 * (n + 1));
  L.t = (long long*)take(sizeof(long long) * (n > 0 ? n : 1));
  L.Ahi = (double*)take(sizeof(double) * (n > 0 ? n : 1));
  L.Alo = (double*)take(sizeof(double) * (n > 0 ? n : 1));
  L.part = (double*)take(sizeof(double) * 2 * nt);
  L.part2 = (double*)take(sizeof(double) * 2 * nt);
  L.scal = (double*)take(sizeof(double) * 16);
  L.t0 = (long long*)take(sizeof(long long) * 2);
  L.maxbits = (unsigned long long*)take(sizeof(unsigned long long) * 2);
  L.E = calib ? (double*)take(sizeof(double) * (n > 0 ? n : 1)) : nullptr;
  L.gE = calib ? (double*)take(sizeof(double) * (n > 0 ? n : 1)) : nullptr;
  L.g = calib ? (double*)take(sizeof(double) * (n > 0 ? n : 1)) : nullptr;
  L.bytes = off;
  return L;
}

void device_sum(const double* w, long long n, double* part, double* out, cudaStream_t s) {
  long long nt = (n + CTILE - 1) / CTILE;
  if (nt < 1) nt = 1;
  sum_reduce_kernel<<<(unsigned)nt, CT, 0, s>>>(w, n, part);
  sum_final_kernel<<<1, 1024, 0, s>>>(part, nt, out);
}

unsigned nblk(long long n) { return (unsigned)((n + CT - 1) / CT); }

// X_k = sum_{i >= k} x_i for k <= t_0 (x_i = a_i, or a_i b_i exactly), given tot = the total
// m = t_0 must be in L.t0 (the forward pass puts it there)
void tail_sums(const double* a, const double* b, long long n, const CalWs& L, const double* tot, double* X,
               cudaStream_t s) {
  const long long nt = (n + CTILE - 1) / CTILE;
  tile_sum_kernel<<<(unsigned)nt, CT, 0, s>>>(a, b, n, L.t0, L.part);
  suffix_partials_kernel<<<1, 1024, 0, s>>>(L.part, nt, L.t0);
  tail_scan_kernel<<<(unsigned)nt, CT, 0, s>>>(a, b, n, L.t0, L.part, tot, X);
}

// E and the per-node forward quantities; S from L.scal, or (sum_S) the sum of w put there
void forward(const double* w, long long n, bool sum_S, double* E, const CalWs& L, cudaStream_t s) {
  const long long nt = (n + CTILE - 1) / CTILE;
  tile_sum_kernel<<<(unsigned)nt, CT, 0, s>>>(w, nullptr, n, nullptr, L.part);
  total_kernel<<<1, 1024, 0, s>>>(L.part, nt, L.scal + 6);
  if (sum_S) scal_from_total_kernel<<<1, 1, 0, s>>>(L.scal + 6, L.scal);
  t0_kernel<<<1, 1, 0, s>>>(w, n, L.scal, L.t0);
  tail_sums(w, nullptr, n, L, L.scal + 6, L.R, s);
  expdeg_kernel<<<nblk(n), CT, 0, s>>>(w, n, L.scal, L.R, E, L.t, L.Ahi, L.Alo);
}

void adjoint(const double* w, const double* gE, long long n, double* gw, const CalWs& L, cudaStream_t s) {
  long long nt = (n + CTILE - 1) / CTILE;
  adj_K_kernel<<<(unsigned)nt, CT, 0, s>>>(w, gE, n, L.Ahi, L.Alo, L.part, L.part2);
  sum_partials_kernel<<<1, 1024, 0, s>>>(L.part, nt, L.scal, L.scal + 4);
  total_kernel<<<1, 1024, 0, s>>>(L.part2, nt, L.scal + 8);  // sum_u gE_u w_u
  tail_sums(gE, w, n, L, L.scal + 8, L.G, s);
  adj_grad_kernel<<<nblk(n), CT, 0, s>>>(w, gE, n, L.scal, L.t, L.Ahi, L.Alo, L.G, L.scal + 4, gw);
}

}  // namespace
}  // namespace cl

using namespace cl;

static cl_status ok_last() { return cudaGetLastError() == cudaSuccess ? CL_OK : CL_ERR_CUDA; }

extern "C" size_t cl_expected_degree_workspace_bytes(int64_t n) {
  if (n < 0) return 0;
  return cal_layout(nullptr, n, false).bytes;
}

extern "C" size_t cl_calibrate_workspace_bytes(int64_t n) {
  if (n < 0) return 0;
  return cal_layout(nullptr, n, true).bytes;
}

static cl_status resolve_S(const double* d_w, int64_t n, double S, const CalWs& L, cudaStream_t s, double* out) {
  if (S > 0) {
    *out = S;
    return CL_OK;
  }
  device_sum(d_w, n, L.part, L.scal, s);
  if (cudaMemcpyAsync(out, L.scal, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CL_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CL_ERR_CUDA;
  return *out > 0 ? CL_OK : CL_ERR_RANGE;
}

extern "C" cl_status cl_expected_degree(const double* d_w, int64_t n, double S, double* d_E, void* d_ws,
                                        size_t ws_bytes, cl_stream_t stream) {
  if (n < 0 || (n > 0 && (!d_w || !d_E))) return CL_ERR_INVALID_ARG;
  if (n == 0) return CL_OK;
  CalWs L = cal_layout(d_ws, n, false);
  if (!d_ws || ws_bytes < L.bytes) return CL_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  cl_status st = resolve_S(d_w, n, S, L, s, &S);
  if (st != CL_OK) return st;
  scal_set_kernel<<<1, 1, 0, s>>>(S, L.scal);
  forward(d_w, n, false, d_E, L, s);
  return ok_last();
}

extern "C" cl_status cl_expected_degree_adjoint(const double* d_w, const double* d_gE, int64_t n, double S,
                                                double* d_gw, void* d_ws, size_t ws_bytes, cl_stream_t stream) {
  if (n < 0 || (n > 0 && (!d_w || !d_gE || !d_gw))) return CL_ERR_INVALID_ARG;
  if (n == 0) return CL_OK;
  CalWs L = cal_layout(d_ws, n, false);
  if (!d_ws || ws_bytes < L.bytes) return CL_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  cl_status st = resolve_S(d_w, n, S, L, s, &S);
  if (st != CL_OK) return st;
  scal_set_kernel<<<1, 1, 0, s>>>(S, L.scal);
  forward(d_w, n, false, nullptr, L, s);  // the forward quantities (R, t, A) the adjoint needs
  adjoint(d_w, d_gE, n, d_gw, L, s);
  return ok_last();
}

extern "C" cl_status cl_calibrate(const double* d_target, int64_t n, double* d_w, const cl_calib_opts* opts,
                                  cl_calib_report* report, void* d_ws, size_t ws_bytes, cl_stream_t stream) {
  if (n <= 0 || !d_target || !d_w) return CL_ERR_INVALID_ARG;
  CalWs L = cal_layout(d_ws, n, true);
  if (!d_ws || ws_bytes < L.bytes) return CL_ERR_WORKSPACE;
  cudaStream_t s = (cudaStream_t)stream;
  double tol = (opts && opts->tol > 0) ? opts->tol : 1e-9;
  int max_iter = (opts && opts->max_iter > 0) ? opts->max_iter : 100;
  if (!(opts && opts->init_from_w))
    if (cudaMemcpyAsync(d_w, d_target, sizeof(double) * n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return CL_ERR_CUDA;
  long long nt = (n + CTILE - 1) / CTILE;
  double S = 0, maxrel = INFINITY;
  int it = 0;
  for (;; ++it) {
    // S = the forward pass's sum of w, kept on the device; one host read per
    // iteration (the convergence test)
    cudaMemsetAsync(L.maxbits, 0, sizeof(unsigned long long), s);
    unsigned long long bits = 0;
    forward(d_w, n, true, L.E, L, s);
    relerr_kernel<<<nblk(n), CT, 0, s>>>(L.E, d_target, n, L.maxbits, L.gE);
    if (cudaMemcpyAsync(&bits, L.maxbits, sizeof(bits), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CL_ERR_CUDA;
    if (cudaMemcpyAsync(&S, L.scal, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CL_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CL_ERR_CUDA;
    std::memcpy(&maxrel, &bits, sizeof(double));
    if (maxrel <= tol || it >= max_iter) break;
    adjoint(d_w, L.gE, n, L.g, L, s);
    step_kernel<<<nblk(n), CT, 0, s>>>(d_w, d_target, L.g, L.Ahi, n, L.scal);
    runmin_tile_kernel<<<(unsigned)nt, CT, 0, s>>>(d_w, n, L.part);
    runmin_partials_kernel<<<1, 1024, 0, s>>>(L.part, nt);
    runmin_apply_kernel<<<(unsigned)nt, CT, 0, s>>>(d_w, n, L.part);
    if (ok_last() != CL_OK) return CL_ERR_CUDA;
  }
  if (report) {
    report->iterations = it;
    report->max_rel_err = maxrel;
    report->S = S;
  }
  return maxrel <= tol ? CL_OK : CL_ERR_RANGE;
}
