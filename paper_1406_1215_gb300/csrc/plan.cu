// plan.cu -- planning kernels: validation and the exact sum S (Algorithm 1,
// first line; Section 4's parallel sum), the weight prefix sigma, item costs
// (Eq. 1-2, Eq. 6), their inclusive prefix (Calc-Cost of Algorithm 2 as a
// device-wide scan) and the task boundaries of Eq. 3.  Also the int32 ->
// int64 exclusive scan that turns per-item edge counts into offsets.
//
// Scans are three-phase (tile reduce, scan of tile partials, tile scan): no
// block ever waits on another block.
#include <cuda_runtime.h>

#include "cl_internal.cuh"

namespace cl {

constexpr int PLAN_THREADS = 256;
constexpr int ANALYZE_CHUNK = 4096;  // weights per analysis block
constexpr int SCAN_ITEMS = 8;        // items per thread in a scan tile
constexpr int SCAN_TILE = PLAN_THREADS * SCAN_ITEMS;
constexpr int F64_BINS = 2048;       // one bin per biased double exponent

// --------------------------------------------------------------- block scans
template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T x = __shfl_up_sync(FULL_MASK, v, o);
    if (lane >= o) v += x;
  }
  return v;
}

// Exclusive block scan of one value per thread; returns the block total in *total.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T* total) {
  __shared__ T warp_tot[32];
  __shared__ T block_tot;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T inc = warp_incl_scan(v);
  if (lane == 31) warp_tot[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T t = lane < nw ? warp_tot[lane] : T(0);
    T ti = warp_incl_scan(t);
    if (lane < nw) warp_tot[lane] = ti - t;
    if (lane == nw - 1) block_tot = ti;
  }
  __syncthreads();
  T res = warp_tot[wid] + inc - v;
  *total = block_tot;
  __syncthreads();
  return res;
}

template <typename T>
__device__ __forceinline__ T block_reduce(T v) {
  __shared__ T red[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL_MASK, v, o);
  if (lane == 0) red[wid] = v;
  __syncthreads();
  T t = T(0);
  if (wid == 0) {
    t = lane < nw ? red[lane] : T(0);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL_MASK, t, o);
  }
  __syncthreads();
  return t;  // valid in warp 0
}

// Single-block exclusive scan of n partials in place; optional segment heads
// (head[i] != 0 restarts the running sum at i).  Returns nothing; total unused.
template <typename T>
__global__ void partials_scan_kernel(T* __restrict__ part, long long n, const unsigned char* __restrict__ head) {
  __shared__ T carry_s;
  if (threadIdx.x == 0) carry_s = T(0);
  __syncthreads();
  for (long long base = 0; base < n; base += blockDim.x) {
    long long i = base + threadIdx.x;
    T v = i < n ? part[i] : T(0);
    bool h = (head != nullptr && i < n) ? head[i] != 0 : false;
    T carry = carry_s;
    if (head == nullptr) {
      T tot;
      T ex = block_excl_scan(v, &tot);
      if (i < n) part[i] = carry + ex;
      if (threadIdx.x == 0) carry_s = carry + tot;
      __syncthreads();
    } else {
      // segmented: sequential within the chunk by thread 0 (partials are few)
      __shared__ T vals[1024];
      __shared__ unsigned char hs[1024];
      vals[threadIdx.x] = v;
      hs[threadIdx.x] = h;
      __syncthreads();
      if (threadIdx.x == 0) {
        T run = carry;
        long long lim = n - base < (long long)blockDim.x ? n - base : (long long)blockDim.x;
        for (long long k = 0; k < lim; ++k) {
          if (hs[k]) run = T(0);
          T x = vals[k];
          vals[k] = run;
          run += x;
        }
        carry_s = run;
      }
      __syncthreads();
      if (i < n) part[i] = vals[threadIdx.x];
      __syncthreads();
    }
  }
}

// --------------------------------------------------------------- analysis
__device__ __forceinline__ int block_graph(const long long* blk_begin, int G, long long b) {
  int lo = 0, hi = G - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (blk_begin[mid] <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// 128-bit bin add: lo with carry into hi (both 64-bit words, order independent).
__device__ __forceinline__ void bin_add_shared(unsigned long long* lo, unsigned long long* hi, unsigned long long m) {
  unsigned long long old = atomicAdd(lo, m);
  if (old + m < old) atomicAdd(hi, 1ull);
}

template <bool F64>
__global__ void __launch_bounds__(PLAN_THREADS) analyze_kernel(const DevGraph* __restrict__ gs,
                                                               const long long* __restrict__ blk_begin, int G,
                                                               const double* __restrict__ heavy_w,
                                                               GraphAnalysis* __restrict__ out,
                                                               unsigned long long* __restrict__ bins) {
  extern __shared__ unsigned long long sbins[];  // F64: 2 * F64_BINS words (lo, hi)
  const long long b = blockIdx.x;
  const int g = block_graph(blk_begin, G, b);
  const DevGraph& gr = gs[g];
  const long long lb = b - blk_begin[g];
  const long long n = gr.n;
  const double hw = heavy_w[g];
  long long i0 = lb * ANALYZE_CHUNK;
  long long i1 = i0 + ANALYZE_CHUNK < n ? i0 + ANALYZE_CHUNK : n;
  unsigned flags = 0;
  unsigned long long heavy = 0, sum = 0;
  double sq = 0.0;
  if (F64) {
    for (int k = threadIdx.x; k < 2 * F64_BINS; k += blockDim.x) sbins[k] = 0;
    __syncthreads();
    const double* w = (const double*)gr.w;
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      double x = w[i];
      if (!(x >= 0.0) || !isfinite(x)) {
        flags |= 2u;
        continue;
      }
      if (i + 1 < n && x < w[i + 1]) flags |= 1u;
      if (x >= hw) ++heavy;
      sq += x * x;
      unsigned long long bits = (unsigned long long)__double_as_longlong(x);
      int e = (int)(bits >> 52);
      unsigned long long m = bits & ((1ull << 52) - 1);
      if (e > 0) m |= 1ull << 52;
      int bin = e > 0 ? e : 1;  // subnormals share the scale of the smallest normal
      if (m) bin_add_shared(&sbins[2 * bin], &sbins[2 * bin + 1], m);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < F64_BINS; k += blockDim.x) {
      unsigned long long lo = sbins[2 * k], hi = sbins[2 * k + 1];
      unsigned long long* gb = bins + ((size_t)g * F64_BINS + k) * 2;
      if (lo) bin_add_shared(&gb[0], &gb[1], lo);  // global atomics, same carry rule
      if (hi) atomicAdd(&gb[1], hi);
    }
  } else {
    // integers only in the loop (int <-> double conversions run at the FP64 rate here):
    // x >= hw  <=>  x >= ceil(hw) for an integer x; squares summed exactly in 128 bits
    const long long hwi = hw <= 0.0 ? 0 : (hw > 4294967296.0 ? (1ll << 33) : (long long)ceil(hw));
    const int* w = (const int*)gr.w;
    unsigned __int128 sq_i = 0;
    for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      int x = w[i];
      if (x < 0) flags |= 2u;
      if (i + 1 < n && x < w[i + 1]) flags |= 1u;
      if ((long long)x >= hwi) ++heavy;
      sum += (unsigned long long)(long long)x;
      sq_i += (unsigned long long)((long long)x * (long long)x);
    }
    sq = (double)(unsigned long long)(sq_i >> 64) * 18446744073709551616.0 + (double)(unsigned long long)sq_i;
  }
  // block reductions
  unsigned long long s = block_reduce(sum);
  unsigned long long h = block_reduce(heavy);
  double q2 = block_reduce(sq);
  unsigned f1 = __syncthreads_or(flags & 1u) ? 1u : 0u;
  unsigned f2 = __syncthreads_or(flags & 2u) ? 2u : 0u;
  unsigned f = f1 | f2;
  if (threadIdx.x == 0) {
    if (!F64 && s) atomicAdd(&out[g].S_i, s);
    if (h) atomicAdd(&out[g].H, h);
    if (q2 > 0.0) atomicAdd(&out[g].S2, q2);
    if (f) atomicOr(&out[g].flags, f);
  }
}

size_t f64_bins_bytes(int G) { return (size_t)G * F64_BINS * 2 * sizeof(unsigned long long); }

// callers zero d_out (and, for double weights, the bins) beforehand
void launch_analyze(const DevGraph* d_graphs, const long long* d_blk_begin, int G, long long nblocks,
                    const double* d_heavy_w, GraphAnalysis* d_out, unsigned long long* d_bins, bool f64,
                    cudaStream_t s) {
  if (nblocks <= 0) return;
  if (f64) {
    size_t smem = 2 * F64_BINS * sizeof(unsigned long long);
    cudaFuncSetAttribute(analyze_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    analyze_kernel<true><<<(unsigned)nblocks, PLAN_THREADS, smem, s>>>(d_graphs, d_blk_begin, G, d_heavy_w, d_out,
                                                                       d_bins);
  } else {
    analyze_kernel<false><<<(unsigned)nblocks, PLAN_THREADS, 0, s>>>(d_graphs, d_blk_begin, G, d_heavy_w, d_out,
                                                                     d_bins);
  }
}

// Exact sum of double weights: the bins hold sum_b m_b 2^(b-1075) exactly as
// 128-bit integers; one thread per graph forms the big integer (base 2^32
// digits, bit 0 = 2^-1074) and rounds it once to nearest-even.
__global__ void f64_sum_finalize_kernel(int G, const unsigned long long* __restrict__ bins,
                                        GraphAnalysis* __restrict__ out) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= G) return;
  constexpr int ND = 72;  // 2304 bits
  unsigned long long acc[ND];
  for (int d = 0; d < ND; ++d) acc[d] = 0;
  const unsigned long long* gb = bins + (size_t)g * F64_BINS * 2;
  for (int b = 1; b < F64_BINS - 1; ++b) {
    unsigned long long lo = gb[2 * b], hi = gb[2 * b + 1];
    if (!lo && !hi) continue;
    int pos = b - 1;  // bit position of 2^(b-1075) relative to 2^-1074
    // add lo at pos, hi at pos + 64, as 32-bit pieces
    unsigned long long parts[4] = {lo & 0xFFFFFFFFull, lo >> 32, hi & 0xFFFFFFFFull, hi >> 32};
    for (int k = 0; k < 4; ++k) {
      if (!parts[k]) continue;
      int p = pos + 32 * k;
      int d = p >> 5, o = p & 31;
      unsigned long long v = parts[k] << o;  // < 2^63
      acc[d] += v & 0xFFFFFFFFull;
      acc[d + 1] += v >> 32;
    }
  }
  for (int d = 0; d + 1 < ND; ++d) {
    acc[d + 1] += acc[d] >> 32;
    acc[d] &= 0xFFFFFFFFull;
  }
  int top = -1;
  for (int d = ND - 1; d >= 0 && top < 0; --d)
    if (acc[d]) top = 32 * d + 31 - __clzll(acc[d] << 32);
  double S = 0.0;
  if (top >= 0) {
    auto bit = [&](int p) -> unsigned long long {
      return p < 0 ? 0ull : (acc[p >> 5] >> (p & 31)) & 1ull;
    };
    if (top <= 52) {
      unsigned long long M = 0;
      for (int p = top; p >= 0; --p) M = (M << 1) | bit(p);
      S = __ll2double_rn((long long)M) * 0x1p-1074;  // exact (fits 53 bits)
    } else {
      unsigned long long M = 0;
      for (int p = top; p > top - 53; --p) M = (M << 1) | bit(p);
      int rb = top - 53;
      unsigned long long round = bit(rb);
      bool sticky = false;
      for (int p = rb - 1; p >= 0 && !sticky; --p) sticky = bit(p) != 0;
      if (round && (sticky || (M & 1ull))) ++M;
      int ex = top - 52 - 1074;
      if (M == (1ull << 53)) {
        M >>= 1;
        ++ex;
      }
      S = ldexp((double)M, ex);  // M has <= 53 bits: exact scaling unless it overflows
    }
  }
  out[g].S_d = S;
}

void launch_f64_sum_finalize(int G, const unsigned long long* d_bins, GraphAnalysis* d_out, cudaStream_t s) {
  f64_sum_finalize_kernel<<<(G + 31) / 32, 32, 0, s>>>(G, d_bins, d_out);
}

// --------------------------------------------------------------- weight prefix
// sigma over the concatenation of the graphs' weight arrays, each followed by
// one zero (so graph g's prefix P[pbase_g + u], u = 0..n_g, differs from
// sigma_u by the constant P[pbase_g], which cancels in every difference the
// costs use).  Exact int64 for integer weights; double for double weights.
template <typename T>
__device__ __forceinline__ T weight_at(const DevGraph& g, long long u) {
  if (u >= g.n) return T(0);
  if (g.wtype == CL_W_F64) return (T)((const double*)g.w)[u];
  return (T)((const int*)g.w)[u];
}

template <typename T>
__global__ void __launch_bounds__(PLAN_THREADS) wprefix_reduce_kernel(const DevGraph* __restrict__ gs,
                                                                      const long long* __restrict__ tbeg, int G,
                                                                      T* __restrict__ part) {
  const long long t = blockIdx.x;
  const int g = block_graph(tbeg, G, t);
  const DevGraph& gr = gs[g];
  const long long e0 = (t - tbeg[g]) * SCAN_TILE, len = gr.n + 1;
  T acc = T(0);
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    long long u = e0 + (long long)k * PLAN_THREADS + threadIdx.x;
    if (u < len) acc += weight_at<T>(gr, u);
  }
  T tot = block_reduce(acc);
  if (threadIdx.x == 0) part[t] = tot;
}

template <typename T>
__global__ void __launch_bounds__(PLAN_THREADS) wprefix_scan_kernel(const DevGraph* __restrict__ gs,
                                                                    const long long* __restrict__ tbeg, int G,
                                                                    const T* __restrict__ part, T* __restrict__ P) {
  const long long t = blockIdx.x;
  const int g = block_graph(tbeg, G, t);
  const DevGraph& gr = gs[g];
  const long long e0 = (t - tbeg[g]) * SCAN_TILE, len = gr.n + 1;
  long long u0 = e0 + (long long)threadIdx.x * SCAN_ITEMS;
  T v[SCAN_ITEMS];
  T loc = T(0);
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    v[k] = (u0 + k < len) ? weight_at<T>(gr, u0 + k) : T(0);
    loc += v[k];
  }
  T tot;
  T ex = block_excl_scan(loc, &tot) + part[t];
  // staged in shared memory (one pad word per thread's 8) and written out coalesced
  __shared__ T res[SCAN_TILE + PLAN_THREADS];
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    res[threadIdx.x * (SCAN_ITEMS + 1) + k] = ex;
    ex += v[k];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    const int q = k * PLAN_THREADS + threadIdx.x;
    if (e0 + q < len) P[gr.pbase + e0 + q] = res[q + q / SCAN_ITEMS];
  }
}

void launch_weight_prefix(const DevGraph* d_graphs, const long long* d_tile_graph_begin, int G, long long ntiles,
                          bool f64, void* d_P, void* d_partials, cudaStream_t s) {
  if (ntiles <= 0) return;
  if (f64) {
    wprefix_reduce_kernel<double><<<(unsigned)ntiles, PLAN_THREADS, 0, s>>>(d_graphs, d_tile_graph_begin, G,
                                                                           (double*)d_partials);
    partials_scan_kernel<double><<<1, 1024, 0, s>>>((double*)d_partials, ntiles, nullptr);
    wprefix_scan_kernel<double><<<(unsigned)ntiles, PLAN_THREADS, 0, s>>>(
        d_graphs, d_tile_graph_begin, G, (const double*)d_partials, (double*)d_P);
  } else {
    wprefix_reduce_kernel<long long><<<(unsigned)ntiles, PLAN_THREADS, 0, s>>>(d_graphs, d_tile_graph_begin, G,
                                                                              (long long*)d_partials);
    partials_scan_kernel<long long><<<1, 1024, 0, s>>>((long long*)d_partials, ntiles, nullptr);
    wprefix_scan_kernel<long long><<<(unsigned)ntiles, PLAN_THREADS, 0, s>>>(
        d_graphs, d_tile_graph_begin, G, (const long long*)d_partials, (long long*)d_P);
  }
}

// --------------------------------------------------------------- weight blocks
// Integer weights sorted non-increasing: node block b of graph g (nodes
// 4096 b .. 4096 b + 4095) is uniform iff its first and last weights are equal.
// blk[bbase_g + b] = (w << 32) | end for a uniform block, end being the first
// node after the block's run (found by bisection over the sorted weights), and
// BLK_MIXED for a block that holds a change of weight.  The sampler reads a
// candidate's weight from this table when its block is uniform (the tail of a
// power law, where the weight array is far larger than L2) and from the weight
// array otherwise (the head, a few MB that stay in L2).
__global__ void __launch_bounds__(PLAN_THREADS) blocks_kernel(const DevGraph* __restrict__ gs, int G,
                                                              long long nblk, unsigned long long* __restrict__ blk) {
  const long long x = blockIdx.x * (long long)PLAN_THREADS + threadIdx.x;
  if (x >= nblk) return;
  int lo = 0, hi = G - 1;  // last graph with bbase <= x
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (gs[mid].bbase <= x) lo = mid;
    else hi = mid - 1;
  }
  const DevGraph& g = gs[lo];
  const int* w = (const int*)g.w;
  const long long n = g.n, a = (x - g.bbase) << BLK_SHIFT;
  long long last = a + (1ll << BLK_SHIFT) - 1;
  if (last > n - 1) last = n - 1;
  const int wa = w[a];
  if (w[last] != wa) {
    blk[x] = BLK_MIXED;
    return;
  }
  long long l = last, h = n;  // first index > last with w < wa, in (last, n]
  while (h - l > 1) {
    long long mid = (l + h) >> 1;
    if (w[mid] == wa) l = mid;
    else h = mid;
  }
  blk[x] = ((unsigned long long)(unsigned)wa << 32) | (unsigned long long)h;
}

void launch_blocks(const DevGraph* d_graphs, int G, long long nblk, unsigned long long* d_blk, cudaStream_t s) {
  if (nblk <= 0) return;
  blocks_kernel<<<(unsigned)((nblk + PLAN_THREADS - 1) / PLAN_THREADS), PLAN_THREADS, 0, s>>>(d_graphs, G, nblk, d_blk);
}

// --------------------------------------------------------------- costs, Eq. 3
// c_i = c0 + (w_u / S) * sum_{v in [j0, end)} w_v  (Eq. 1-2; for a light row
// [u+1, n) this is Eq. 6: (w_u / S)(S - sigma_u - w_u) + c0), in fixed point
// with 1/16-edge units so that its prefix is an exact integer.  The constant
// term is the work of an item apart from its edges; Eq. 1 counts it as 1, but
// here an item's set-up and end (bounds, first weight and L_p, the lane refill,
// the count and the staging flush) cost about as much as 4 loop iterations, so
// c0 = 4: tasks of equal cost then take equal time whether they hold a few long
// items or many short ones.  Costs only schedule work, so single precision is
// enough for their value (FP64 runs at 1/75 of FP32 here).
constexpr long long ITEM_COST_16 = 64;  // c0 = 4 edges, in 1/16-edge units

template <typename T>
__global__ void __launch_bounds__(PLAN_THREADS) costs_kernel(const DevGraph* __restrict__ gs, int G,
                                                             long long n_items, const T* __restrict__ P,
                                                             long long* __restrict__ C, int* __restrict__ slot,
                                                             int tiny_slots) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n_items) return;
  int g = G == 1 ? 0 : graph_of_item(gs, G, i);
  const DevGraph& gr = gs[g];
  unsigned u, seg, j0, end;
  item_bounds(gr, i - gr.item_begin, u, seg, j0, end);
  constexpr bool ints = T(1) / T(2) == T(0);  // integer weights, int64 prefix
  float wu, dP, len;
  if (ints) {
    wu = u32_to_f((unsigned)((const int*)gr.w)[u]);
    dP = u64_to_f((unsigned long long)(P[gr.pbase + end] - P[gr.pbase + j0]));
    len = u32_to_f(end - j0);
  } else {
    wu = (float)weight_at<T>(gr, u);
    dP = (float)(P[gr.pbase + end] - P[gr.pbase + j0]);
    len = (float)(end - j0);
  }
  float e = wu * dP * gr.invS_f;  // expected edges of the item (uncapped)
  e = fminf(e, 1e15f);
  C[i] = ITEM_COST_16 + f_floor_to_ll(16.0f * e + 0.5f);
  if (slot) {
    // staging slot: e + 6 sd + 6 entries in whole sectors, at most the item's length
    float want = tiny_slots ? 8.0f : e + 6.0f * sqrtf(e) + 6.0f;
    want = fminf(want, len);
    want = fminf(want, 1e9f);
    slot[i] = (f_ceil_to_i(want) + 7) & ~7;
  }
}

__global__ void __launch_bounds__(PLAN_THREADS) tile_reduce_i64_kernel(const long long* __restrict__ x, long long n,
                                                                       long long* __restrict__ part) {
  long long e0 = blockIdx.x * (long long)SCAN_TILE;
  long long acc = 0;
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    long long i = e0 + (long long)k * PLAN_THREADS + threadIdx.x;
    if (i < n) acc += x[i];
  }
  long long tot = block_reduce(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// in-place inclusive scan of int64 with tile partials
__global__ void __launch_bounds__(PLAN_THREADS) tile_incl_scan_i64_kernel(long long* __restrict__ x, long long n,
                                                                          const long long* __restrict__ part) {
  long long i0 = blockIdx.x * (long long)SCAN_TILE + (long long)threadIdx.x * SCAN_ITEMS;
  long long v[SCAN_ITEMS];
  long long loc = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    v[k] = i0 + k < n ? x[i0 + k] : 0;
    loc += v[k];
  }
  long long tot;
  long long run = block_excl_scan(loc, &tot) + part[blockIdx.x];
  __shared__ long long res[SCAN_TILE + PLAN_THREADS];
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    run += v[k];
    res[threadIdx.x * (SCAN_ITEMS + 1) + k] = run;
  }
  __syncthreads();
  const long long t0 = blockIdx.x * (long long)SCAN_TILE;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    const int q = k * PLAN_THREADS + threadIdx.x;
    if (t0 + q < n) x[t0 + q] = res[q + q / SCAN_ITEMS];
  }
}

// Eq. 3: the lower boundary of task t is the first item whose inclusive
// cumulative cost reaches t * Zbar, Zbar = C_total / T, i.e. the first i with
// C_i * T >= t * C_total -- compared exactly in 128-bit integers.
__global__ void task_bounds_kernel(const long long* __restrict__ C, long long n_items,
                                   long long* __restrict__ task_start, int T) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t > T) return;
  if (t == 0) {
    task_start[0] = 0;
    return;
  }
  if (t == T) {
    task_start[T] = n_items;
    return;
  }
  const unsigned __int128 goal = (unsigned __int128)(unsigned long long)t * (unsigned long long)C[n_items - 1];
  long long lo = 0, hi = n_items;  // first i in [lo, hi) with C_i * T >= goal
  while (lo < hi) {
    long long mid = (lo + hi) >> 1;
    if ((unsigned __int128)(unsigned long long)C[mid] * (unsigned long long)T >= goal)
      hi = mid;
    else
      lo = mid + 1;
  }
  task_start[t] = lo;
}

// The paper's consecutive partition (CP, Section 4), kept for comparison with
// Eq. 3: task t takes the rows [t N / T, (t+1) N / T) of the plan's N nodes
// (graphs concatenated), i.e. the items from the first item of row t N / T on.
// Tasks only schedule work, so the output is the same as under Eq. 3.
__global__ void cp_bounds_kernel(const DevGraph* __restrict__ gs, int G, long long n_nodes, long long n_items,
                                 long long* __restrict__ task_start, int T) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t > T) return;
  if (t == T) {
    task_start[T] = n_items;
    return;
  }
  const long long N = (long long)((unsigned __int128)(unsigned long long)t * (unsigned long long)n_nodes /
                                  (unsigned long long)T);
  // graph g holds the nodes [pbase_g - g, pbase_g - g + n_g): its prefix has n_g + 1 entries
  int lo = 0, hi = G - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (gs[mid].pbase - mid <= N)
      lo = mid;
    else
      hi = mid - 1;
  }
  const DevGraph& g = gs[lo];
  const long long u = N - (g.pbase - lo);
  long long first = u < g.Hh ? heavy_items_before(u, g.n) : g.n_heavy + (u > g.H ? u - g.H : 0);
  if (first > g.n_items) first = g.n_items;
  task_start[t] = g.item_begin + first;
}

// Round robin (RRP, Section 4): task t holds the items t, t + T, t + 2T, ...;
// its table entry is its first item.
__global__ void rrp_bounds_kernel(long long n_items, long long* __restrict__ task_start, int T) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t > T) return;
  task_start[t] = t == T ? n_items : (t < n_items ? t : n_items);
}

long long scan_partials_needed(long long n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 1; }

void launch_costs_and_tasks(const DevGraph* d_graphs, int G, long long n_items, bool f64, const void* d_P,
                            long long* d_C, long long* d_partials, long long* d_task_start, int T, int* d_slot32,
                            int tiny_slots, int partition, long long n_nodes, cudaStream_t s) {
  if (n_items <= 0) {
    // empty plan: a single empty task
    cudaMemsetAsync(d_task_start, 0, 2 * sizeof(long long), s);
    return;
  }
  unsigned nb = (unsigned)((n_items + PLAN_THREADS - 1) / PLAN_THREADS);
  if (f64)
    costs_kernel<double><<<nb, PLAN_THREADS, 0, s>>>(d_graphs, G, n_items, (const double*)d_P, d_C, d_slot32,
                                                     tiny_slots);
  else
    costs_kernel<long long><<<nb, PLAN_THREADS, 0, s>>>(d_graphs, G, n_items, (const long long*)d_P, d_C, d_slot32,
                                                        tiny_slots);
  long long nt = (n_items + SCAN_TILE - 1) / SCAN_TILE;
  tile_reduce_i64_kernel<<<(unsigned)nt, PLAN_THREADS, 0, s>>>(d_C, n_items, d_partials);
  partials_scan_kernel<long long><<<1, 1024, 0, s>>>(d_partials, nt, nullptr);
  tile_incl_scan_i64_kernel<<<(unsigned)nt, PLAN_THREADS, 0, s>>>(d_C, n_items, d_partials);
  if (partition == CL_PART_RRP)
    rrp_bounds_kernel<<<(T + 1 + 255) / 256, 256, 0, s>>>(n_items, d_task_start, T);
  else if (partition == CL_PART_CP)
    cp_bounds_kernel<<<(T + 1 + 255) / 256, 256, 0, s>>>(d_graphs, G, n_nodes, n_items, d_task_start, T);
  else
    task_bounds_kernel<<<(T + 1 + 255) / 256, 256, 0, s>>>(d_C, n_items, d_task_start, T);
}

// --------------------------------------------------------------- count scan
__global__ void __launch_bounds__(PLAN_THREADS) count_reduce_kernel(const int* __restrict__ x, long long n,
                                                                    long long* __restrict__ part) {
  long long e0 = blockIdx.x * (long long)SCAN_TILE;
  long long acc = 0;
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    long long i = e0 + (long long)k * PLAN_THREADS + threadIdx.x;
    if (i < n) acc += x[i];
  }
  long long tot = block_reduce(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(PLAN_THREADS) count_scan_kernel(const int* __restrict__ x, long long n,
                                                                  const long long* __restrict__ part,
                                                                  long long* __restrict__ out, long long nt,
                                                                  const long long* base) {
  const long long b0 = base ? *base : 0;  // out[0] == *base when base == out: rewritten unchanged
  long long i0 = blockIdx.x * (long long)SCAN_TILE + (long long)threadIdx.x * SCAN_ITEMS;
  int v[SCAN_ITEMS];
  long long loc = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    v[k] = i0 + k < n ? x[i0 + k] : 0;
    loc += v[k];
  }
  long long tot;
  long long run = block_excl_scan(loc, &tot) + part[blockIdx.x] + b0;
  // results staged in shared memory (one pad word per thread's 8: 2-way bank
  // access) and written out coalesced
  __shared__ long long res[SCAN_TILE + PLAN_THREADS];
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    res[threadIdx.x * (SCAN_ITEMS + 1) + k] = run;
    run += v[k];
  }
  __syncthreads();
  const long long t0 = blockIdx.x * (long long)SCAN_TILE;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    const int q = k * PLAN_THREADS + threadIdx.x;
    if (t0 + q < n) out[t0 + q] = res[q + q / SCAN_ITEMS];
  }
  if (blockIdx.x == nt - 1 && threadIdx.x == 0) out[n] = part[blockIdx.x] + tot + b0;
}

void launch_count_scan(const int* d_counts, long long n, long long* d_offsets, long long* d_partials,
                       cudaStream_t s, const long long* d_base) {
  if (n <= 0) {
    if (!d_base) cudaMemsetAsync(d_offsets, 0, sizeof(long long), s);
    return;
  }
  long long nt = (n + SCAN_TILE - 1) / SCAN_TILE;
  count_reduce_kernel<<<(unsigned)nt, PLAN_THREADS, 0, s>>>(d_counts, n, d_partials);
  partials_scan_kernel<long long><<<1, 1024, 0, s>>>(d_partials, nt, nullptr);
  count_scan_kernel<<<(unsigned)nt, PLAN_THREADS, 0, s>>>(d_counts, n, d_partials, d_offsets, nt, d_base);
}

// One int64 from device memory to a (possibly host-mapped) address, by a
// kernel: unlike a copy-engine transfer it does not queue behind large
// host copies in flight.
__global__ void copy_i64_kernel(const long long* __restrict__ src, long long* dst) { *dst = *src; }

void launch_copy_i64(const long long* d_src, long long* dst, cudaStream_t s) {
  copy_i64_kernel<<<1, 1, 0, s>>>(d_src, dst);
}

// The end of a piece of consecutive items whose edges fit in `cap`: the last
// b in (a, ie] with offsets[b] - offsets[a] <= cap (a itself when item a
// alone holds more than cap edges), by binary search; stored into *out.
__global__ void piece_end_kernel(const long long* __restrict__ offsets, long long a, long long ie, long long cap,
                                 long long* __restrict__ out) {
  const long long base = offsets[a];
  long long lo = a, hi = ie;  // invariant: offsets[lo] - base <= cap
  while (lo < hi) {
    const long long mid = lo + (hi - lo + 1) / 2;
    if (offsets[mid] - base <= cap)
      lo = mid;
    else
      hi = mid - 1;
  }
  *out = lo;
}

void launch_piece_end(const long long* d_offsets, long long a, long long ie, long long cap, long long* dst,
                      cudaStream_t s) {
  piece_end_kernel<<<1, 1, 0, s>>>(d_offsets, a, ie, cap, dst);
}

// Successive piece ends by binary search, one thread (a few dozen searches):
// out[0] = pieces k, out[1] = offsets[ib], out[2 + 2j] = end item of piece j,
// out[3 + 2j] = offsets at that end.
__global__ void pieces_kernel(const long long* __restrict__ offsets, long long ib, long long ie, long long cap,
                              long long* __restrict__ out, int max_pieces) {
  long long a = ib;
  int k = 0;
  out[1] = offsets[ib];
  while (a < ie && k < max_pieces) {
    const long long base = offsets[a];
    long long lo = a, hi = ie;
    while (lo < hi) {
      const long long mid = lo + (hi - lo + 1) / 2;
      if (offsets[mid] - base <= cap)
        lo = mid;
      else
        hi = mid - 1;
    }
    if (lo == a) break;  // item a alone holds more than cap edges
    out[2 + 2 * k] = lo;
    out[3 + 2 * k] = offsets[lo];
    ++k;
    a = lo;
  }
  out[0] = k;
}

void launch_pieces(const long long* d_offsets, long long ib, long long ie, long long cap, long long* dst,
                   int max_pieces, cudaStream_t s) {
  pieces_kernel<<<1, 1, 0, s>>>(d_offsets, ib, ie, cap, dst, max_pieces);
}

__global__ void gather_task_slots_kernel(const long long* __restrict__ slot_base,
                                         const long long* __restrict__ task_start, int T,
                                         long long* __restrict__ out) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t <= T) out[t] = slot_base[task_start[t]];
}

void launch_gather_task_slots(const long long* d_slot_base, const long long* d_task_start, int T, long long* dst,
                              cudaStream_t s) {
  gather_task_slots_kernel<<<(unsigned)((T + 1 + 255) / 256), 256, 0, s>>>(d_slot_base, d_task_start, T, dst);
}

}  // namespace cl
