// cl_internal.cuh -- device-side plan layout shared by the library's kernels.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>

#include "../../include/cl.h"

namespace cl {

constexpr int SEG_LOG2 = 16;  // heavy rows are cut at absolute multiples of 2^16 of v
constexpr unsigned LIGHT_SEG = 0xFFFFFFFFu;
constexpr unsigned FULL_MASK = 0xFFFFFFFFu;

// Per-graph constants of -ln(1 - Q/S): zS = clz(S), sh = max(0, 41 - zS)
// (so S >> sh has at most 23 bits), cS = 64 / (S >> sh) in float, the
// series bound Ssmall = S >> 12 (p < 2^-12 below it) and 1/S as a
// float-float pair (hi = 1/S rounded to float, lo = the rounded remainder,
// formed from the exact integer 2^k - m S).
struct LpConst {
  int zS, sh;
  float cS;
  float iS_hi, iS_lo;
  unsigned long long Ssmall;
};
__host__ __device__ inline LpConst lp_const(unsigned long long S) {
#ifdef __CUDA_ARCH__
  const int z = __clzll(S);
#else
  const int z = S ? __builtin_clzll(S) : 64;
#endif
  const int sh = z < 41 ? 41 - z : 0;
  LpConst c{z, sh, (float)(64.0 / (double)(S >> sh)), 0.0f, 0.0f, S >> 12};
  if (S > 0) {
    const float hi = (float)(1.0 / (double)S);
    int ex;
    const double m = frexp((double)hi, &ex);  // hi = m 2^ex, m in [1/2, 1)
    const long long M = (long long)ldexp(m, 24);
    const int k = 24 - ex;  // hi = M 2^-k, 2^k > M S since hi ~ 1/S
    // remainder 1 - hi S = (2^k - M S) 2^-k, exact in 128-bit integers (k < 90)
    const __int128 num = ((__int128)1 << k) - (__int128)M * (__int128)S;
    c.iS_hi = hi;
    c.iS_lo = (float)(ldexp((double)num, -k) / (double)S);
  }
  return c;
}

// Per-graph constants of -ln(1 - Q/S) for double weights: S's 53-bit significand
// s_m and biased exponent s_e, cS = 64 / (s_m >> 30) in float, 1/S as a float-float
// pair, and the series bound S_small = S 2^-12.
struct LpConstD {
  unsigned long long s_m;
  int s_e;
  float cS;
  float iS_hi, iS_lo;
  double S_small;
};
inline LpConstD lp_const_d(double S) {
  LpConstD c{0ull, 0, 0.0f, 0.0f, 0.0f, 0.0};
  if (!(S > 0.0) || !std::isfinite(S)) return c;
  unsigned long long b;
  std::memcpy(&b, &S, sizeof b);
  c.s_e = (int)((b >> 52) & 0x7FF);
  c.s_m = (b & ((1ull << 52) - 1)) | (1ull << 52);
  c.cS = (float)(64.0 / (double)(c.s_m >> 30));
  const long double iS = 1.0L / (long double)S;
  c.iS_hi = (float)iS;
  c.iS_lo = (float)(iS - (long double)c.iS_hi);
  c.S_small = std::ldexp(S, -12);
  return c;
}

// The same constants formed on the device (diagnostics; 1/S from a double division,
// within 2^-53 of the host's).
__device__ inline LpConstD lp_const_d_dev(double S) {
  LpConstD c{0ull, 0, 0.0f, 0.0f, 0.0f, 0.0};
  const unsigned long long b = (unsigned long long)__double_as_longlong(S);
  c.s_e = (int)((b >> 52) & 0x7FF);
  c.s_m = (b & ((1ull << 52) - 1)) | (1ull << 52);
  c.cS = (float)(64.0 / (double)(c.s_m >> 30));
  const double iS = 1.0 / S;
  c.iS_hi = (float)iS;
  c.iS_lo = (float)(iS - (double)c.iS_hi);
  c.S_small = S * 0x1p-12;
  return c;
}

// One graph of a plan, as the kernels see it (lives in the plan workspace).
struct DevGraph {
  const void* w;          // device weights, sorted non-increasing
  long long n;            // nodes
  long long S_i;          // exact integer sum (integer weights)
  double S_d;             // weight sum as a double
  unsigned key0, key1;    // Philox key = seed
  unsigned rk[20];        // Philox round keys of that key (key + r * Weyl constants)
  long long H;            // heavy rows (w_u >= heavy_w): a prefix
  long long Hh;           // heavy rows that have items: min(H, n - 1)
  long long n_heavy;      // items of the heavy rows
  long long item_begin;   // first global item
  long long n_items;      // items of this graph
  long long pbase;        // offset of this graph's weight prefix (n + 1 entries)
  int wtype;              // cl_wtype
  LpConst lp;             // constants of -ln(1 - Q/S) (integer weights)
  LpConstD lpd;           // the same for double weights
  float invS_f;           // 1 / S in single precision (costs only)
  long long bbase;        // offset of this graph's entries in the uniform-block table (integer weights)
  const unsigned long long* blkp;  // this graph's entries of that table (set by cl_plan_build)
};

// Per-graph results of the analysis kernel (scratch of cl_plan_create).
struct GraphAnalysis {
  unsigned long long S_i;       // integer sum
  unsigned long long H;         // count of w >= heavy_w
  unsigned int flags;           // bit 0: unsorted, bit 1: negative / non-finite
  unsigned int pad_;
  double S_d;                   // correctly rounded sum (double weights)
  double S2;                    // sum of w^2 (sizes the staging pool only)
};

// Items of heavy rows [0, U): sum_{u<U} K_u, K_u = N1 - ((u+1) >> 16) + 1,
// N1 = (n-1) >> 16; uses sum_{x=0}^{U} floor(x / 2^16) in closed form.
__host__ __device__ __forceinline__ long long heavy_items_before(long long U, long long n) {
  const long long B = 1ll << SEG_LOG2;
  long long N1 = (n - 1) >> SEG_LOG2;
  long long q = U >> SEG_LOG2;
  long long F = B * q * (q - 1) / 2 + q * (U - q * B + 1);
  return U * (N1 + 1) - F;
}

// Position of a graph's local item: source row u and segment field (LIGHT_SEG
// for a light row).  Heavy row u has the segments (u + 1) >> 16 .. N1.
struct ItemPos {
  long long local;
  unsigned u, seg;
};

// By bisection over the heavy rows (for an item with no known neighbour).
__device__ __forceinline__ ItemPos item_pos(const DevGraph& g, long long local) {
  if (local >= g.n_heavy) return ItemPos{local, (unsigned)(g.H + (local - g.n_heavy)), LIGHT_SEG};
  long long lo = 0, hi = g.Hh - 1;  // last r with heavy_items_before(r) <= local
  while (lo < hi) {
    long long mid = (lo + hi + 1) >> 1;
    if (heavy_items_before(mid, g.n) <= local)
      lo = mid;
    else
      hi = mid - 1;
  }
  const long long k = ((lo + 1) >> SEG_LOG2) + (local - heavy_items_before(lo, g.n));
  return ItemPos{local, (unsigned)lo, (unsigned)k};
}

// Integer <-> float conversions run on the FP64-class pipe of this GPU (1/75 of
// the FP32 rate); the per-item plan kernels build them from bit patterns
// instead (for 0 <= x < 2^16 the float with bits 0x4B000000 | x is 2^23 + x).
__device__ __forceinline__ float u16_to_f(unsigned x) { return __int_as_float(0x4B000000 | x) - 8388608.0f; }
// float(x), correctly rounded
__device__ __forceinline__ float u32_to_f(unsigned x) { return fmaf(u16_to_f(x >> 16), 65536.0f, u16_to_f(x & 0xFFFFu)); }
// float(v) for 0 <= v < 2^64 to within an ulp
__device__ __forceinline__ float u64_to_f(unsigned long long v) {
  return fmaf(u32_to_f((unsigned)(v >> 32)), 4294967296.0f, u32_to_f((unsigned)v));
}
// floor(f) for 0 <= f < 2^62
__device__ __forceinline__ long long f_floor_to_ll(float f) {
  if (f < 8388608.0f) return (long long)(__float_as_int(__fadd_rd(f, 8388608.0f)) - 0x4B000000);
  const unsigned b = __float_as_uint(f);  // an integer: the significand shifted left
  return (long long)((b & 0x7FFFFFu) | 0x800000u) << ((b >> 23) - 150u);
}
// ceil(f) for 0 <= f < 2^30
__device__ __forceinline__ int f_ceil_to_i(float f) {
  if (f < 8388608.0f) return __float_as_int(__fadd_ru(f, 8388608.0f)) - 0x4B000000;
  const unsigned b = __float_as_uint(f);
  return (int)(((b & 0x7FFFFFu) | 0x800000u) << ((b >> 23) - 150u));
}

// Same as item_pos, for the per-item plan kernels: rows u with u + 1 < 2^16
// all have the K0 = N1 + 1 segments 0 .. N1, so an item among their
// K0 * min(Hh, 2^16 - 1) items is row local / K0, segment local % K0 (a float
// quotient corrected to the exact one) with no bisection.  (The samplers keep
// item_pos: they call it once per task, and the extra code costs registers.)
__device__ __forceinline__ ItemPos item_pos_direct(const DevGraph& g, long long local) {
  const long long K0 = ((g.n - 1) >> SEG_LOG2) + 1;
  const long long U0 = g.Hh < (1ll << SEG_LOG2) - 1 ? g.Hh : (1ll << SEG_LOG2) - 1;
  if (local >= U0 * K0) return item_pos(g, local);
  long long u = f_floor_to_ll(__fmul_rz(u64_to_f((unsigned long long)local), __frcp_rn(u32_to_f((unsigned)K0))));
  long long r = local - u * K0;
  while (r < 0) {
    --u;
    r += K0;
  }
  while (r >= K0) {
    ++u;
    r -= K0;
  }
  return ItemPos{local, (unsigned)u, (unsigned)r};
}

// The position d >= 0 items after p (p.local + d an item of g): segments
// advance within the row, and a step past the row's last segment moves to the
// first segment of the next row -- one loop turn per row crossed.
__device__ __forceinline__ ItemPos item_advance(const DevGraph& g, ItemPos p, long long d) {
  const long long t = p.local + d;
  if (t >= g.n_heavy) return ItemPos{t, (unsigned)(g.H + (t - g.n_heavy)), LIGHT_SEG};
  const long long N1 = (g.n - 1) >> SEG_LOG2;
  unsigned u = p.u;
  long long k = (long long)p.seg + d;
  while (k > N1) {
    k -= N1 + 1;
    ++u;
    k += (long long)((u + 1) >> SEG_LOG2);
  }
  return ItemPos{t, u, (unsigned)k};
}

// Candidate range [j0, end) of the item at p.
__device__ __forceinline__ void pos_bounds(const DevGraph& g, ItemPos p, unsigned& j0, unsigned& end) {
  if (p.seg == LIGHT_SEG) {
    j0 = p.u + 1;
    end = (unsigned)g.n;
    return;
  }
  const long long s0 = (long long)p.seg << SEG_LOG2, s1 = s0 + (1ll << SEG_LOG2);
  j0 = (unsigned)(s0 > (long long)p.u + 1 ? s0 : (long long)p.u + 1);
  end = (unsigned)(s1 < g.n ? s1 : g.n);
}

// Bounds of a graph's local item: source row u, segment field, [j0, end).
__device__ __forceinline__ void item_bounds(const DevGraph& g, long long local, unsigned& u, unsigned& seg,
                                            unsigned& j0, unsigned& end) {
  const ItemPos p = item_pos_direct(g, local);
  u = p.u;
  seg = p.seg;
  pos_bounds(g, p, j0, end);
}

// Walk a cursor (graph gi, position p of the global item it stands on) d items
// forward across graph boundaries; the result must be an item of the plan.
__device__ __forceinline__ void cursor_advance(const DevGraph* gs, int& gi, ItemPos& p, long long d) {
  while (p.local + d >= gs[gi].n_items) {  // past this graph: continue at local 0 of the next
    d -= gs[gi].n_items - p.local;
    ++gi;
    p = gs[gi].n_heavy > 0 ? ItemPos{0, 0u, 0u} : ItemPos{0, (unsigned)gs[gi].H, LIGHT_SEG};
  }
  p = item_advance(gs[gi], p, d);
}

// Graph owning a global item (binary search over item_begin; G is small).
__device__ __forceinline__ int graph_of_item(const DevGraph* gs, int G, long long item) {
  int lo = 0, hi = G - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (gs[mid].item_begin <= item)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Kernel-facing view of a built plan.
// uniform-block table of integer-weight plans (see blocks_kernel)
constexpr int BLK_SHIFT = 12;
constexpr unsigned long long BLK_MIXED = ~0ull;  // never (w << 32) | end, since w < 2^31

struct DevPlan {
  const DevGraph* graphs;
  int G;
  long long n_items;
  const long long* task_start;  // T + 1 entries
  int T;
  unsigned* task_ctr;           // dynamic task counter (reset before each sampler launch)
  int* err;                     // device error word (first error wins)
  unsigned long long* stats;    // iterations, fallbacks, ties
  unsigned* pool;               // staging pool of destination nodes
  unsigned long long pool_cap;  // its entries: a slot ending past them counts as size 0 (never staged)
  const long long* slot_base;   // per item: first pool entry of its slot (n_items + 1 entries)
  unsigned long long pool_entries;  // allocated pool entries (pool_cap may be a window's lower limit)
  long long pool_shift;         // item i's slot sits at pool entry slot_base[i] - pool_shift (0 except
                                // for the windows of cl_generate_stream, which reuse the pool)
  int* overflow;                // set when an item outgrew its slot
  long long* ovf_list;          // items that outgrew their slot (first ovf_cap of them)
  unsigned* ovf_count;
  unsigned ovf_cap;
  int wf64;                     // the plan's weights are doubles
  const unsigned long long* blk;  // integer weights: uniform-block table (BLK_MIXED or (w << 32) | run end)
  int rrp;                      // round-robin partition: task t holds the items t, t + T, t + 2T, ...
  unsigned long long* task_ns;  // nullable: per task, the global timer (ns) when a warp took it and
                                // when that warp took its next task or finished (count passes)
  int copy_chunk;               // items per claim of the copy kernel (a multiple of 32)
};

// Staging slot of item i in entries (0: the item is never staged, its slot
// would end past the pool).
__device__ __forceinline__ unsigned slot_size(const DevPlan& P, long long i) {
  const long long b = P.slot_base[i + 1];
  return (unsigned long long)(b - P.pool_shift) <= P.pool_cap ? (unsigned)(b - P.slot_base[i]) : 0u;
}

// ---- launchers implemented in plan.cu / sample.cu / diag.cu ----
constexpr int ANALYZE_CHUNK_HOST = 4096;  // weights per analysis block (matches plan.cu)
constexpr int SCAN_TILE_HOST = 2048;      // elements per scan tile (matches plan.cu)
void launch_analyze(const DevGraph* d_graphs, const long long* d_blk_begin, int G, long long nblocks,
                    const double* d_heavy_w, GraphAnalysis* d_out, unsigned long long* d_bins, bool f64,
                    cudaStream_t s);
void launch_f64_sum_finalize(int G, const unsigned long long* d_bins, GraphAnalysis* d_out, cudaStream_t s);
size_t f64_bins_bytes(int G);

// Weight prefix over the graphs' concatenated weights (int64 for integer weights, double
// for double weights); graph g's entries start at pbase_g.
void launch_weight_prefix(const DevGraph* d_graphs, const long long* d_tile_graph_begin, int G, long long ntiles,
                          bool f64, void* d_P, void* d_partials, cudaStream_t s);
// Run table of integer weights (see plan.cu).
void launch_blocks(const DevGraph* d_graphs, int G, long long nblk, unsigned long long* d_blk, cudaStream_t s);
// Item costs (fixed point, 1/16 edge), their exact inclusive prefix C in place and the
// task boundaries of Eq. 3; when d_slot32 is given, also every item's staging slot size.
void launch_costs_and_tasks(const DevGraph* d_graphs, int G, long long n_items, bool f64, const void* d_P,
                            long long* d_C, long long* d_partials, long long* d_task_start, int T, int* d_slot32,
                            int tiny_slots, int partition, long long n_nodes, cudaStream_t s);
// Exclusive int32 -> int64 scan with the total at out[n]; with d_base, every
// output is offset by *d_base (read on the device: a scan of a later range of
// items continues from the total of the earlier ones, with no host round trip).
void launch_count_scan(const int* d_counts, long long n, long long* d_offsets, long long* d_partials,
                       cudaStream_t s, const long long* d_base = nullptr);
long long scan_partials_needed(long long n);
void launch_copy_i64(const long long* d_src, long long* dst, cudaStream_t s);
// *dst = the last b in [a, ie] with d_offsets[b] - d_offsets[a] <= cap
void launch_piece_end(const long long* d_offsets, long long a, long long ie, long long cap, long long* dst,
                      cudaStream_t s);
// Cuts items [ib, ie) into consecutive pieces of at most cap edges: dst[0] = number of
// pieces k (at most max_pieces; fewer when the items run out or one item alone exceeds
// cap), dst[1] = d_offsets[ib], dst[2 + 2j] = the end item of piece j (piece j starts
// where piece j - 1 ends), dst[3 + 2j] = d_offsets at that end.
void launch_pieces(const long long* d_offsets, long long ib, long long ie, long long cap, long long* dst,
                   int max_pieces, cudaStream_t s);
// dst[t] = slot_base[task_start[t]], t = 0..T (staging slot bases at the task boundaries)
void launch_gather_task_slots(const long long* d_slot_base, const long long* d_task_start, int T, long long* dst,
                              cudaStream_t s);

// Items [ib, ie) of a sampling launch; tasks are taken from t0 on (the first
// task that reaches ib), and edges[0] of an emitting launch holds the first
// edge of item ob (ob = ib: the range's own array; ob = 0: absolute offsets).
struct SampleRange {
  long long ib, ie;
  int t0;
  long long ob;
};

// `single`: host copy of the plan's only graph (G == 1), passed to the kernels by value; else nullptr
void launch_count(const DevPlan& P, const DevGraph* single, int* d_counts, bool stage, int block, int grid,
                  cudaStream_t s);
void launch_count_range(const DevPlan& P, const DevGraph* single, int* d_counts, bool stage, const SampleRange& r,
                        int block, int grid, cudaStream_t s);
// copy_grid > 0 caps the copy kernel's grid (to leave SMs to a concurrent launch)
void launch_emit(const DevPlan& P, const DevGraph* single, const long long* d_offsets, const SampleRange& r,
                 int etype, void* d_edges, long long capacity, bool staged, int block, int grid, int copy_grid,
                 cudaStream_t s);
void launch_graph_offsets(const DevGraph* d_graphs, int G, const long long* d_offsets, long long n_items,
                          long long* d_graph_offsets, long long capacity, int* d_status, cudaStream_t s);
int sampler_max_blocks_per_sm(int block, bool emit, int etype);

}  // namespace cl
