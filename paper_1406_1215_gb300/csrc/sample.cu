// sample.cu -- the count and emit passes: Algorithm 1 (Create-Edges) run per
// item by one lane each.
//
// Scheduling (Section 4 analogue): a persistent grid; each warp pulls the
// next equal-cost task (Eq. 3) from a counter; inside the warp every lane
// runs one item's skip loop and, when its item ends, takes the task's next
// item (warp-ballot refill), so lanes stay busy while item lengths vary.
// Which lane or warp runs an item never changes its output: the random
// stream is keyed by (seed; draw, segment, u).
//
// Per loop iteration of an item (source u, position j, end, Q_prev):
//   block = Philox4x32-10(key, (t, seg, u, 0)), t += 1
//   delta = 0 if Q_prev = S (p = 1), else floor(L_r / L_p) with
//           L_r = -ln(r_s), L_p = -ln(1 - Q_prev/S)    (exact real floor)
//   stop if delta >= end - j;  v = j + delta
//   Q_v = min(w_u w_v, S); accept iff r_a Q_prev < Q_v (exact, 128-bit)
//   Q_prev = Q_v (recompute L_p if it changed); j = v + 1
#include <cuda_runtime.h>

#include "cl_internal.cuh"
#include "clmath.cuh"
#include "philox.cuh"

namespace cl {

constexpr int SAMPLER_THREADS = 256;

__device__ __forceinline__ void set_error(int* err, int code) { atomicCAS(err, 0, code); }

// Exact test (2k+1) * Qprev < 2^53 * Qv for 0 <= Qv < Qprev < 2^53.
__device__ __forceinline__ bool accept_i(unsigned long long k, unsigned long long Qprev, unsigned long long Qv) {
  unsigned long long a = 2ull * k + 1ull;
  unsigned long long lo = a * Qprev, hi = __umul64hi(a, Qprev);
  unsigned long long rhi = Qv >> 11, rlo = Qv << 53;
  return hi < rhi || (hi == rhi && lo < rlo);
}

template <bool EMIT, typename E>
__global__ void __launch_bounds__(SAMPLER_THREADS) sample_kernel(DevPlan P, long long ib, long long ie,
                                                                 const long long* __restrict__ offsets,
                                                                 E* __restrict__ edges, long long capacity,
                                                                 int* __restrict__ counts) {
  const int lane = threadIdx.x & 31;
  const unsigned lanemask_lt = (1u << lane) - 1u;
  long long off_base = 0;
  if (EMIT) {
    off_base = offsets[ib];
    if (offsets[ie] - off_base > capacity) {
      if (blockIdx.x == 0 && threadIdx.x == 0) set_error(P.err, CL_ERR_CAPACITY);
      return;  // nothing is written when the range does not fit
    }
  }
  // warp-uniform task cursor
  long long next = 0, tend = 0;
  bool tasks_left = true;
  // lane state
  bool have = false;
  long long item = 0, obase = 0;
  const int* w = nullptr;
  unsigned u = 0, seg = 0, j = 0, end = 0, t = 0, k = 0, key0 = 0, key1 = 0;
  unsigned long long S = 0, Qprev = 0;
  int wu = 0;
  ff Lp{0.f, 0.f};
  unsigned long long n_iter = 0, n_fb = 0, n_tie = 0;

  while (true) {
    // ---- refill lanes that have no item
    unsigned need = __ballot_sync(FULL_MASK, !have);
    while (need) {
      if (next >= tend) {
        if (!tasks_left) break;
        unsigned tix = 0;
        if (lane == 0) tix = atomicAdd(P.task_ctr, 1u);
        tix = __shfl_sync(FULL_MASK, tix, 0);
        if (tix >= (unsigned)P.T) {
          tasks_left = false;
          break;
        }
        long long a = P.task_start[tix], b = P.task_start[tix + 1];
        next = a > ib ? a : ib;
        tend = b < ie ? b : ie;
        continue;
      }
      long long avail = tend - next;
      int rank = __popc(need & lanemask_lt);
      int taken = __popc(need);
      if (!have && rank < avail) {
        item = next + rank;
        // ---- item set-up
        int gi = P.G == 1 ? 0 : graph_of_item(P.graphs, P.G, item);
        const DevGraph& g = P.graphs[gi];
        unsigned j0;
        item_bounds(g, item - g.item_begin, u, seg, j0, end);
        w = (const int*)g.w;
        S = (unsigned long long)g.S_i;
        key0 = g.key0;
        key1 = g.key1;
        wu = __ldg(&w[u]);
        j = j0;
        t = 0;
        k = 0;
        unsigned long long q = (unsigned long long)((long long)wu * (long long)__ldg(&w[j0]));
        Qprev = q < S ? q : S;
        if (EMIT) obase = offsets[item] - off_base;
        if (Qprev == 0 || j0 >= end) {
          if (!EMIT) counts[item] = 0;  // empty item: no draw at all
        } else {
          have = true;
          if (Qprev < S) Lp = ff_neglog_ratio(S - Qprev, S);
        }
      }
      next += taken < avail ? taken : avail;
      need = __ballot_sync(FULL_MASK, !have);  // empty items and unserved lanes retry at once
    }
    if (!__any_sync(FULL_MASK, have)) {
      if (!tasks_left) break;
      continue;
    }
    // ---- one iteration of the skip loop
    if (have) {
      u32x4 b = philox4x32_10(u32x4{t, seg, u, 0u}, key0, key1);
      ++t;
      ++n_iter;
      long long R = (long long)end - (long long)j;
      long long delta = 0;
      if (Qprev != S) {
        unsigned long long Ar = 2ull * grid52(b.x, b.y) + 1ull;
        ff Lr = ff_neglog_ratio(Ar, 1ull << 53);
        delta = floor_decide_ff(ff_div(Lr, Lp), R);
        if (delta == SKIP_UNDECIDED) {
          bool tie;
          delta = skip_fallback_dd(Ar, S - Qprev, S, R, &tie);
          ++n_fb;
          n_tie += tie;
        }
      }
      bool done = false;
      if (delta >= R) {
        done = true;
      } else {
        unsigned v = j + (unsigned)delta;
        int wv = __ldg(&w[v]);
        unsigned long long q = (unsigned long long)((long long)wu * (long long)wv);
        unsigned long long Qv = q < S ? q : S;
        bool acc = (Qv == Qprev) || accept_i(grid52(b.z, b.w), Qprev, Qv);
        if (acc) {
          if (EMIT) {
            long long pos = obase + k;
            if (pos < capacity) {
              E e;
              e.x = u;
              e.y = v;
              edges[pos] = e;
            }
          }
          ++k;
        }
        if (Qv != Qprev) {
          Qprev = Qv;
          if (Qv == 0)
            done = true;
          else if (Qv < S)
            Lp = ff_neglog_ratio(S - Qv, S);
        }
        j = v + 1;
        if (j >= end) done = true;
      }
      if (done) {
        if (EMIT) {
          long long expect = offsets[item + 1] - offsets[item];
          if ((long long)k != expect) set_error(P.err, CL_ERR_DEVICE);
        } else {
          counts[item] = (int)k;
        }
        have = false;
      }
    }
  }
  if (!EMIT) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      n_iter += __shfl_xor_sync(FULL_MASK, n_iter, o);
      n_fb += __shfl_xor_sync(FULL_MASK, n_fb, o);
      n_tie += __shfl_xor_sync(FULL_MASK, n_tie, o);
    }
    if (lane == 0) {
      atomicAdd(&P.stats[0], n_iter);
      if (n_fb) atomicAdd(&P.stats[1], n_fb);
      if (n_tie) atomicAdd(&P.stats[2], n_tie);
    }
  }
}

int sampler_max_blocks_per_sm(int block, bool emit, int etype) {
  int nb = 0;
  if (!emit)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sample_kernel<false, int2>, block, 0);
  else if (etype == CL_E_I32)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sample_kernel<true, int2>, block, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sample_kernel<true, longlong2>, block, 0);
  return nb;
}

void launch_count(const DevPlan& P, int* d_counts, int block, int grid, cudaStream_t s) {
  cudaMemsetAsync(P.task_ctr, 0, sizeof(unsigned), s);
  sample_kernel<false, int2><<<grid, block, 0, s>>>(P, 0, P.n_items, nullptr, nullptr, 0, d_counts);
}

void launch_emit(const DevPlan& P, const long long* d_offsets, long long ib, long long ie, int etype, void* d_edges,
                 long long capacity, int block, int grid, cudaStream_t s) {
  cudaMemsetAsync(P.task_ctr, 0, sizeof(unsigned), s);
  if (etype == CL_E_I32)
    sample_kernel<true, int2><<<grid, block, 0, s>>>(P, ib, ie, d_offsets, (int2*)d_edges, capacity, nullptr);
  else
    sample_kernel<true, longlong2>
        <<<grid, block, 0, s>>>(P, ib, ie, d_offsets, (longlong2*)d_edges, capacity, nullptr);
}

// Per-graph edge offsets of a batch and the capacity status.
__global__ void graph_offsets_kernel(const DevGraph* __restrict__ gs, int G, const long long* __restrict__ offsets,
                                     long long n_items, long long* __restrict__ goff, long long capacity,
                                     int* __restrict__ status) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < G) goff[g] = offsets[gs[g].item_begin];
  if (g == 0) {
    goff[G] = offsets[n_items];
    *status = offsets[n_items] > capacity ? CL_ERR_CAPACITY : CL_OK;
  }
}

void launch_graph_offsets(const DevGraph* d_graphs, int G, const long long* d_offsets, long long n_items,
                          long long* d_graph_offsets, long long capacity, int* d_status, cudaStream_t s) {
  graph_offsets_kernel<<<(G + 255) / 256, 256, 0, s>>>(d_graphs, G, d_offsets, n_items, d_graph_offsets, capacity,
                                                      d_status);
}

}  // namespace cl
