// sample.cu -- the sampling passes: Algorithm 1 (Create-Edges) run per item
// by one lane each, and the copy of staged destinations into the edge list.
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
// A new item's first position is handled by the same weight-lookup and
// L_p stages as a candidate (Q_prev = Q(j0)), so set-up shares the code of
// the loop body instead of running as a separate divergent branch; when that
// position is capped (p = 1), the whole capped run is taken at once
// (capped_run: the same edges and draws as one iteration per position).
//
// Modes: COUNT writes per-item edge counts; STAGE also writes each item's
// destinations, in order, into the item's slot of a staging pool (slot sizes
// come from the plan: expected edges + 6 sd + 6, in whole 32-byte sectors;
// an item that outgrows its slot is regenerated by EMIT).  Each accepted
// destination is stored at once: a lane's consecutive 4-byte stores complete a
// sector within a few passes, in L2 (collecting 8 in shared memory to write
// whole sectors cost a branch per pass and was slower: 58.4 against 55.8 ms);
// EMIT regenerates items and writes (u, v) pairs.  The copy kernel turns
// staged destinations into (u, v) pairs at the scanned offsets, so a count
// + copy does the sampling arithmetic once.
#include <cuda_runtime.h>

#include "cl_internal.cuh"
#include "clmath.cuh"
#include "philox.cuh"

namespace cl {

constexpr int SAMPLER_THREADS = 256;
// resident blocks per SM the sampler is compiled for: 3 x 256 threads leave 85 registers
// per thread, enough for the loop state without spills (4 blocks: 64 registers, spills)
constexpr int SAMPLER_MIN_BLOCKS = 3;
constexpr unsigned GROUP = 8;  // entries per whole-sector store of a capped run: one 32-byte sector

enum { MODE_COUNT = 0, MODE_STAGE = 1, MODE_EMIT = 2 };

__device__ __forceinline__ void set_error(int* err, int code) { atomicCAS(err, 0, code); }

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Exact test (2k+1) * Qprev < 2^53 * Qv for 0 <= Qv < Qprev < 2^53.
__device__ __forceinline__ bool accept_i(unsigned long long k, unsigned long long Qprev, unsigned long long Qv) {
  unsigned long long a = 2ull * k + 1ull;
  unsigned long long lo = a * Qprev, hi = __umul64hi(a, Qprev);
  unsigned long long rhi = Qv >> 11, rlo = Qv << 53;
  return hi < rhi || (hi == rhi && lo < rlo);
}

// Software pipelining: a lane issues the load of its candidate's weight and,
// while it is in flight, computes the Philox block and -ln r_s of its next
// draw; the candidate is then accepted or rejected with the draw it was made
// with.  Single-graph plans read the graph's parameters from the kernel
// parameter (constant bank) instead of per-lane registers.
// Weight types: integer weights work with exact 64-bit products and float-float
// logarithms; double weights (calibrated sequences) with the rounded product
// capped at S, the double logarithm for L_p and the exact sign of a fused
// multiply-add for the acceptance.
template <bool WF>
struct Wt;
template <>
struct Wt<false> {
  using w_t = int;
  using q_t = unsigned long long;
  using lp_t = ff;
  static __device__ __forceinline__ q_t S(const DevGraph& g) { return (q_t)g.S_i; }
  static __device__ __forceinline__ q_t Q(w_t a, w_t b, q_t S) {
    q_t q = (q_t)((long long)a * (long long)b);
    return q < S ? q : S;
  }
  static __device__ __forceinline__ lp_t Lp(q_t Q, q_t S, const DevGraph& g) { return ff_neglog1m(Q, S, g.lp); }
  static __device__ __forceinline__ int skip1(ff Lr, lp_t Lp, int R) { return floor_decide_ff32(ff_div(Lr, Lp), R); }
  static __device__ __forceinline__ long long skip2(unsigned long long Ar, q_t Q, q_t S, long long R, bool* tie) {
    return skip_fallback_dd(Ar, S - Q, S, R, tie);
  }
  static __device__ __forceinline__ bool accept(unsigned long long k, q_t Qprev, q_t Qv) {
    return accept_i(k, Qprev, Qv);
  }
};
template <>
struct Wt<true> {
  using w_t = double;
  using q_t = double;
  using lp_t = ff;
  static __device__ __forceinline__ q_t S(const DevGraph& g) { return g.S_d; }
  static __device__ __forceinline__ q_t Q(w_t a, w_t b, q_t S) {
    q_t q = a * b;
    return q >= S ? S : q;  // capped iff the rounded product reaches S
  }
  // float-float from the doubles (tier 1 as for integer weights; the double-double tier
  // below decides what the 2^-40 window leaves open)
  static __device__ __forceinline__ lp_t Lp(q_t Q, q_t S, const DevGraph& g) { return ff_neglog1m_d(Q, S, g.lpd); }
  static __device__ __forceinline__ int skip1(ff Lr, lp_t Lp, int R) { return floor_decide_ff32(ff_div(Lr, Lp), R); }
  static __device__ __forceinline__ long long skip2(unsigned long long Ar, q_t Q, q_t S, long long R, bool* tie) {
    return skip_fallback_dd_f64(Ar, Q, S, R, tie);
  }
  static __device__ __forceinline__ bool accept(unsigned long long k, q_t Qprev, q_t Qv) {
    double r = (double)(2ull * k + 1ull) * 0x1p-53;  // exact
    return fma(r, Qprev, -Qv) < 0.0;                  // the sign of r Qprev - Qv, exactly
  }
};

// Philox draws of a lane's item: with the precomputed round keys of a
// single-graph plan (kernel parameter, so the key schedule costs no
// instruction), or from the seed of the lane's graph in a batch.  (Keeping the
// item-constant part of the first two rounds per lane saves 2 of the 20 wide
// multiplies but costs the registers that the loop needs: measured slower.)
template <bool SINGLE>
struct Keys;
template <>
struct Keys<true> {
  __device__ __forceinline__ u32x4 draw(const DevGraph& g, unsigned t, unsigned seg, unsigned u) const {
    return philox4x32_10_rk(u32x4{t, seg, u, 0u}, g.rk);
  }
};
template <>
struct Keys<false> {
  unsigned k0, k1;
  __device__ __forceinline__ u32x4 draw(const DevGraph&, unsigned t, unsigned seg, unsigned u) const {
    return philox4x32_10(u32x4{t, seg, u, 0u}, k0, k1);
  }
};

// Acceptance r_a < Q_t / Q_prev with Q_t <= Q_prev, exactly.  Integer weights:
// while Q_prev < S neither product is capped and the ratio is w_t / w_prev
// (w_u cancels): (2k+1) w_prev < 2^53 w_t, with 2k+1 < 2^53 and w < 2^31, is
// L < w_t 2^21 for L = floor((2k+1) w_prev / 2^32) (the low 32 bits of the
// product cannot decide it); a capped Q_prev = S takes the 128-bit test.
__device__ __forceinline__ bool accept_ratio(unsigned long long k, unsigned w_prev, unsigned w_t) {
  const unsigned long long a = 2ull * k + 1ull;
  const unsigned a_lo = (unsigned)a, a_hi = (unsigned)(a >> 32);
  const unsigned long long L = (unsigned long long)a_hi * w_prev + __umulhi(a_lo, w_prev);
  return L < ((unsigned long long)w_t << 21);
}

// A capped run at an item's first position `target` (p = 1 there): the weights are
// sorted, so every position from target up to the first v with Q(v) < S (or the
// item's end) has p = 1, and Algorithm 1 takes each of them as an edge (skip 0,
// acceptance certain), one draw per position.  The run's end is found by bisection
// over the weights and its edges are written in one go (staged in whole sectors, or
// emitted) instead of one loop iteration per edge.  The draw that follows the run
// (number L of the item's stream) is made here too.
struct RunEnd {
  unsigned L, z, w;
  ff lr;
};
template <int MODE, bool WF, typename E>
__device__ __forceinline__ RunEnd capped_run(const typename Wt<WF>::w_t* __restrict__ W, typename Wt<WF>::w_t wu,
                                          typename Wt<WF>::q_t S, unsigned target, unsigned end, unsigned u,
                                          unsigned seg, unsigned key0, unsigned key1, unsigned* pool,
                                          unsigned long long sbase, unsigned ssize, int* overflow, E* edges,
                                          long long capacity) {
  using T = Wt<WF>;
  unsigned lo = target + 1, hi = end;
  while (lo < hi) {
    const unsigned mid = lo + ((hi - lo) >> 1);
    if (T::Q(wu, __ldg(&W[mid]), S) < S)
      hi = mid;
    else
      lo = mid + 1;
  }
  const unsigned L = lo - target;
  if (MODE == MODE_STAGE) {
    const unsigned m = L < ssize ? L : ssize;  // the slot is a multiple of 8 entries
    unsigned g = 0;
    for (; g + GROUP <= m; g += GROUP) {
      uint4* dst = (uint4*)(pool + sbase + g);
      const unsigned v = target + g;
      dst[0] = make_uint4(v, v + 1, v + 2, v + 3);
      dst[1] = make_uint4(v + 4, v + 5, v + 6, v + 7);
    }
    for (; g < m; ++g) pool[sbase + g] = target + g;
    if (L > ssize) atomicExch(overflow, 1);  // the item outgrew its slot: EMIT regenerates it
  }
  if (MODE == MODE_EMIT) {
    for (unsigned i = 0; i < L; ++i) {
      const long long pos = (long long)sbase + i;
      if (pos < capacity) {
        E e;
        e.x = u;
        e.y = target + i;
        edges[pos] = e;
      }
    }
  }
  const u32x4 nb = philox4x32_10(u32x4{L, seg, u, 0u}, key0, key1);
  return RunEnd{L, nb.z, nb.w, ff_neglog_r53_w(nb.x, nb.y)};
}

// A warp's queue of up to 32 upcoming items with their set-up data, and the
// feed it is filled from (shared memory; see sample_kernel).
template <typename w_t>
struct WarpQueue {
  long long item[32];
  unsigned long long sb[32];  // STAGE: slot base; EMIT: output position of the item's first edge
  long long cnt[32];          // EMIT: the item's edge count
  unsigned u[32], seg[32], ss[32];
  int g[32];
  w_t w[32];
  unsigned ok;                // bit r: entry r holds an item to run
  int tasks_left, cg;
  unsigned rtask, cu, cseg;   // round robin: the task's first item; consecutive: cursor at fnext
  long long fnext, fend;      // items (or list entries, or round-robin steps) not yet queued
};

// The persistent sampling kernel.  Lanes run items; a warp keeps a queue of
// up to 32 upcoming items of its current task, one per lane, with their
// set-up data (row, segment, w_u, staging slot or output offset) loaded
// ahead, 32 items at a time with coalesced loads; a lane whose item ends takes
// the next queue entry by shuffle.  Queue sources: consecutive items of an
// Eq. 3 task (a warp cursor walks row/segment positions), the regeneration
// list (EMIT), or the strided items of a round-robin task.
template <int MODE, bool SINGLE, bool WF, typename E>
__global__ void __launch_bounds__(SAMPLER_THREADS, SAMPLER_MIN_BLOCKS)
    sample_kernel(DevPlan P, DevGraph G1, long long ib, long long ie, const long long* __restrict__ offsets,
                  E* __restrict__ edges, long long capacity, int* __restrict__ counts, int regen_only, int t0,
                  long long ob) {
  using T = Wt<WF>;
  using w_t = typename T::w_t;
  using q_t = typename T::q_t;
  const int lane = threadIdx.x & 31;
  const unsigned lanemask_lt = (1u << lane) - 1u;
  long long off_base = 0;
  bool list_mode = false;  // regeneration driven by the list of items that outgrew their slots
  long long n_list = 0;
  if (MODE == MODE_EMIT) {
    if (regen_only) {
      unsigned nov = *(volatile unsigned*)P.ovf_count;
      if (nov == 0) return;  // every item fit in its slot
      if (nov <= P.ovf_cap) {
        list_mode = true;
        n_list = nov;
      }
    }
    off_base = offsets[ob];  // edges[0] holds the first edge of item ob
    if (offsets[ie] - off_base > capacity) {
      if (blockIdx.x == 0 && threadIdx.x == 0) set_error(P.err, CL_ERR_CAPACITY);
      return;  // nothing is written when the range does not fit
    }
  }
  const bool rrp = P.rrp != 0 && !list_mode;
  const bool scattered = list_mode || rrp;
  const int wid = threadIdx.x >> 5;
  // the warp's queue and feed (shared memory: they are touched once per item, not per iteration)
  __shared__ WarpQueue<w_t> wqs[SAMPLER_THREADS / 32];
  __shared__ long long s_item[SAMPLER_THREADS];  // the lane's current item
  WarpQueue<w_t>& Q = wqs[wid];
  if (lane == 0) {
    Q.fnext = 0;
    Q.fend = 0;
    Q.tasks_left = 1;
  }
  __syncwarp();
  int qn = 0, qh = 0;  // entries [qh, qn) of the queue are still to be taken (warp-uniform)
  // ---- lane state
  bool have = false, fresh = false;
  unsigned long long sbase = 0;  // STAGE: slot base; EMIT: output position of edge 0
  unsigned ssize = 0;
  long long expect = 0;
  unsigned u = 0, seg = 0, j = 0, end = 0, t = 0, k = 0;
  q_t Qprev = 0;
  typename T::lp_t Lp{};
  w_t wu = 0;
  unsigned wprev = 0;        // integer weights: w of the last candidate (Q_prev = w_u w_prev unless capped)
  unsigned pz = 0, pw = 0;   // the lane's next draw (index t): acceptance words ...
  ff pLr{0.f, 0.f};          // ... and its -ln r_s
  int gi_l = 0;              // graph of the lane's item (batched plans)
  const w_t* w_l = nullptr;
  q_t S_l = 0;
  Keys<SINGLE> keys{};
  unsigned n_iter = 0;
  int cur_task = -1;  // the task the warp took last (per-task clock)
  const bool clock_tasks = MODE != MODE_EMIT && P.task_ns != nullptr;

  // Fills the queue with up to 32 items (fetching tasks as needed); false when none is left.
  auto reload = [&]() -> bool {
    long long fnext = Q.fnext, fend = Q.fend;
    while (fnext >= fend) {
      if (!Q.tasks_left) return false;
      unsigned tix = 0;
      if (lane == 0) tix = atomicAdd(P.task_ctr, 1u);
      tix = __shfl_sync(FULL_MASK, tix, 0);
      bool stop = false;
      if (MODE == MODE_EMIT && list_mode) {
        if ((long long)tix * 32 >= n_list) {
          stop = true;
        } else {
          fnext = (long long)tix * 32;
          fend = fnext + 32 < n_list ? fnext + 32 : n_list;
        }
      } else {
        tix += (unsigned)t0;  // the range's first task
        if (clock_tasks && lane == 0 && tix < (unsigned)P.T) {
          const unsigned long long now = global_ns();
          if (cur_task >= 0) P.task_ns[2 * cur_task + 1] = now;
          P.task_ns[2 * tix] = now;
        }
        if (tix < (unsigned)P.T) cur_task = (int)tix;
        if (rrp) {
          if (tix >= (unsigned)P.T || (long long)tix >= P.n_items) {
            stop = true;
          } else {
            if (lane == 0) Q.rtask = tix;
            fnext = 0;
            fend = (P.n_items - (long long)tix + P.T - 1) / P.T;
          }
        } else if (tix >= (unsigned)P.T || P.task_start[tix] >= ie) {
          stop = true;
        } else {
          const long long a = P.task_start[tix], b = P.task_start[tix + 1];
          fnext = a > ib ? a : ib;
          fend = b < ie ? b : ie;
          if (fnext < fend && lane == 0) {  // position of the task's first item (once per task)
            const int g0 = SINGLE ? 0 : graph_of_item(P.graphs, P.G, fnext);
            const DevGraph& g = SINGLE ? G1 : P.graphs[g0];
            const ItemPos cp = item_pos(g, fnext - g.item_begin);
            Q.cg = g0;
            Q.cu = cp.u;
            Q.cseg = cp.seg;
          }
        }
      }
      if (stop) {
        if (lane == 0) Q.tasks_left = 0;
        __syncwarp();
        return false;
      }
      __syncwarp();
    }
    const long long left = fend - fnext;
    const int avail = left < 32 ? (int)left : 32;
    bool ok = lane < avail;
    long long it = 0;
    int gq = 0;
    ItemPos ip{0, 0u, 0u};
    if (scattered) {
      if (ok) {
        it = (MODE == MODE_EMIT && list_mode) ? P.ovf_list[fnext + lane]
                                              : (long long)Q.rtask + (fnext + lane) * (long long)P.T;
        ok = it >= ib && it < ie;
      }
      if (ok) {
        gq = SINGLE ? 0 : graph_of_item(P.graphs, P.G, it);
        const DevGraph& g = SINGLE ? G1 : P.graphs[gq];
        ip = item_pos(g, it - g.item_begin);
      }
    } else {
      const int cg = Q.cg;
      const unsigned cu = Q.cu, cseg = Q.cseg;
      __syncwarp();  // every lane has read the cursor before lane 0 moves it
      it = fnext + lane;
      gq = cg;
      ip = ItemPos{fnext - (SINGLE ? 0ll : P.graphs[cg].item_begin), cu, cseg};
      if (SINGLE) {
        ip = item_advance(G1, ip, ok ? lane : 0);
      } else if (ok) {
        cursor_advance(P.graphs, gq, ip, lane);
      }
      // the warp cursor moves past the queued items
      if (fnext + avail < fend && lane == 0) {
        int cg2 = cg;
        ItemPos cp{fnext - (SINGLE ? 0ll : P.graphs[cg].item_begin), cu, cseg};
        if (SINGLE)
          cp = item_advance(G1, cp, avail);
        else
          cursor_advance(P.graphs, cg2, cp, avail);
        Q.cg = cg2;
        Q.cu = cp.u;
        Q.cseg = cp.seg;
      }
    }
    if (ok) {
      const w_t* Wq = SINGLE ? (const w_t*)G1.w : (const w_t*)P.graphs[gq].w;
      Q.w[lane] = __ldg(&Wq[ip.u]);
      Q.u[lane] = ip.u;
      Q.seg[lane] = ip.seg;
      Q.item[lane] = it;
      if (!SINGLE) Q.g[lane] = gq;
      if (MODE == MODE_STAGE) {
        const unsigned long long sb = (unsigned long long)(P.slot_base[it] - P.pool_shift);
        unsigned ss = slot_size(P, it);
        // a slot outside the pool, or not on a 32-byte boundary (the staged groups are written as
        // aligned 16-byte stores): never staged (checked, reported)
        if (ss > 0 && (sb + ss > P.pool_entries || (sb & 7ull) != 0)) {
          set_error(P.err, CL_ERR_DEVICE);
          ss = 0;
        }
        Q.sb[lane] = sb;
        Q.ss[lane] = ss;
      }
      if (MODE == MODE_EMIT) {
        const long long o0 = offsets[it];
        const long long cnt = offsets[it + 1] - o0;
        Q.sb[lane] = (unsigned long long)(o0 - off_base);
        Q.cnt[lane] = cnt;
        if (regen_only && !list_mode && cnt <= (long long)slot_size(P, it)) ok = false;  // staged: copied
      }
    }
    const unsigned okm = __ballot_sync(FULL_MASK, ok);
    if (lane == 0) {
      Q.ok = okm;
      Q.fnext = fnext + avail;
      Q.fend = fend;
    }
    __syncwarp();
    qn = avail;
    qh = 0;
    return true;
  };

  bool ended = false;  // the lane's item has ended; its count and staging are written at the next step (2)
  while (true) {
    unsigned target = 0;
    bool look = false;
    {
      const q_t S = SINGLE ? T::S(G1) : S_l;
      // ---- (1) one skip for running items, with the precomputed draw t
      if (have && !ended) {
        ++t;
        ++n_iter;
        const int R = (int)(end - j);  // >= 1; end <= n < 2^31
        int delta = 0;
        if (Qprev != S) {
          delta = T::skip1(pLr, Lp, R);
          if (delta == (int)SKIP_UNDECIDED) {
            bool tie;
            // rare: regenerate the draw's skip words rather than keep them in registers
            const u32x4 d = keys.draw(G1, t - 1u, seg, u);
            delta = (int)T::skip2(2ull * grid52(d.x, d.y) + 1ull, Qprev, S, R, &tie);
            atomicAdd(&P.stats[1], 1ull);
            if (tie) atomicAdd(&P.stats[2], 1ull);
          }
        }
        if (delta >= R) {
          ended = true;  // the candidate falls past the end of the item
        } else {
          target = j + (unsigned)delta;
          look = true;
        }
      }
    }
    // ---- (2) end of the items that ended in this skip or in the last pass's look
    if (have && ended) {
      if (MODE == MODE_EMIT) {
        if ((long long)k != expect) set_error(P.err, CL_ERR_DEVICE);
      } else {
        const long long item = s_item[threadIdx.x];
        counts[item] = (int)k;
        if (MODE == MODE_STAGE && k > ssize) {  // remember it for the regeneration pass
          unsigned idx = atomicAdd(P.ovf_count, 1u);
          if (idx < P.ovf_cap) P.ovf_list[idx] = item;
        }
      }
      have = false;
      ended = false;
    }
    // ---- (3) lanes without an item take the next queue entries
    unsigned need = __ballot_sync(FULL_MASK, !have);
    while (need) {
      if (qh >= qn && !reload()) break;
      const int rank = __popc(need & lanemask_lt);
      const int avail = qn - qh;
      if (!have && rank < avail) {
        const int e = qh + rank;
        if ((Q.ok >> e) & 1u) {
          have = true;
          fresh = true;
          s_item[threadIdx.x] = Q.item[e];
          u = Q.u[e];
          seg = Q.seg[e];
          wu = Q.w[e];
          if (!SINGLE) gi_l = Q.g[e];
          if (MODE != MODE_COUNT) sbase = Q.sb[e];
          if (MODE == MODE_STAGE) ssize = Q.ss[e];
          if (MODE == MODE_EMIT) expect = Q.cnt[e];
        }
      }
      const int taken = __popc(need);
      qh += taken < avail ? taken : avail;
      need = __ballot_sync(FULL_MASK, !have);
    }
    if (!__any_sync(FULL_MASK, have)) break;

    // ---- (4) set-up of new items: bounds (and the graph's constants in a batch)
    if (have && fresh) {
      unsigned j0;
      if (SINGLE) {
        pos_bounds(G1, ItemPos{0, u, seg}, j0, end);
      } else {
        const DevGraph& g = P.graphs[gi_l];
        pos_bounds(g, ItemPos{0, u, seg}, j0, end);
        w_l = (const w_t*)g.w;
        S_l = T::S(g);
        if constexpr (!SINGLE) {
          keys.k0 = g.key0;
          keys.k1 = g.key1;
        }
      }
      t = 0;
      k = 0;
      target = j0;  // first position: p = Q(j0) / S
      look = true;
    }
    const w_t* W = SINGLE ? (const w_t*)G1.w : w_l;
    const q_t S = SINGLE ? T::S(G1) : S_l;
    if (look) {
      // ---- (5) weight of the candidate (or of the first position); meanwhile the next draw
      w_t wt;
      if (WF) {
        wt = __ldg(&W[target]);
      } else {  // integer weights: the uniform-block table (an L1/L2-resident read; no per-lane cache)
        const unsigned long long* blk = SINGLE ? G1.blkp : P.graphs[gi_l].blkp;
        const unsigned long long be = __ldg(&blk[target >> BLK_SHIFT]);  // (w << 32) | run end, or mixed
        wt = (w_t)(int)(unsigned)(be >> 32);
        if (be == BLK_MIXED) wt = (w_t)__ldg(&((const int*)W)[target]);
      }
      const unsigned az = pz, aw = pw;  // acceptance words of the draw that made the candidate
      {
        const u32x4 nb = keys.draw(G1, t, seg, u);
        pz = nb.z;
        pw = nb.w;
        pLr = ff_neglog_r53_w(nb.x, nb.y);
      }
      const q_t Qt = T::Q(wu, wt, S);
      // ---- (6) acceptance r_a < q / p, with the draw that made the candidate
      {
        bool acc;
        if (!WF) {
          // equal weights pass the ratio test ((2k+1) w < 2^53 w), so they need no branch of
          // their own; the test is cheap enough to run for a new item's first position too and
          // be masked, which keeps a branch on `fresh` out of the loop
          if (Qprev != S)
            acc = accept_ratio(grid52(az, aw), wprev, (unsigned)wt);
          else
            acc = T::accept(grid52(az, aw), Qprev, Qt);
          acc = acc && !fresh;
        } else if (fresh) {
          acc = false;
        } else if (Qt == Qprev) {
          acc = true;
        } else {
          acc = T::accept(grid52(az, aw), Qprev, Qt);
        }
        if (acc) {
          if (MODE == MODE_EMIT) {
            long long pos = (long long)sbase + k;
            if (pos < capacity) {
              E e;
              e.x = u;
              e.y = target;
              edges[pos] = e;
            }
          }
          if (MODE == MODE_STAGE) {
            if (k < ssize) {
              P.pool[sbase + k] = target;
            } else if (k == ssize) {
              atomicExch(P.overflow, 1);  // the item outgrew its slot: EMIT regenerates it
            }
          }
          ++k;
        }
      }
      if (!WF) wprev = (unsigned)wt;
      // ---- (7) p <- q: a new L_p when q changed (and for a new item)
      if (WF) {
        if (fresh || Qt != Qprev) {
          Qprev = Qt;
          if (Qt == 0)
            ended = true;  // p = 0: no further edge
          else if (Qt < S)
            Lp = T::Lp(Qt, S, SINGLE ? G1 : P.graphs[gi_l]);
        }
      } else {
        // integer weights: in the series range (p < 2^-12, most candidates) L_p is
        // formed at every look -- the same value when q is unchanged -- which takes a
        // divergent branch out of the loop (measured 61.9 -> 60.4 ms on n = 10^8); the
        // table range keeps the test for a change of q
        const bool changed = fresh || Qt != Qprev;
        const LpConst& lpc = SINGLE ? G1.lp : P.graphs[gi_l].lp;
        Qprev = Qt;
        if (Qt == 0) ended = true;  // p = 0: no further edge
        if ((unsigned long long)Qt < lpc.Ssmall) {
          const unsigned long long Qi = (unsigned long long)Qt;  // < 2^41: two exact 23-bit chunks
          const ff q = ff_fast_two_sum(u23_to_f_2p23((unsigned)(Qi >> 23)), u23_to_f((unsigned)Qi & 0x7FFFFFu));
          Lp = ff_neglog1m_series(ff_mul(q, ff{lpc.iS_hi, lpc.iS_lo}));
        } else if (changed && Qt < S) {
          Lp = ff_neglog1m_table((unsigned long long)Qt, (unsigned long long)S, lpc);
        }
      }
      if (fresh && Qt == S && Qt != 0) {  // a capped run from the first position (S = 0: no edge)
        const unsigned key0 = SINGLE ? G1.key0 : P.graphs[gi_l].key0, key1 = SINGLE ? G1.key1 : P.graphs[gi_l].key1;
        const RunEnd r = capped_run<MODE, WF, E>(W, wu, S, target, end, u, seg, key0, key1, P.pool, sbase, ssize,
                                                 P.overflow, edges, capacity);
        k = r.L;  // its positions' draws are consumed: the next draw is number L
        t = r.L;
        n_iter += r.L;
        j = target + r.L;
        pz = r.z;
        pw = r.w;
        pLr = r.lr;
      } else {
        j = fresh ? target : target + 1;
      }
      if (j >= end) ended = true;
      fresh = false;
    }
  }
  if (clock_tasks && lane == 0 && cur_task >= 0) P.task_ns[2 * cur_task + 1] = global_ns();
  unsigned long long n_iter64 = n_iter;
  if (MODE != MODE_EMIT) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      n_iter64 += __shfl_xor_sync(FULL_MASK, n_iter64, o);
    }
    if (lane == 0) {
      atomicAdd(&P.stats[0], n_iter64);
    }
  }
}

// ---- copy of staged destinations.  A warp takes a claim of consecutive items
// from a counter (32 items, or 256 when items average under 8 edges: the small
// graphs of a batch, 5.8e8 items, took 1.8e7 claims of 32 on one counter, whose
// atomics alone then set the copy's time) and walks it 32 items at a time, one
// item per lane; their edges form one contiguous output range.  Items with at
// least 32 staged edges are copied by the whole warp, one item at a time (lane =
// edge); the others are flattened: the lanes cover their
// edges edge by edge (consecutive lanes write consecutive pairs), each lane
// finding its edge's item by a 5-step search over the warp's inclusive count
// prefix, so every load is independent of the others.  A memory-latency-bound
// kernel: 8 resident blocks per SM keep the loads in flight.
constexpr int COPY_THREADS = 256;

template <typename E>
__global__ void __launch_bounds__(COPY_THREADS, 8) copy_kernel(DevPlan P, long long ib, long long ie, long long ob,
                                                            const long long* __restrict__ offsets,
                                                            E* __restrict__ edges, long long capacity) {
  const int lane = threadIdx.x & 31;
  const long long off_base = offsets[ob];  // edges[0] holds the first edge of item ob
  if (offsets[ie] - off_base > capacity) {
    if (blockIdx.x == 0 && threadIdx.x == 0) set_error(P.err, CL_ERR_CAPACITY);
    return;
  }
  const int chunk = P.copy_chunk;
  while (true) {
    unsigned c = 0;
    if (lane == 0) c = atomicAdd(P.task_ctr, 1u);
    c = __shfl_sync(FULL_MASK, c, 0);
    const long long c0 = ib + (long long)c * chunk;
    if (c0 >= ie) break;
    const long long c1 = c0 + chunk < ie ? c0 + chunk : ie;
    // position of the claim's first item (one graph search per claim); a warp cursor
    // walks the claim 32 items at a time
    int g0 = P.G == 1 ? 0 : graph_of_item(P.graphs, P.G, c0);
    ItemPos p0 = item_pos(P.graphs[g0], c0 - P.graphs[g0].item_begin);
    for (long long i0 = c0; i0 < c1; i0 += 32) {
      if (i0 > c0) cursor_advance(P.graphs, g0, p0, 32);
      const long long i = i0 + lane;
      long long o = 0, pos = 0;
      int cnt = 0;
      unsigned uu = 0;
      if (i < c1) {
        o = offsets[i] - off_base;
        long long cc = offsets[i + 1] - offsets[i];
        pos = P.slot_base[i] - P.pool_shift;
        if (cc <= (long long)slot_size(P, i)) cnt = (int)cc;  // else: not staged, regenerated
        if (cnt > 0 && (pos < 0 || (unsigned long long)(pos + cnt) > P.pool_entries)) {  // checked, reported
          set_error(P.err, CL_ERR_DEVICE);
          cnt = 0;
        }
        if (cnt > 0) {
          int gi = g0;
          ItemPos ip = p0;
          cursor_advance(P.graphs, gi, ip, lane);
          uu = ip.u;
        }
      }
      // items with at least 32 staged edges: the whole warp copies one item at a
      // time (lane = edge, coalesced, four loads in flight per lane)
      unsigned big = __ballot_sync(FULL_MASK, cnt >= 32);
      while (big) {
        const int l = __ffs(big) - 1;
        big &= big - 1;
        const int cl = __shfl_sync(FULL_MASK, cnt, l);
        const long long ol = __shfl_sync(FULL_MASK, o, l);
        const long long pl = __shfl_sync(FULL_MASK, pos, l);
        const unsigned su = __shfl_sync(FULL_MASK, uu, l);
        for (int e0 = lane; e0 < cl; e0 += 32 * 4) {
          unsigned v[4];
  #pragma unroll
          for (int q = 0; q < 4; ++q) v[q] = e0 + 32 * q < cl ? P.pool[pl + e0 + 32 * q] : 0u;
  #pragma unroll
          for (int q = 0; q < 4; ++q)
            if (e0 + 32 * q < cl) {
              E pr;
              pr.x = su;
              pr.y = v[q];
              edges[ol + e0 + 32 * q] = pr;
            }
        }
      }
      if (cnt >= 32) cnt = 0;  // done above; the rest are flattened edge by edge
      int incl = cnt;
  #pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        int y = __shfl_up_sync(FULL_MASK, incl, d);
        if (lane >= d) incl += y;
      }
      const int total = __shfl_sync(FULL_MASK, incl, 31);
      // edges per lane per step: 1 measured fastest (13.0 against 13.6 ms for 4 and
      // 14.4 ms for 8 on a 3.9e9-edge emit): the warps, not the lanes, keep the loads in flight
      constexpr int U = 1;
      for (int base = 0; base < total; base += 32 * U) {
        long long dst[U];
        unsigned src_u[U];
        unsigned val[U];
        bool ok[U];
  #pragma unroll
        for (int q = 0; q < U; ++q) {
          int e = base + 32 * q + lane;
          // smallest lane l with incl_l > e (it has cnt_l > 0)
          int lo = 0, hi = 31;
  #pragma unroll
          for (int it = 0; it < 5; ++it) {
            int mid = (lo + hi) >> 1;
            int iv = __shfl_sync(FULL_MASK, incl, mid);
            if (iv > e)
              hi = mid;
            else
              lo = mid + 1;
          }
          int il = __shfl_sync(FULL_MASK, incl, lo);
          int cl = __shfl_sync(FULL_MASK, cnt, lo);
          long long ol = __shfl_sync(FULL_MASK, o, lo);
          long long pl = __shfl_sync(FULL_MASK, pos, lo);
          src_u[q] = __shfl_sync(FULL_MASK, uu, lo);
          ok[q] = e < total;
          int local = e - (il - cl);
          dst[q] = ol + local;
          val[q] = ok[q] ? P.pool[pl + local] : 0u;
        }
  #pragma unroll
        for (int q = 0; q < U; ++q) {
          if (ok[q]) {
            E pr;
            pr.x = src_u[q];
            pr.y = val[q];
            edges[dst[q]] = pr;
          }
        }
      }
    }
  }
}

int sampler_max_blocks_per_sm(int block, bool emit, int etype) {
  int nb = 0;
  if (!emit)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sample_kernel<MODE_STAGE, false, false, int2>, block, 0);
  else if (etype == CL_E_I32)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sample_kernel<MODE_EMIT, false, false, int2>, block, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sample_kernel<MODE_EMIT, false, false, longlong2>, block, 0);
  return nb;
}

template <int MODE, bool WF, typename E>
static void launch_sampler_w(const DevPlan& P, const DevGraph* single, const SampleRange& r, const long long* offsets,
                             E* edges, long long capacity, int* counts, int regen, int block, int grid,
                             cudaStream_t s) {
  if (single)
    sample_kernel<MODE, true, WF, E><<<grid, block, 0, s>>>(P, *single, r.ib, r.ie, offsets, edges, capacity, counts,
                                                            regen, r.t0, r.ob);
  else
    sample_kernel<MODE, false, WF, E><<<grid, block, 0, s>>>(P, DevGraph{}, r.ib, r.ie, offsets, edges, capacity,
                                                             counts, regen, r.t0, r.ob);
}

template <int MODE, typename E>
static void launch_sampler(const DevPlan& P, const DevGraph* single, const SampleRange& r, const long long* offsets,
                           E* edges, long long capacity, int* counts, int regen, int block, int grid,
                           cudaStream_t s) {
  if (P.wf64)
    launch_sampler_w<MODE, true, E>(P, single, r, offsets, edges, capacity, counts, regen, block, grid, s);
  else
    launch_sampler_w<MODE, false, E>(P, single, r, offsets, edges, capacity, counts, regen, block, grid, s);
}

void launch_count(const DevPlan& P, const DevGraph* single, int* d_counts, bool stage, int block, int grid,
                  cudaStream_t s) {
  if (stage) {
    cudaMemsetAsync(P.overflow, 0, sizeof(int), s);
    cudaMemsetAsync(P.ovf_count, 0, sizeof(unsigned), s);
  }
  launch_count_range(P, single, d_counts, stage, SampleRange{0, P.n_items, 0, 0}, block, grid, s);
}

void launch_count_range(const DevPlan& P, const DevGraph* single, int* d_counts, bool stage, const SampleRange& r,
                        int block, int grid, cudaStream_t s) {
  cudaMemsetAsync(P.task_ctr, 0, sizeof(unsigned), s);
  if (stage)
    launch_sampler<MODE_STAGE, int2>(P, single, r, nullptr, nullptr, 0, d_counts, 0, block, grid, s);
  else
    launch_sampler<MODE_COUNT, int2>(P, single, r, nullptr, nullptr, 0, d_counts, 0, block, grid, s);
}

void launch_emit(const DevPlan& P, const DevGraph* single, const long long* d_offsets, const SampleRange& r,
                 int etype, void* d_edges, long long capacity, bool staged, int block, int grid, int copy_grid,
                 cudaStream_t s) {
  cudaMemsetAsync(P.task_ctr, 0, sizeof(unsigned), s);
  if (staged) {
    // warps deal the output's COPY_EDGES-edge chunks round-robin; the item count bounds
    // the useful grid from above (a chunk holds at least one item)
    long long cg = (r.ie - r.ib + 8 * 32 - 1) / (8 * 32);
    int cgrid = (int)(cg < 4096 ? (cg < 1 ? 1 : cg) : 4096);
    if (copy_grid > 0 && cgrid > copy_grid) cgrid = copy_grid;
    if (etype == CL_E_I32)
      copy_kernel<int2><<<cgrid, COPY_THREADS, 0, s>>>(P, r.ib, r.ie, r.ob, d_offsets, (int2*)d_edges, capacity);
    else
      copy_kernel<longlong2>
          <<<cgrid, COPY_THREADS, 0, s>>>(P, r.ib, r.ie, r.ob, d_offsets, (longlong2*)d_edges, capacity);
    // items that outgrew their slots are regenerated (the kernel returns at
    // once when none did)
    cudaMemsetAsync(P.task_ctr, 0, sizeof(unsigned), s);
  }
  int regen = staged ? 1 : 0;
  if (etype == CL_E_I32)
    launch_sampler<MODE_EMIT, int2>(P, single, r, d_offsets, (int2*)d_edges, capacity, nullptr, regen, block, grid, s);
  else
    launch_sampler<MODE_EMIT, longlong2>(P, single, r, d_offsets, (longlong2*)d_edges, capacity, nullptr, regen, block,
                                         grid, s);
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
