/*
 * cl.h -- C ABI of a single-GPU (GB300, sm_103a) Chung-Lu random-network
 * generator: the edge-skipping sampler of Algorithm 1 of Alam & Khan,
 * "Parallel Algorithms for Generating Random Networks with Given Degree
 * Sequences" (Section 3), parallelised over source nodes with the paper's
 * cost model (Eq. 1, Eq. 2, Eq. 6) and uniform cost partitioning (Eq. 3,
 * Algorithm 2), plus capped expected degrees and their adjoint for weight
 * calibration.
 *
 * Problem statement (Section 3): n nodes with non-negative weights
 * w_0 >= w_1 >= ... >= w_{n-1} (sorted non-increasing), S = sum_k w_k; each
 * pair (u, v), u < v, is an edge independently with probability
 * min(w_u w_v / S, 1).  A weight sequence and a seed go in; an edge list
 * (u, v), u < v, comes out, in canonical order (u ascending, then v
 * ascending) -- exactly the order of Algorithm 1 run sequentially.
 *
 * Conventions for every call:
 *   - pointers named d_* are CUDA device pointers owned by the caller; h_*
 *     are host pointers owned by the caller.  The library never allocates
 *     device memory: scratch and workspace are caller-provided.
 *   - calls are asynchronous on `stream` unless documented as synchronizing.
 *   - every call returns a cl_status; device-side consistency failures are
 *     recorded in a device error word and reported by the next synchronizing
 *     call (cl_check, cl_stats, cl_scan with a non-null h_total).  No kernel
 *     traps, asserts or waits on another block.
 *   - CL_ERR_CUDA after a launch comes from the runtime's last-error state,
 *     read (and cleared) right after the launch: it can also report an error
 *     that earlier, unrelated CUDA work left pending on the calling thread.
 *   - vertex ids are positions in the sorted order; relabelling is the
 *     caller's job.
 *
 * The random stream (fixes every output bit; independent of launch shape):
 *   item    = a light row u (w_u < heavy_w): v in [u+1, n), segment field
 *             0xFFFFFFFF; or a heavy row u (w_u >= heavy_w) cut at absolute
 *             multiples of 2^16 of v: v in [max(u+1, k 2^16), min(n, (k+1) 2^16)),
 *             segment field k.
 *   draw t  = Philox4x32-10, key (seed_lo, seed_hi), counter (t, segment,
 *             u_lo, u_hi); words 0-1 give the skip uniform, words 2-3 the
 *             acceptance uniform, each r = (2k+1)/2^53 from the top 52 bits.
 *   loop    = Algorithm 1 per item: p = Q_prev/S with Q(v) = min(w_u w_v, S);
 *             delta = floor(ln r / ln(1 - p)) (the exact real floor; 0 when
 *             p = 1); v = j + delta; stop when v leaves the item; accept iff
 *             r_a * Q_prev < Q_v exactly; Q_prev <- Q_v; j <- v + 1; stop when
 *             Q_prev = 0.
 */
#ifndef CL_H
#define CL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* cl_stream_t; /* a cudaStream_t; NULL is the legacy default stream */

typedef enum {
  CL_OK = 0,
  CL_ERR_INVALID_ARG = 1, /* null pointer, bad enum, negative size, bad item range */
  CL_ERR_UNSORTED = 2,    /* weights not non-increasing (Section 3 precondition) */
  CL_ERR_NONFINITE = 3,   /* a weight is negative, NaN or infinite */
  CL_ERR_RANGE = 4,       /* n >= 2^31 (int32 ids) or n >= 2^32, S >= 2^53, or size overflow */
  CL_ERR_CAPACITY = 5,    /* the output buffer is smaller than the edge count */
  CL_ERR_WORKSPACE = 6,   /* scratch or workspace smaller than required */
  CL_ERR_TIMEOUT = 7,     /* reserved: no call of this library waits on the device */
  CL_ERR_CUDA = 8,        /* a CUDA runtime call failed */
  CL_ERR_STATE = 9,       /* call order violated (e.g. cl_count before cl_plan_build) */
  CL_ERR_DEVICE = 10,     /* a device-side consistency check failed (see cl_check) */
  CL_ERR_STOPPED = 11     /* cl_generate_stream: the caller's sink returned non-zero */
} cl_status;

typedef enum { CL_W_I32 = 0, CL_W_F64 = 1 } cl_wtype;
typedef enum { CL_E_I32 = 0, CL_E_I64 = 1 } cl_etype;

/* One Chung-Lu instance.  heavy_w and the segment width (2^16) are stream
 * parameters: they change which random numbers are drawn, hence the output.
 * For CL_W_I32 the weights are integers (expected degrees) and S must be
 * < 2^53; for CL_W_F64 they are finite non-negative doubles. */
typedef struct {
  int64_t n;          /* nodes; n < 2^31 */
  int32_t wtype;      /* cl_wtype */
  const void* d_w;    /* device array of n weights, sorted non-increasing; read only */
  uint64_t seed;      /* Philox key */
  double heavy_w;     /* rows with w_u >= heavy_w are segmented (default 8192) */
} cl_graph;

/* Performance knobs only: no choice changes any output bit. */
typedef struct {
  int32_t tasks;         /* number of equal-cost tasks (Eq. 3 partitions); 0 = automatic: about
                          * 10^4 edges of cost each, 4 to 64 per resident warp of the count pass */
  int32_t block;         /* threads per block of the sampler kernels, multiple of 32, <= 256; 0 = 256 */
  int32_t blocks_per_sm; /* resident blocks per SM for the persistent sampler grid; 0 = automatic */
  int32_t no_stage;      /* 1: cl_count only counts and cl_emit regenerates every item (smaller
                          * workspace, twice the sampling work); 0: cl_count also stages each
                          * item's destinations in a slot of e + 6 sqrt(e) + 6 entries (e = the
                          * item's uncapped expected edges, Eq. 1) and cl_emit copies them;
                          * items that outgrow their slot are regenerated by cl_emit */
  double stage_factor;   /* 0; a negative value shrinks every slot to 8 entries, so that most
                          * items take the regeneration path (for testing that path) */
  int32_t partition;     /* task split: CL_PART_UCP (0, default) = equal Eq. 1 cost per task
                          * (Eq. 3, the uniform cost partition); CL_PART_CP (1) = equal node counts
                          * (the paper's consecutive partition, Section 4); CL_PART_RRP (2) = round
                          * robin (Section 4): task t holds the items t, t + T, t + 2T, ...; the
                          * last two are for comparing partitions (cl_generate_host refuses
                          * CL_PART_RRP); other values: CL_ERR_INVALID_ARG */
  int64_t max_pool_entries; /* 0; > 0 caps the staging pool (4 bytes per entry): items whose slot
                          * lies beyond the cap are regenerated by cl_emit (for graphs whose full
                          * staging would not fit in device memory, e.g. with cl_generate_stream) */
} cl_tuning;

enum { CL_PART_UCP = 0, CL_PART_CP = 1, CL_PART_RRP = 2 };

typedef struct {
  int64_t n, H;           /* nodes, heavy rows */
  int64_t n_items;        /* items of this graph */
  int64_t item_begin;     /* first global item index of this graph in the plan */
  int64_t S_i64;          /* exact weight sum (CL_W_I32) */
  double S;               /* weight sum as a double (CL_W_F64: correctly rounded) */
  int32_t status;         /* cl_status of this graph's validation */
} cl_graph_info;

typedef struct {
  int64_t iterations;     /* loop iterations (Philox blocks) of the last count pass */
  int64_t fallbacks;      /* skips decided by the double-double tier (last count pass) */
  int64_t ties;           /* skips within 2^-96 x of an integer (took the nearest integer) */
  int32_t error;          /* device error word (0 = none) */
} cl_run_stats;

typedef struct cl_plan cl_plan; /* opaque host handle */

const char* cl_status_string(cl_status s);

/* --- planning (Section 4: the sum S, the cost model Eq. 1-2 / Eq. 6 and the
 *     uniform cost partition Eq. 3 / Algorithm 2) ------------------------- */

/* Bytes of device scratch cl_plan_create needs for G graphs. */
size_t cl_plan_scratch_bytes(int32_t G);

/* Validates every graph (sorted non-increasing, non-negative, finite), computes
 * S = sum_k w_k exactly (Algorithm 1, first line; integer weights: exact int64
 * sum; double weights: the correctly rounded value of the exact sum), the
 * heavy rows and the item space.  SYNCHRONIZING (reads the results back).
 * graphs: host array of G descriptors (copied; the device weight arrays must
 * stay alive and unchanged for the plan's lifetime).  d_scratch: at least
 * cl_plan_scratch_bytes(G) bytes, 256-byte aligned (as cudaMalloc returns;
 * otherwise CL_ERR_INVALID_ARG), free again when the call returns.
 * Errors: CL_ERR_INVALID_ARG, CL_ERR_RANGE, CL_ERR_UNSORTED, CL_ERR_NONFINITE
 * (the first failing graph's status; per-graph status via cl_plan_graph_info),
 * CL_ERR_WORKSPACE, CL_ERR_CUDA.  On error *out is NULL. */
cl_status cl_plan_create(const cl_graph* graphs, int32_t G, const cl_tuning* tuning, void* d_scratch,
                         size_t scratch_bytes, cl_stream_t stream, cl_plan** out);

/* Device workspace bytes cl_plan_build needs (cost prefix, task table, scan
 * partials, counters). */
cl_status cl_plan_workspace_bytes(const cl_plan* plan, size_t* bytes);

/* Builds the equal-cost task split of Eq. 3 in the workspace: per item
 * c = c0 + (w_u / S) * sum_{v in item} w_v (Eq. 1-2; Eq. 6 for light rows;
 * c0 = 4, the measured work of an item apart from its edges, where Eq. 1 has 1),
 * C = inclusive prefix of c (Calc-Cost of Algorithm 2 as a device-wide scan),
 * task t starts at the first item with C >= t * Zbar, Zbar = C_total / tasks
 * (Eq. 3; found as the items where floor(C / Zbar) changes, the rule of
 * Find-Boundaries).  Asynchronous; capturable in a CUDA graph.  d_ws: at least
 * cl_plan_workspace_bytes bytes (else CL_ERR_WORKSPACE), 256-byte aligned (as
 * cudaMalloc returns; else CL_ERR_INVALID_ARG), reserved for the plan until
 * cl_plan_destroy.  Tasks only schedule work: the
 * output does not depend on them. */
cl_status cl_plan_build(cl_plan* plan, void* d_ws, size_t ws_bytes, cl_stream_t stream);

cl_status cl_plan_items(const cl_plan* plan, int64_t* n_items);

/* The task split that cl_plan_build made (Section 4: Eq. 1-2 costs, Eq. 3
 * boundaries), for inspection and tests.  *T = number of tasks (always set).
 * d_task_start (nullable, T + 1 int64): task t holds the items
 * [d_task_start[t], d_task_start[t + 1]) (Eq. 3's lower boundaries n_t, with
 * d_task_start[T] = n_items); under CL_PART_RRP task t holds the items
 * t, t + T, t + 2T, ... and d_task_start[t] = min(t, n_items).
 * d_cost_prefix (nullable, n_items int64): the inclusive prefix C_i of the
 * item costs c_i = c0 + (w_u / S) sum_{v in item} w_v in units of 1/16 edge
 * (c0 = 4 edges; each term rounded to the unit from single precision).
 * Asynchronous device-to-device copies on `stream`; requires cl_plan_build. */
cl_status cl_plan_tasks(const cl_plan* plan, int32_t* T, int64_t* d_task_start, int64_t* d_cost_prefix,
                        cl_stream_t stream);
cl_status cl_plan_graph_info(const cl_plan* plan, int32_t g, cl_graph_info* out);

/* Per-task timing of the count passes (the runtime-follows-cost measurement of
 * Section 5, Figs. 1 and 5, at task granularity).  d_task_ns: a caller-owned
 * device array of 2 T uint64 (T from cl_plan_tasks), or NULL to stop.  Every
 * later count pass stores, for each task a warp takes, the GPU's global timer
 * (ns) at the moment the warp took it (d_task_ns[2t]) and at the moment the
 * same warp took its next task or finished (d_task_ns[2t + 1]) -- with one task
 * per warp, the task's run time.  Entries of tasks no warp took are left as
 * they were.  Host-side setting only; no synchronisation. */
cl_status cl_plan_task_clock(cl_plan* plan, uint64_t* d_task_ns);

/* The launch shape of the count pass: grid (blocks; persistent, resident
 * blocks per SM times SMs) and threads per block.  T = count_grid * block / 32
 * tasks give one task per resident warp. */
cl_status cl_plan_launch_info(const cl_plan* plan, int32_t* count_grid, int32_t* block);

/* --- sampling (Algorithm 1, Create-Edges, per item) ---------------------- */

/* Count pass (Algorithm 1, Create-Edges, run per item with the stream above;
 * Section 3): d_counts[i] = number of edges of global item i (int32, n_items
 * entries, caller-owned).  Unless the tuning disabled staging, the pass also
 * stores each item's destination nodes, in order, in the plan workspace, so
 * that cl_emit only has to copy them (the sampling arithmetic runs once).
 * Asynchronous. */
cl_status cl_count(cl_plan* plan, int32_t* d_counts, cl_stream_t stream);

/* Exclusive scan of the counts -- the prefix-sum step of Calc-Cost
 * (Algorithm 2, Section 4) applied to the items' edge counts instead of their
 * costs, which places every item's edges in one array in canonical order:
 * d_offsets[i] = sum_{k<i} d_counts[k] for
 * i = 0..n_items (n_items + 1 int64 entries; d_offsets[n_items] = m).  If
 * h_total is non-null the call SYNCHRONIZES and writes m there, and reports a
 * pending device error as CL_ERR_DEVICE.  d_counts and d_offsets must not
 * overlap. */
cl_status cl_scan(cl_plan* plan, const int32_t* d_counts, int64_t* d_offsets, int64_t* h_total,
                  cl_stream_t stream);

/* Emit pass (Algorithm 1's output: the accepted pairs (u, v); Section 3): writes the
 * edges of items [item_begin, item_end) -- copied from
 * the staging of the last cl_count when there is one, otherwise (and for items
 * that did not fit in the staging pool) regenerated -- edge k of
 * item i to d_edges[d_offsets[i] - d_offsets[item_begin] + k] as a (u, v)
 * pair of etype (CL_E_I32: 2 x int32 = 8 bytes; CL_E_I64: 2 x int64 = 16
 * bytes), u < v, local vertex ids of the item's graph.  capacity = edges that
 * fit in d_edges; a range whose edges exceed it is not written and sets
 * CL_ERR_CAPACITY in the device error word (the host cannot see m without a
 * synchronisation).  Asynchronous.  d_offsets from cl_scan of the same plan. */
cl_status cl_emit(cl_plan* plan, const int64_t* d_offsets, int32_t etype, void* d_edges, int64_t capacity,
                  int64_t item_begin, int64_t item_end, cl_stream_t stream);

/* Algorithm 1 over every item (Section 3) with the count prefix of Algorithm 2
 * placing the edges: cl_count + cl_scan + cl_emit over all items in one call, with no host
 * round trip: d_counts and d_offsets are filled as by cl_count and cl_scan,
 * edge k of item i goes to d_edges[d_offsets[i] + k].  h_total (nullable):
 * synchronizes and returns m; m > capacity returns CL_ERR_CAPACITY (nothing is
 * written to d_edges then).  Asynchronous when h_total is NULL. */
cl_status cl_generate(cl_plan* plan, int32_t etype, void* d_edges, int64_t capacity, int32_t* d_counts,
                      int64_t* d_offsets, int64_t* h_total, cl_stream_t stream);

/* Algorithm 1 (Section 3) for every graph of a multi-graph plan, the items of
 * all graphs in one item space split by Eq. 3 (Section 4):
 * count + scan + emit for every graph of the plan, with no host round trip:
 * graph g's edges start at d_graph_offsets[g] (G + 1 int64 entries,
 * d_graph_offsets[G] = total edges) and carry the graph's local vertex ids.
 * d_counts (n_items int32) and d_offsets (n_items + 1 int64) are caller
 * scratch.  If the total exceeds capacity nothing is written to d_edges and
 * *d_status (device int32) is set to CL_ERR_CAPACITY, else to CL_OK.
 * Asynchronous; capturable in a CUDA graph (the batched path of a CUDA-graph
 * replay).  Requires cl_plan_build. */
cl_status cl_generate_batch(cl_plan* plan, int32_t etype, void* d_edges, int64_t capacity,
                            int64_t* d_graph_offsets, int32_t* d_counts, int64_t* d_offsets,
                            int32_t* d_status, cl_stream_t stream);

/* Count + scan + emit of the whole plan with the edge list delivered to host
 * memory h_edges (Algorithm 1's output as in cl_emit: same order and ids).
 *  - d_edges != NULL (device buffer of `capacity` edges): the items are cut into
 *    at least `chunks` windows of whole Eq. 3 tasks (0: 8; at most
 *    CL_HOST_MAX_CHUNKS; each window's staging fits in half of the plan's pool);
 *    window w is counted and scanned on a second stream of the plan while window
 *    w - 1 is emitted into d_edges at its final offsets and copied to h_edges at
 *    the same offsets on a third (copy engines).  One counting launch per window
 *    lets a window's longest items run beside its other items.  h_edges should be
 *    page-locked for full speed.
 *  - d_edges == NULL: the items are cut into `chunks` ranges of equal Eq. 3 cost,
 *    and the emitting kernels store straight into h_edges, on `copy_sms` SMs (0:
 *    16) that the counting launch leaves free.  h_edges must then be host memory
 *    the device can address: page-locked and mapped (cudaHostAlloc; on
 *    unified-addressing systems every page-locked buffer is mapped), or any host
 *    memory where the GPU reads and writes pageable memory (a coherent CPU-GPU
 *    link); otherwise CL_ERR_INVALID_ARG.
 * d_counts (n_items int32) and d_offsets (n_items + 1 int64) are caller
 * device scratch, filled as by cl_count and cl_scan.  Synchronous: returns
 * after the last edge is in host memory, with *h_total = m; m > capacity
 * returns CL_ERR_CAPACITY (windows or ranges that do not fit are not written).
 * Refuses CL_PART_RRP plans.  Not capturable in a CUDA graph. */
#define CL_HOST_MAX_CHUNKS 64
cl_status cl_generate_host(cl_plan* plan, int32_t etype, void* h_edges, int64_t capacity, void* d_edges,
                           int32_t* d_counts, int64_t* d_offsets, int32_t chunks, int32_t copy_sms,
                           int64_t* h_total, cl_stream_t stream);

/* Out-of-core delivery: Algorithm 1 over every item (Section 3), the edge
 * list handed to the caller's sink piece by piece through a bounded ring, so
 * that a graph larger than device and host memory can be produced (the
 * paper's 1-billion-node, 249-billion-edge network of Section 5 is ~2 TB as
 * int32 pairs).  Items go in consecutive ranges of Eq. 3 tasks (Section 4)
 * whose cost is about a quarter of the ring; a range is counted and scanned
 * (d_counts / d_offsets as by cl_count / cl_scan, for all items), then emitted
 * into the device ring in pieces of at most ring_edges / 2 edges (more than
 * one only when a range came out larger), each copied to the host ring and
 * passed to sink(user, h_edges, first_edge, n_edges, item_begin, item_end):
 * h_edges holds n_edges pairs of etype, the edges first_edge ..
 * first_edge + n_edges - 1 of the canonical edge list, which are those of
 * items [item_begin, item_end).  The sink runs on the calling thread, in edge
 * order, while the next range is being counted on the GPU; the data is valid
 * until it returns.  A non-zero return stops the generation:
 * CL_ERR_STOPPED, *h_total = edges handed over.  d_ring: device buffer of
 * ring_edges edges of etype; h_ring: host buffer of the same size, page-locked
 * for full speed (both caller-owned; ring_edges >= 2).  An item with more edges
 * than half the ring returns CL_ERR_CAPACITY.  SYNCHRONOUS; refuses
 * CL_PART_RRP plans.  Staged plans copy from the staging pool (items whose
 * slot lies beyond the pool are regenerated), so a plan built with no_stage or
 * a capped pool (cl_tuning.max_pool_entries) suits graphs whose staging would not fit. */
typedef int32_t (*cl_edge_sink)(void* user, const void* h_edges, int64_t first_edge, int64_t n_edges,
                                int64_t item_begin, int64_t item_end);
cl_status cl_generate_stream(cl_plan* plan, int32_t etype, void* h_ring, void* d_ring, int64_t ring_edges,
                             int32_t* d_counts, int64_t* d_offsets, cl_edge_sink sink, void* user,
                             int64_t* h_total, cl_stream_t stream);

/* --- expected degrees and weight calibration (Section 3: E[d_i] = w_i - w_i^2/S
 *     without capping; with the cap min(1, .) of Algorithm 1,
 *     E_u = sum_{v != u} min(1, w_u w_v / S), S = sum w) ----------------------
 * Weights are doubles sorted non-increasing (CL_W_F64 convention: the pair is
 * capped iff fl(w_u w_v) >= S).  S <= 0 means "compute S = sum w on the device
 * (double-double, rounded once)"; the call then synchronizes to read it. */
typedef struct {
  double tol;          /* stop when max_u |E_u - d_u| / d_u <= tol; 0 = 1e-9 */
  int32_t max_iter;    /* 0 = 100 */
  int32_t init_from_w; /* 1: start from the weights in d_w; 0: start from the targets */
} cl_calib_opts;

typedef struct {
  int32_t iterations;  /* gradient steps taken */
  double max_rel_err;  /* max_u |E_u - d_u| / d_u at the returned weights */
  double S;            /* sum of the returned weights */
} cl_calib_report;

size_t cl_expected_degree_workspace_bytes(int64_t n);
/* d_E[u] = E_u for the n weights d_w (device arrays of n doubles). */
cl_status cl_expected_degree(const double* d_w, int64_t n, double S, double* d_E, void* d_ws, size_t ws_bytes,
                             cl_stream_t stream);
/* d_gw = gradient of L = sum_u d_gE[u] E_u(w) with respect to w, S = sum w included:
 * d_gw[k] = [gE_k A_k + sum_{u != k, (u,k) uncapped} gE_u w_u - K] / S with
 * A_u = sum_{v != u, uncapped} w_v and K = sum_u gE_u (w_u / S) A_u. */
cl_status cl_expected_degree_adjoint(const double* d_w, const double* d_gE, int64_t n, double S, double* d_gw,
                                     void* d_ws, size_t ws_bytes, cl_stream_t stream);
size_t cl_calibrate_workspace_bytes(int64_t n);
/* Fits d_w so that E(w) matches the target degrees d_target (n doubles, sorted
 * non-increasing, positive) by preconditioned gradient descent on
 * L = sum_u (E_u - d_u)^2 / d_u: each step w <- w - g / H with g = dL/dw (the
 * adjoint above) and the diagonal Gauss-Newton preconditioner
 * H_u = 2 (dE_u/dw_u)^2 / d_u, dE_u/dw_u = A_u / S; w is kept positive and
 * non-increasing.  SYNCHRONIZING (one read-back per step).  Returns CL_OK when
 * max relative error <= tol, else CL_ERR_RANGE with the best weights reached. */
cl_status cl_calibrate(const double* d_target, int64_t n, double* d_w, const cl_calib_opts* opts,
                       cl_calib_report* report, void* d_ws, size_t ws_bytes, cl_stream_t stream);

/* Work counters of Algorithm 1's loop (Section 3; Eq. 1 models an item's work
 * as its edges + 1, the realized work is its loop iterations):
 * SYNCHRONIZING: the run statistics of the last cl_count (flagged skips) and
 * the device error word; resets the counters. */
cl_status cl_stats(cl_plan* plan, cl_run_stats* out, cl_stream_t stream);

/* SYNCHRONIZING: returns the device error word as a status and clears it. */
cl_status cl_check(cl_plan* plan, cl_stream_t stream);

void cl_plan_destroy(cl_plan* plan);

/* --- for callers that cannot allocate device memory ----------------------
 * The paper has no counterpart to this entry point: it exists for code that
 * cannot call cudaMalloc -- a host callback or real-time loop that must not
 * take cudaMalloc's implicit device synchronisation, a plug-in whose host
 * framework owns all device memory, a fixed memory budget.
 *
 * cl_scan_noalloc computes exactly what cl_scan computes (d_offsets[i] =
 * sum_{k<i} d_counts[k] for i = 0..n, d_offsets[n] = total, int64) without a
 * plan or workspace and without allocating: its scratch (one int64 per 2048
 * counts) is a fixed 1 MiB array inside the library, held on every GPU that
 * loads the library until the process exits.  n must be <= 2^28
 * (268,435,456); larger n returns CL_ERR_RANGE.  Every call looks up that
 * array's device address on the current device (so a cudaDeviceReset between
 * calls is harmless); the first call on a device also loads the library's
 * device code there, so make it before any stream capture.  All calls share the one array
 * (its contents are rewritten by each call, nothing needs clearing), so two
 * calls that may run at the same time on the GPU -- on different streams, or
 * from different host threads -- race and corrupt each other's result:
 * serialise them.  Asynchronous on `stream`; d_counts and d_offsets are
 * caller-owned device arrays of n and n + 1 entries and must not overlap.
 * Errors: CL_ERR_INVALID_ARG, CL_ERR_RANGE, CL_ERR_CUDA (as for every call of
 * this library, the launch check reads and clears the calling thread's last
 * CUDA error, so an error left pending by earlier, unrelated work is reported
 * here too). */
cl_status cl_scan_noalloc(const int32_t* d_counts, int64_t n, int64_t* d_offsets, cl_stream_t stream);

/* --- diagnostics (exercise one primitive over arrays; for tests) ---------- */

/* d_out[4i..4i+3] = Philox4x32-10(counter d_ctr[4i..4i+3], key (seed_lo, seed_hi)). */
cl_status cl_diag_philox(const uint32_t* d_ctr, int64_t count, uint64_t seed, uint32_t* d_out,
                         cl_stream_t stream);
/* Same with NVIDIA cuRAND's device Philox4x32-10 (an independent implementation). */
cl_status cl_diag_philox_curand(const uint32_t* d_ctr, int64_t count, uint64_t seed, uint32_t* d_out,
                                cl_stream_t stream);
/* -ln(A_i / B_i) for integers 1 <= A_i < B_i <= 2^55: d_ff[2i..2i+1] = float-float
 * (hi, lo); d_dd[2i..2i+1] = double-double (hi, lo). */
cl_status cl_diag_neglog(const uint64_t* d_A, const uint64_t* d_B, int64_t count, float* d_ff, double* d_dd,
                         cl_stream_t stream);
/* Skip of Algorithm 1 for r = (2 a_i + 1)/2^53, p = Q_i / S_i, remaining length R_i:
 * d_delta[i] = min(floor(ln r / ln(1 - p)), R_i) (integer weights, 0 < Q_i < S_i < 2^53);
 * d_tier[i] = 0 (float-float decided), 1 (double-double decided), 2 (tie: nearest integer). */
cl_status cl_diag_skip(const uint64_t* d_a, const uint64_t* d_Q, const uint64_t* d_S, const int64_t* d_R,
                       int64_t count, int64_t* d_delta, int32_t* d_tier, cl_stream_t stream);

/* -ln(1 - Q_i / S_i) for doubles 0 < Q_i < S_i, evaluated as the sampler does for
 * double weights (float-float from the doubles): d_ff[2i..2i+1] = (hi, lo); NaN
 * outside the domain. */
cl_status cl_diag_neglog1m_f64(const double* d_Q, const double* d_S, int64_t count, float* d_ff,
                               cl_stream_t stream);

/* Throughput of the sampler's random stream on this GPU: Philox4x32-10 blocks
 * per second (into *blocks_per_s) over a grid of resident blocks, each thread
 * running `iters` dependent blocks.  One block is drawn per loop iteration of
 * Algorithm 1, so the rate is an upper bound on the sampler's iterations per
 * second (the measured peak of its arithmetic roofline).  d_sink: one
 * caller-owned device uint64 (written only by a chance match).  SYNCHRONIZING. */
cl_status cl_diag_philox_rate(int64_t iters, uint64_t seed, uint64_t* d_sink, double* blocks_per_s,
                              cl_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* CL_H */
