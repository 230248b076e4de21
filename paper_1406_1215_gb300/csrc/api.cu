// api.cu -- the C ABI (include/cl.h): plan life cycle, count / scan / emit,
// the batched path, statistics and error words.  Host code only; kernels live
// in plan.cu and sample.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <new>
#include <vector>

#include "cl_internal.cuh"
#include "philox.cuh"

using namespace cl;

struct cl_plan {
  int G = 0;
  int wtype = 0;
  int device = 0;
  int sms = 0;
  std::vector<cl_graph> graphs;
  std::vector<cl_graph_info> info;
  std::vector<DevGraph> dg;
  std::vector<long long> tile_begin;  // G + 1 prefix of weight-prefix tiles
  long long ntiles = 0;
  long long n_items = 0;
  long long psize = 0;  // sum of (n_g + 1)
  long long csize = 0;  // sum of ceil(n_g / 4096): uniform-block table entries
  int T = 1;
  int block = 256;
  int grid_count = 0, grid_emit32 = 0, grid_emit64 = 0;
  long long max_n = 0;
  bool stage = true;                  // cl_count stages destinations
  unsigned long long pool_cap = 0;    // staging pool entries
  bool staged = false;                // the last cl_count staged (cl_emit copies)
  bool tiny_slots = false;            // testing knob: 8-entry slots (most items regenerate)
  int partition = CL_PART_UCP;        // task split: Eq. 3 (default) or the consecutive partition
  unsigned ovf_cap = 1;               // regeneration list entries
  int copy_chunk = 32;                // items per claim of the copy kernel
  // workspace (after cl_plan_build)
  bool built = false;
  size_t ws_bytes = 0;
  DevGraph* d_graphs = nullptr;
  long long* d_tile_begin = nullptr;
  void* d_P = nullptr;
  long long* d_C = nullptr;
  long long* d_part = nullptr;
  long long* d_scan_part = nullptr;
  long long* d_task = nullptr;
  unsigned* d_ctr = nullptr;
  int* d_err = nullptr;
  unsigned long long* d_stats = nullptr;
  unsigned* d_pool = nullptr;
  int* d_slot32 = nullptr;
  long long* d_slot_base = nullptr;
  int* d_overflow = nullptr;
  long long* d_ovf_list = nullptr;
  unsigned* d_ovf_count = nullptr;
  unsigned long long* d_blk = nullptr;
  unsigned* d_snap = nullptr;  // per-chunk snapshots of the regeneration list length
  unsigned long long* d_task_ns = nullptr;  // caller's per-task clock array (nullable)
  // host-output pipeline (cl_generate_host): a second stream and its events, made on first use
  cudaStream_t side = nullptr;
  cudaStream_t aux = nullptr;  // counts the second range beside the first
  std::vector<cudaEvent_t> events;
  long long* h_ends = nullptr;  // page-locked, mapped: each chunk's edge total, for its host copy
  long long* h_sbuf = nullptr;  // page-locked, mapped: cl_generate_stream's task slot bases and pieces
  size_t h_sbuf_n = 0;
};

namespace {
constexpr unsigned OVF_CAP = 1u << 20;  // items listed for regeneration (beyond: scan all items)
}

namespace {

constexpr size_t ALIGN = 256;
size_t align_up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base((char*)b) {}
  template <typename T>
  T* take(size_t count) {
    T* p = base ? (T*)(base + off) : nullptr;
    off = align_up(off + count * sizeof(T));
    return p;
  }
};

cl_status cuda_ok(cudaError_t e) { return e == cudaSuccess ? CL_OK : CL_ERR_CUDA; }
cl_status last_ok() { return cudaGetLastError() == cudaSuccess ? CL_OK : CL_ERR_CUDA; }

bool all_same_wtype(const cl_graph* g, int G) {
  for (int i = 1; i < G; ++i)
    if (g[i].wtype != g[0].wtype) return false;
  return true;
}

// scratch of cl_plan_create
struct ScratchLayout {
  DevGraph* graphs;
  long long* blk_begin;
  double* heavy_w;
  GraphAnalysis* res;
  unsigned long long* bins;
  size_t bytes;
};

ScratchLayout scratch_layout(void* base, int G, bool f64) {
  Carver c(base);
  ScratchLayout L;
  L.graphs = c.take<DevGraph>(G);
  L.blk_begin = c.take<long long>(G + 1);
  L.heavy_w = c.take<double>(G);
  L.res = c.take<GraphAnalysis>(G);
  L.bins = f64 ? c.take<unsigned long long>(f64_bins_bytes(G) / sizeof(unsigned long long)) : nullptr;
  L.bytes = c.off;
  return L;
}

struct WsLayout {
  DevGraph* graphs;
  long long* tile_begin;
  void* P;
  long long* C;
  long long* part;
  long long* scan_part;
  long long* task;
  unsigned* ctr;
  int* err;
  unsigned long long* stats;
  int* overflow;
  int* slot32;
  long long* slot_base;
  long long* ovf_list;
  unsigned* ovf_count;
  unsigned long long* blk;
  unsigned* snap;
  unsigned* pool;
  size_t bytes;
};

WsLayout ws_layout(void* base, const cl_plan* p) {
  Carver c(base);
  WsLayout L;
  long long nt_items = scan_partials_needed(p->n_items);
  long long nt = (p->ntiles > nt_items ? p->ntiles : nt_items) + 1;
  L.graphs = c.take<DevGraph>(p->G);
  L.tile_begin = c.take<long long>(p->G + 1);
  L.P = c.take<long long>(p->psize > 0 ? p->psize : 1);  // int64 or double prefix
  L.C = c.take<long long>(p->n_items > 0 ? p->n_items : 1);
  L.part = c.take<long long>(nt);
  L.scan_part = c.take<long long>(nt_items + 1);
  L.task = c.take<long long>(p->T + 1);
  L.ctr = c.take<unsigned>(4);
  L.err = c.take<int>(4);
  L.stats = c.take<unsigned long long>(4);
  L.overflow = c.take<int>(4);
  L.slot32 = p->stage ? c.take<int>(p->n_items > 0 ? p->n_items : 1) : nullptr;
  L.slot_base = p->stage ? c.take<long long>(p->n_items + 1) : nullptr;
  L.ovf_list = p->stage ? c.take<long long>(p->ovf_cap) : nullptr;
  L.ovf_count = c.take<unsigned>(4);
  const bool runs = p->wtype == CL_W_I32;
  L.blk = runs ? c.take<unsigned long long>(p->csize > 0 ? p->csize : 1) : nullptr;
  L.snap = c.take<unsigned>(CL_HOST_MAX_CHUNKS);
  L.pool = p->stage ? c.take<unsigned>(p->pool_cap > 0 ? p->pool_cap : 1) : nullptr;
  L.bytes = c.off;
  return L;
}

DevPlan dev_plan(const cl_plan* p) {
  DevPlan P;
  P.graphs = p->d_graphs;
  P.G = p->G;
  P.n_items = p->n_items;
  P.task_start = p->d_task;
  P.T = p->T;
  P.task_ctr = p->d_ctr;
  P.err = p->d_err;
  P.stats = p->d_stats;
  P.pool = p->d_pool;
  P.slot_base = p->d_slot_base;
  P.overflow = p->d_overflow;
  P.ovf_list = p->d_ovf_list;
  P.ovf_count = p->d_ovf_count;
  P.ovf_cap = p->ovf_cap;
  P.wf64 = p->wtype == CL_W_F64 ? 1 : 0;
  P.pool_cap = p->pool_cap;
  P.blk = p->d_blk;
  P.pool_shift = 0;
  P.pool_entries = p->pool_cap;
  P.rrp = p->partition == CL_PART_RRP ? 1 : 0;
  P.task_ns = p->d_task_ns;
  P.copy_chunk = p->copy_chunk;
  return P;
}

}  // namespace

extern "C" {

const char* cl_status_string(cl_status s) {
  switch (s) {
    case CL_OK: return "ok";
    case CL_ERR_INVALID_ARG: return "invalid argument";
    case CL_ERR_UNSORTED: return "weights are not sorted non-increasing";
    case CL_ERR_NONFINITE: return "a weight is negative, NaN or infinite";
    case CL_ERR_RANGE: return "size or value out of the supported range";
    case CL_ERR_CAPACITY: return "output buffer too small";
    case CL_ERR_WORKSPACE: return "scratch or workspace too small";
    case CL_ERR_TIMEOUT: return "device wait expired";
    case CL_ERR_CUDA: return "CUDA runtime error";
    case CL_ERR_STATE: return "call order violated";
    case CL_ERR_DEVICE: return "device-side consistency check failed";
    case CL_ERR_STOPPED: return "the caller's edge sink asked to stop";
  }
  return "unknown status";
}

size_t cl_plan_scratch_bytes(int32_t G) {
  if (G <= 0) return 0;
  return scratch_layout(nullptr, G, true).bytes;  // large enough for either weight type
}

cl_status cl_plan_create(const cl_graph* graphs, int32_t G, const cl_tuning* tuning, void* d_scratch,
                         size_t scratch_bytes, cl_stream_t stream, cl_plan** out) {
  if (!out) return CL_ERR_INVALID_ARG;
  *out = nullptr;
  if (!graphs || G <= 0) return CL_ERR_INVALID_ARG;
  if (!all_same_wtype(graphs, G)) return CL_ERR_INVALID_ARG;
  const int wtype = graphs[0].wtype;
  if (wtype != CL_W_I32 && wtype != CL_W_F64) return CL_ERR_INVALID_ARG;
  for (int g = 0; g < G; ++g) {
    if (graphs[g].n < 0) return CL_ERR_INVALID_ARG;
    if (graphs[g].n > 0 && !graphs[g].d_w) return CL_ERR_INVALID_ARG;
    if (graphs[g].n >= (1ll << 31)) return CL_ERR_RANGE;
    if (std::isnan(graphs[g].heavy_w)) return CL_ERR_INVALID_ARG;
  }
  const bool f64 = wtype == CL_W_F64;
  ScratchLayout SL = scratch_layout(d_scratch, G, f64);
  if (!d_scratch || scratch_bytes < SL.bytes) return CL_ERR_WORKSPACE;
  if (((uintptr_t)d_scratch & (ALIGN - 1)) != 0) return CL_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;

  cl_plan* p = new (std::nothrow) cl_plan();
  if (!p) return CL_ERR_INVALID_ARG;
  p->G = G;
  p->wtype = wtype;
  p->graphs.assign(graphs, graphs + G);
  p->info.resize(G);
  p->dg.resize(G);
  cudaGetDevice(&p->device);
  cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device);

  // analysis: one block per 4096 weights of each graph
  std::vector<long long> blk(G + 1, 0);
  std::vector<double> hw(G);
  for (int g = 0; g < G; ++g) {
    DevGraph& d = p->dg[g];
    std::memset(&d, 0, sizeof(d));
    d.w = graphs[g].d_w;
    d.n = graphs[g].n;
    d.wtype = wtype;
    d.key0 = (unsigned)graphs[g].seed;
    d.key1 = (unsigned)(graphs[g].seed >> 32);
    round_keys(d.key0, d.key1, d.rk);
    blk[g + 1] = blk[g] + (graphs[g].n + ANALYZE_CHUNK_HOST - 1) / ANALYZE_CHUNK_HOST;
    hw[g] = graphs[g].heavy_w;
  }
  cl_status st = CL_OK;
  std::vector<GraphAnalysis> res(G);
  do {
    if ((st = cuda_ok(cudaMemcpyAsync(SL.graphs, p->dg.data(), sizeof(DevGraph) * G, cudaMemcpyHostToDevice, s))))
      break;
    if ((st = cuda_ok(cudaMemcpyAsync(SL.blk_begin, blk.data(), sizeof(long long) * (G + 1), cudaMemcpyHostToDevice,
                                      s))))
      break;
    if ((st = cuda_ok(cudaMemcpyAsync(SL.heavy_w, hw.data(), sizeof(double) * G, cudaMemcpyHostToDevice, s)))) break;
    if ((st = cuda_ok(cudaMemsetAsync(SL.res, 0, sizeof(GraphAnalysis) * G, s)))) break;
    if (f64 && (st = cuda_ok(cudaMemsetAsync(SL.bins, 0, f64_bins_bytes(G), s)))) break;
    launch_analyze(SL.graphs, SL.blk_begin, G, blk[G], SL.heavy_w, SL.res, SL.bins, f64, s);
    if (f64) launch_f64_sum_finalize(G, SL.bins, SL.res, s);
    if ((st = last_ok())) break;
    if ((st = cuda_ok(cudaMemcpyAsync(res.data(), SL.res, sizeof(GraphAnalysis) * G, cudaMemcpyDeviceToHost, s))))
      break;
    if ((st = cuda_ok(cudaStreamSynchronize(s)))) break;
  } while (0);
  if (st != CL_OK) {
    delete p;
    return st;
  }

  // item space and per-graph status
  cl_status first_bad = CL_OK;
  long long items = 0, pbase = 0, cbase = 0;
  p->tile_begin.assign(G + 1, 0);
  for (int g = 0; g < G; ++g) {
    DevGraph& d = p->dg[g];
    cl_graph_info& I = p->info[g];
    const long long n = graphs[g].n;
    cl_status gs = CL_OK;
    if (res[g].flags & 2u)
      gs = CL_ERR_NONFINITE;
    else if (res[g].flags & 1u)
      gs = CL_ERR_UNSORTED;
    if (f64) {
      d.S_i = 0;
      d.S_d = res[g].S_d;
      d.lpd = lp_const_d(d.S_d);  // for the per-candidate -ln(1 - p) in float-float
      if (gs == CL_OK && !std::isfinite(d.S_d)) gs = CL_ERR_NONFINITE;
    } else {
      d.S_i = (long long)res[g].S_i;
      d.S_d = (double)d.S_i;
      d.lp = lp_const((unsigned long long)d.S_i);  // for the per-candidate -ln(1 - p)
      if (gs == CL_OK && res[g].S_i >= (1ull << 53)) gs = CL_ERR_RANGE;
    }
    d.invS_f = d.S_d > 0 ? (float)(1.0 / d.S_d) : 0.0f;
    d.H = (long long)res[g].H;
    d.Hh = d.H < n - 1 ? d.H : (n > 0 ? n - 1 : 0);
    d.n_heavy = d.Hh > 0 ? heavy_items_before(d.Hh, n) : 0;
    long long light = n - 1 - d.H;
    d.n_items = d.n_heavy + (light > 0 ? light : 0);
    if (gs != CL_OK) d.n_items = 0, d.n_heavy = 0;
    d.item_begin = items;
    d.pbase = pbase;
    d.bbase = cbase;
    cbase += (n + (1ll << BLK_SHIFT) - 1) >> BLK_SHIFT;
    items += d.n_items;
    pbase += n + 1;
    p->tile_begin[g + 1] = p->tile_begin[g] + (n + 1 + SCAN_TILE_HOST - 1) / SCAN_TILE_HOST;
    if (n > p->max_n) p->max_n = n;
    I.n = n;
    I.H = d.H;
    I.n_items = d.n_items;
    I.item_begin = d.item_begin;
    I.S_i64 = d.S_i;
    I.S = d.S_d;
    I.status = gs;
    if (gs != CL_OK && first_bad == CL_OK) first_bad = gs;
  }
  if (first_bad != CL_OK) {
    delete p;
    return first_bad;
  }
  p->n_items = items;
  p->psize = pbase;
  p->csize = cbase;
  p->ntiles = p->tile_begin[G];

  // launch shape (performance knobs only)
  p->block = (tuning && tuning->block > 0) ? tuning->block : 256;
  if (p->block % 32 != 0 || p->block > 256) {
    delete p;
    return CL_ERR_INVALID_ARG;
  }
  int bps_c = sampler_max_blocks_per_sm(p->block, false, 0);
  int bps_e32 = sampler_max_blocks_per_sm(p->block, true, CL_E_I32);
  int bps_e64 = sampler_max_blocks_per_sm(p->block, true, CL_E_I64);
  if (tuning && tuning->blocks_per_sm > 0) {
    bps_c = bps_c < tuning->blocks_per_sm ? bps_c : tuning->blocks_per_sm;
    bps_e32 = bps_e32 < tuning->blocks_per_sm ? bps_e32 : tuning->blocks_per_sm;
    bps_e64 = bps_e64 < tuning->blocks_per_sm ? bps_e64 : tuning->blocks_per_sm;
  }
  p->grid_count = p->sms * (bps_c > 0 ? bps_c : 1);
  p->grid_emit32 = p->sms * (bps_e32 > 0 ? bps_e32 : 1);
  p->grid_emit64 = p->sms * (bps_e64 > 0 ? bps_e64 : 1);
  long long warps = (long long)p->grid_count * (p->block / 32);
  // staging pool: item slots of e_i + 6 sqrt(e_i) + 6 entries (rounded up to 8), e_i the
  // uncapped expected edges of item i, sum_i e_i = (S^2 - sum w^2) / (2 S); by
  // Cauchy-Schwarz sum_i sqrt(e_i) <= sqrt(items * sum_i e_i), so this bounds the pool
  p->stage = !(tuning && tuning->no_stage);
  p->tiny_slots = tuning && tuning->stage_factor < 0;
  p->partition = tuning ? tuning->partition : CL_PART_UCP;
  if (p->partition != CL_PART_UCP && p->partition != CL_PART_CP && p->partition != CL_PART_RRP) {
    delete p;
    return CL_ERR_INVALID_ARG;
  }
  p->ovf_cap = (unsigned)(items < (long long)OVF_CAP ? (items > 0 ? items : 1) : OVF_CAP);
  double em = 0;  // uncapped expected edges of the plan
  for (int g = 0; g < G; ++g) {
    double S = p->dg[g].S_d;
    if (S > 0) em += (S * S - res[g].S2) / (2.0 * S);
  }
  if (em < 0) em = 0;
  // copy claims: 32 items, or 256 when items average under 8 edges (so that a claim
  // still holds a few hundred edges and the claim counter is not the bottleneck)
  p->copy_chunk = items > 0 && em < 8.0 * (double)items ? 256 : 32;
  if (p->stage) {
    // slots are ceil8(e + 6 sqrt(e) + 6) <= e + 6 sqrt(e) + 13 with e the item's uncapped expected
    // edges (sum em; Cauchy-Schwarz bounds the square roots); 2^-10 em covers the FP32 costs
    double cap = em * (1.0 + 0x1p-10) + 6.0 * std::sqrt((double)items * em) + 14.0 * (double)items + 1024.0;
    p->pool_cap = (unsigned long long)cap;
    if (tuning && tuning->max_pool_entries > 0 && p->pool_cap > (unsigned long long)tuning->max_pool_entries)
      p->pool_cap = (unsigned long long)tuning->max_pool_entries;
  }
  // default task count: tasks of about 10^4 edges of cost (Eq. 1 with the per-item
  // constant 4), between 4 and 64 per resident warp -- fewer, larger tasks cost less
  // to hand out on small graphs (n = 10^7: 9.6 against 10.5 ms per count pass), and
  // 64 per warp keeps the end of a large pass short
  long long T = 64 * warps;
  if (tuning && tuning->tasks > 0) {
    T = tuning->tasks;
  } else {
    double want = (em + 4.0 * (double)items) / 1e4;
    if (want < 4.0 * (double)warps) want = 4.0 * (double)warps;
    if (want < (double)T) T = (long long)want;
  }
  long long cap = (items + 31) / 32;
  if (T > cap) T = cap;
  if (T < 1) T = 1;
  if (T > (1ll << 30)) T = 1ll << 30;
  p->T = (int)T;
  *out = p;
  return CL_OK;
}

cl_status cl_plan_workspace_bytes(const cl_plan* plan, size_t* bytes) {
  if (!plan || !bytes) return CL_ERR_INVALID_ARG;
  *bytes = ws_layout(nullptr, plan).bytes;
  return CL_OK;
}

cl_status cl_plan_build(cl_plan* p, void* d_ws, size_t ws_bytes, cl_stream_t stream) {
  if (!p) return CL_ERR_INVALID_ARG;
  WsLayout L = ws_layout(d_ws, p);
  if (!d_ws || ws_bytes < L.bytes) return CL_ERR_WORKSPACE;
  // every array carved from it keeps the base's alignment: the staging pool needs its
  // 32-byte slot boundaries for the sampler's 16-byte stores and the copy's 16-byte chunks
  if (((uintptr_t)d_ws & (ALIGN - 1)) != 0) return CL_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  p->ws_bytes = ws_bytes;
  p->d_graphs = L.graphs;
  p->d_tile_begin = L.tile_begin;
  p->d_P = L.P;
  p->d_C = L.C;
  p->d_part = L.part;
  p->d_scan_part = L.scan_part;
  p->d_task = L.task;
  p->d_ctr = L.ctr;
  p->d_err = L.err;
  p->d_stats = L.stats;
  p->d_pool = L.pool;
  p->d_slot32 = L.slot32;
  p->d_slot_base = L.slot_base;
  p->d_overflow = L.overflow;
  p->d_ovf_list = L.ovf_list;
  p->d_ovf_count = L.ovf_count;
  p->d_blk = L.blk;
  p->d_snap = L.snap;
  for (int g = 0; g < p->G; ++g) p->dg[g].blkp = L.blk ? L.blk + p->dg[g].bbase : nullptr;
  cl_status st;
  if ((st = cuda_ok(cudaMemcpyAsync(L.graphs, p->dg.data(), sizeof(DevGraph) * p->G, cudaMemcpyHostToDevice, s))))
    return st;
  if ((st = cuda_ok(cudaMemcpyAsync(L.tile_begin, p->tile_begin.data(), sizeof(long long) * (p->G + 1),
                                    cudaMemcpyHostToDevice, s))))
    return st;
  if ((st = cuda_ok(cudaMemsetAsync(L.ctr, 0, 4 * sizeof(unsigned) + 0, s)))) return st;
  if ((st = cuda_ok(cudaMemsetAsync(L.err, 0, 4 * sizeof(int), s)))) return st;
  if ((st = cuda_ok(cudaMemsetAsync(L.stats, 0, 4 * sizeof(unsigned long long), s)))) return st;
  if ((st = cuda_ok(cudaMemsetAsync(L.overflow, 0, 4 * sizeof(int), s)))) return st;
  if ((st = cuda_ok(cudaMemsetAsync(L.ovf_count, 0, 4 * sizeof(unsigned), s)))) return st;
  const bool f64 = p->wtype == CL_W_F64;
  launch_weight_prefix(L.graphs, L.tile_begin, p->G, p->ntiles, f64, L.P, L.part, s);
  if (!f64) launch_blocks(L.graphs, p->G, p->csize, L.blk, s);
  long long n_nodes = 0;
  for (int g = 0; g < p->G; ++g) n_nodes += p->dg[g].n;
  launch_costs_and_tasks(L.graphs, p->G, p->n_items, f64, L.P, L.C, L.part, L.task, p->T, L.slot32,
                         p->tiny_slots ? 1 : 0, p->partition, n_nodes, s);
  if (p->stage) launch_count_scan(L.slot32, p->n_items, L.slot_base, L.scan_part, s);  // slot bases
  if ((st = last_ok())) return st;
  p->built = true;
  return CL_OK;
}

cl_status cl_plan_items(const cl_plan* plan, int64_t* n_items) {
  if (!plan || !n_items) return CL_ERR_INVALID_ARG;
  *n_items = plan->n_items;
  return CL_OK;
}

cl_status cl_plan_tasks(const cl_plan* p, int32_t* T, int64_t* d_task_start, int64_t* d_cost_prefix,
                        cl_stream_t stream) {
  if (!p || !T) return CL_ERR_INVALID_ARG;
  *T = p->T;
  if (!d_task_start && !d_cost_prefix) return CL_OK;
  if (!p->built) return CL_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  cl_status st;
  if (d_task_start &&
      (st = cuda_ok(cudaMemcpyAsync(d_task_start, p->d_task, sizeof(int64_t) * (p->T + 1), cudaMemcpyDeviceToDevice,
                                    s))))
    return st;
  if (d_cost_prefix && p->n_items > 0 &&
      (st = cuda_ok(cudaMemcpyAsync(d_cost_prefix, p->d_C, sizeof(int64_t) * p->n_items, cudaMemcpyDeviceToDevice,
                                    s))))
    return st;
  return CL_OK;
}

cl_status cl_plan_task_clock(cl_plan* p, uint64_t* d_task_ns) {
  if (!p) return CL_ERR_INVALID_ARG;
  p->d_task_ns = (unsigned long long*)d_task_ns;
  return CL_OK;
}

cl_status cl_plan_launch_info(const cl_plan* p, int32_t* count_grid, int32_t* block) {
  if (!p || !count_grid || !block) return CL_ERR_INVALID_ARG;
  *count_grid = p->grid_count;
  *block = p->block;
  return CL_OK;
}

cl_status cl_plan_graph_info(const cl_plan* plan, int32_t g, cl_graph_info* out) {
  if (!plan || !out || g < 0 || g >= plan->G) return CL_ERR_INVALID_ARG;
  *out = plan->info[g];
  return CL_OK;
}

cl_status cl_count(cl_plan* p, int32_t* d_counts, cl_stream_t stream) {
  if (!p || (!d_counts && p->n_items > 0)) return CL_ERR_INVALID_ARG;
  if (!p->built) return CL_ERR_STATE;
  if (p->n_items == 0) return CL_OK;
  cudaStream_t s = (cudaStream_t)stream;
  cudaMemsetAsync(p->d_stats, 0, 4 * sizeof(unsigned long long), s);
  launch_count(dev_plan(p), p->G == 1 ? &p->dg[0] : nullptr, d_counts, p->stage, p->block, p->grid_count, s);
  p->staged = p->stage;
  return last_ok();
}

cl_status cl_scan(cl_plan* p, const int32_t* d_counts, int64_t* d_offsets, int64_t* h_total, cl_stream_t stream) {
  if (!p || !d_offsets || (!d_counts && p->n_items > 0)) return CL_ERR_INVALID_ARG;
  if (!p->built) return CL_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  launch_count_scan(d_counts, p->n_items, (long long*)d_offsets, p->d_scan_part, s);
  cl_status st = last_ok();
  if (st != CL_OK || !h_total) return st;
  int err = 0;
  if ((st = cuda_ok(cudaMemcpyAsync(h_total, d_offsets + p->n_items, sizeof(int64_t), cudaMemcpyDeviceToHost, s))))
    return st;
  if ((st = cuda_ok(cudaMemcpyAsync(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, s)))) return st;
  if ((st = cuda_ok(cudaStreamSynchronize(s)))) return st;
  return err ? CL_ERR_DEVICE : CL_OK;
}

cl_status cl_emit(cl_plan* p, const int64_t* d_offsets, int32_t etype, void* d_edges, int64_t capacity,
                  int64_t item_begin, int64_t item_end, cl_stream_t stream) {
  if (!p || !d_offsets || capacity < 0) return CL_ERR_INVALID_ARG;
  if (etype != CL_E_I32 && etype != CL_E_I64) return CL_ERR_INVALID_ARG;
  if (item_begin < 0 || item_end < item_begin || item_end > p->n_items) return CL_ERR_INVALID_ARG;
  if (capacity > 0 && !d_edges) return CL_ERR_INVALID_ARG;
  if (!p->built) return CL_ERR_STATE;
  if (item_end == item_begin) return CL_OK;
  cudaStream_t s = (cudaStream_t)stream;
  launch_emit(dev_plan(p), p->G == 1 ? &p->dg[0] : nullptr, (const long long*)d_offsets,
              SampleRange{item_begin, item_end, 0, item_begin}, etype, d_edges, capacity, p->staged, p->block,
              etype == CL_E_I32 ? p->grid_emit32 : p->grid_emit64, 0, s);
  return last_ok();
}

cl_status cl_generate(cl_plan* p, int32_t etype, void* d_edges, int64_t capacity, int32_t* d_counts,
                      int64_t* d_offsets, int64_t* h_total, cl_stream_t stream) {
  if (!p || !d_offsets || capacity < 0) return CL_ERR_INVALID_ARG;
  if (etype != CL_E_I32 && etype != CL_E_I64) return CL_ERR_INVALID_ARG;
  if (p->n_items > 0 && !d_counts) return CL_ERR_INVALID_ARG;
  if (capacity > 0 && !d_edges) return CL_ERR_INVALID_ARG;
  if (!p->built) return CL_ERR_STATE;
  cl_status st;
  if ((st = cl_count(p, d_counts, stream))) return st;
  if ((st = cl_scan(p, d_counts, d_offsets, nullptr, stream))) return st;
  if (p->n_items > 0 && (st = cl_emit(p, d_offsets, etype, d_edges, capacity, 0, p->n_items, stream))) return st;
  if (!h_total) return CL_OK;
  cudaStream_t s = (cudaStream_t)stream;
  int err = 0;
  if ((st = cuda_ok(cudaMemcpyAsync(h_total, d_offsets + p->n_items, sizeof(int64_t), cudaMemcpyDeviceToHost, s))))
    return st;
  if ((st = cuda_ok(cudaMemcpyAsync(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, s)))) return st;
  if ((st = cuda_ok(cudaStreamSynchronize(s)))) return st;
  if (*h_total > capacity) return CL_ERR_CAPACITY;
  return err ? (cl_status)err : CL_OK;
}

cl_status cl_generate_batch(cl_plan* p, int32_t etype, void* d_edges, int64_t capacity, int64_t* d_graph_offsets,
                            int32_t* d_counts, int64_t* d_offsets, int32_t* d_status, cl_stream_t stream) {
  if (!p || !d_graph_offsets || !d_offsets || !d_status || capacity < 0) return CL_ERR_INVALID_ARG;
  if (etype != CL_E_I32 && etype != CL_E_I64) return CL_ERR_INVALID_ARG;
  if (p->n_items > 0 && !d_counts) return CL_ERR_INVALID_ARG;
  if (capacity > 0 && !d_edges) return CL_ERR_INVALID_ARG;
  if (!p->built) return CL_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  cl_status st;
  if ((st = cl_count(p, d_counts, stream))) return st;
  if ((st = cl_scan(p, d_counts, d_offsets, nullptr, stream))) return st;
  launch_graph_offsets(p->d_graphs, p->G, (const long long*)d_offsets, p->n_items, (long long*)d_graph_offsets,
                       capacity, d_status, s);
  if ((st = last_ok())) return st;
  if (p->n_items == 0) return CL_OK;
  launch_emit(dev_plan(p), p->G == 1 ? &p->dg[0] : nullptr, (const long long*)d_offsets,
              SampleRange{0, p->n_items, 0, 0}, etype, d_edges, capacity, p->staged, p->block,
              etype == CL_E_I32 ? p->grid_emit32 : p->grid_emit64, 0, s);
  return last_ok();
}

cl_status cl_stats(cl_plan* p, cl_run_stats* out, cl_stream_t stream) {
  if (!p || !out) return CL_ERR_INVALID_ARG;
  if (!p->built) return CL_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long st[4] = {0, 0, 0, 0};
  int err = 0;
  cl_status r;
  if ((r = cuda_ok(cudaMemcpyAsync(st, p->d_stats, sizeof(st), cudaMemcpyDeviceToHost, s)))) return r;
  if ((r = cuda_ok(cudaMemcpyAsync(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, s)))) return r;
  if ((r = cuda_ok(cudaStreamSynchronize(s)))) return r;
  out->iterations = (int64_t)st[0];
  out->fallbacks = (int64_t)st[1];
  out->ties = (int64_t)st[2];
  out->error = err;
  cudaMemsetAsync(p->d_err, 0, sizeof(int), s);
  return cuda_ok(cudaStreamSynchronize(s));
}

cl_status cl_check(cl_plan* p, cl_stream_t stream) {
  if (!p) return CL_ERR_INVALID_ARG;
  if (!p->built) return CL_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  int err = 0;
  cl_status r;
  if ((r = cuda_ok(cudaMemcpyAsync(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, s)))) return r;
  if ((r = cuda_ok(cudaStreamSynchronize(s)))) return r;
  cudaMemsetAsync(p->d_err, 0, sizeof(int), s);
  if ((r = cuda_ok(cudaStreamSynchronize(s)))) return r;
  return (cl_status)err;
}

// The host-delivery pipeline of a plan (made on first use, freed by cl_plan_destroy):
// a copy stream, a second counting stream, `events` events and a page-locked,
// mapped array of CL_HOST_MAX_CHUNKS + 1 totals (*d_ends: its device address).
static cl_status host_pipe(cl_plan* p, int events, long long** d_ends) {
  cl_status st;
  if (!p->side && (st = cuda_ok(cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking)))) return st;
  if (!p->aux && (st = cuda_ok(cudaStreamCreateWithFlags(&p->aux, cudaStreamNonBlocking)))) return st;
  if (!p->h_ends && (st = cuda_ok(cudaHostAlloc((void**)&p->h_ends, (CL_HOST_MAX_CHUNKS + 1) * sizeof(long long),
                                                cudaHostAllocMapped))))
    return st;
  if ((st = cuda_ok(cudaHostGetDevicePointer((void**)d_ends, p->h_ends, 0)))) return st;
  while ((int)p->events.size() < events) {
    cudaEvent_t e;
    if ((st = cuda_ok(cudaEventCreateWithFlags(&e, cudaEventDisableTiming)))) return st;
    p->events.push_back(e);
  }
  return CL_OK;
}

// Reads a value a kernel stored into mapped host memory, once the event that
// follows the kernel has completed.
static long long read_mapped(const long long* h, cudaEvent_t after, cl_status* st) {
  *st = cuda_ok(cudaEventSynchronize(after));
  return *(const volatile long long*)h;
}

constexpr int STREAM_MAX_PIECES = 4096;  // pieces of one window computed at a time

// Entries of each half of the staging pool used by cl_generate_stream: a multiple of
// 8 entries (32 bytes), so that slot bases stay multiples of 8 after the shift --
// the sampler writes staged groups as aligned 16-byte stores.
static unsigned long long pool_half(const cl_plan* p) { return (p->pool_cap / 2) & ~7ull; }

// Count windows shared by cl_generate_stream and cl_generate_host: consecutive whole Eq. 3
// tasks, each counted (and staged) in one launch on the plan's counting stream into one half
// of the staging pool (alternating), scanned (continuing the offsets) and cut into pieces of at
// most `cap` edges; window w + 2 reuses the halves of window w once its emits are done.
struct Windows {
  cl_plan* p;
  cudaStream_t s, cs;
  int32_t* d_counts;
  int64_t* d_offsets;
  long long cap;
  std::vector<long long> task, win;
  long long* h_sb = nullptr;
  long long* h_pc[2] = {nullptr, nullptr};
  long long* d_pc[2] = {nullptr, nullptr};
  cudaEvent_t evCount[2], evDone[2];
  int W = 0;

  // min_windows windows at least; false with *st set on a CUDA error
  cl_status setup(int min_windows) {
    cl_status st;
    long long* d_ends = nullptr;
    if ((st = host_pipe(p, 8, &d_ends))) return st;
    const size_t need = (size_t)(p->T + 1) + 2 * (2 + 2 * (size_t)STREAM_MAX_PIECES);
    if (p->h_sbuf_n < need) {
      if (p->h_sbuf) cudaFreeHost(p->h_sbuf);
      p->h_sbuf = nullptr;
      p->h_sbuf_n = 0;
      if ((st = cuda_ok(cudaHostAlloc((void**)&p->h_sbuf, need * sizeof(long long), cudaHostAllocMapped)))) return st;
      p->h_sbuf_n = need;
    }
    long long* d_sbuf = nullptr;
    if ((st = cuda_ok(cudaHostGetDevicePointer((void**)&d_sbuf, p->h_sbuf, 0)))) return st;
    h_sb = p->h_sbuf;  // staging slot bases at the task boundaries
    // pieces of a window (launch_pieces): region 0 written on the counting stream, region 1
    // on the caller's stream (a window with more than STREAM_MAX_PIECES pieces)
    h_pc[0] = p->h_sbuf + (p->T + 1);
    h_pc[1] = h_pc[0] + 2 + 2 * STREAM_MAX_PIECES;
    d_pc[0] = d_sbuf + (p->T + 1);
    d_pc[1] = d_pc[0] + 2 + 2 * STREAM_MAX_PIECES;
    task.assign(p->T + 1, 0);
    if ((st = cuda_ok(cudaMemcpyAsync(task.data(), p->d_task, sizeof(long long) * (p->T + 1),
                                      cudaMemcpyDeviceToHost, s))))
      return st;
    if (p->stage) launch_gather_task_slots(p->d_slot_base, p->d_task, p->T, d_sbuf, s);
    if ((st = last_ok())) return st;
    if ((st = cuda_ok(cudaStreamSynchronize(s)))) return st;
    if (min_windows < 1) min_windows = 1;
    win.assign(1, 0);
    if (p->stage) {  // at most half of the pool each
      const unsigned long long H = pool_half(p);
      const unsigned long long total = (unsigned long long)h_sb[p->T];
      unsigned long long target = (total + min_windows - 1) / min_windows;
      if (target > H) target = H;
      if (target < 1) target = 1;
      long long a = 0;
      while (a < p->T) {
        long long b = a + 1;
        while (b < p->T && (unsigned long long)(h_sb[b + 1] - h_sb[a]) <= target) ++b;
        win.push_back(b);
        a = b;
      }
    } else {
      const long long q = (p->T + min_windows - 1) / min_windows;
      for (long long a = q; a < p->T; a += q) win.push_back(a);
      win.push_back(p->T);
    }
    W = (int)win.size() - 1;
    cs = p->aux;
    evCount[0] = p->events[0];
    evCount[1] = p->events[1];
    evDone[0] = p->events[2];
    evDone[1] = p->events[3];
    return CL_OK;
  }
  // the plan view of window w: pool half, regeneration-list half, separate task counters
  DevPlan view(int w, bool counting) const {
    DevPlan V = dev_plan(p);
    const int h = w & 1;
    if (p->stage) {
      const unsigned long long H = pool_half(p);
      V.pool_shift = h_sb[win[w]] - (long long)(h * H);
      V.pool_cap = (unsigned long long)(h + 1) * H;
      const unsigned half = V.ovf_cap / 2 > 0 ? V.ovf_cap / 2 : 1;
      V.ovf_list = V.ovf_list + (h ? V.ovf_cap - half : 0);
      V.ovf_cap = half;
      V.ovf_count = V.ovf_count + h;
      V.overflow = V.overflow + h;
    }
    if (counting) V.task_ctr = V.task_ctr + 2;
    return V;
  }
  long long ib(int w) const { return task[win[w]]; }
  long long ie(int w) const { return task[win[w + 1]]; }
  cl_status count(int w) {
    const long long b = ib(w), e = ie(w);
    cudaStreamWaitEvent(cs, evDone[w & 1], 0);  // the window two back (same halves) is emitted
    const DevPlan V = view(w, true);
    if (p->stage) {
      cudaMemsetAsync(V.overflow, 0, sizeof(int), cs);
      cudaMemsetAsync(V.ovf_count, 0, sizeof(unsigned), cs);
    }
    if (e > b) {
      launch_count_range(V, p->G == 1 ? &p->dg[0] : nullptr, d_counts, p->stage, SampleRange{b, e, (int)win[w], b},
                         p->block, p->grid_count, cs);
      launch_count_scan(d_counts + b, e - b, (long long*)d_offsets + b, p->d_scan_part, cs,
                        (const long long*)d_offsets + b);
    }
    launch_pieces((const long long*)d_offsets, b, e, cap, d_pc[0], STREAM_MAX_PIECES, cs);
    cudaEventRecord(evCount[w & 1], cs);
    return last_ok();
  }
  // the resets made on the caller's stream happen before the first count
  void start() {
    cudaMemsetAsync(p->d_stats, 0, 4 * sizeof(unsigned long long), s);
    cudaEventRecord(evDone[0], s);
    cudaEventRecord(evDone[1], s);
  }
  cl_status fail(cl_status r) {
    cudaStreamSynchronize(cs);
    cudaStreamSynchronize(p->side);
    cudaStreamSynchronize(s);
    return r;
  }
};

cl_status cl_generate_stream(cl_plan* p, int32_t etype, void* h_ring, void* d_ring, int64_t ring_edges,
                             int32_t* d_counts, int64_t* d_offsets, cl_edge_sink sink, void* user, int64_t* h_total,
                             cl_stream_t stream) {
  if (!p || !d_offsets || !h_total || !sink || !h_ring || !d_ring) return CL_ERR_INVALID_ARG;
  if (etype != CL_E_I32 && etype != CL_E_I64) return CL_ERR_INVALID_ARG;
  if (ring_edges < 2) return CL_ERR_INVALID_ARG;
  if (p->n_items > 0 && !d_counts) return CL_ERR_INVALID_ARG;
  if (p->partition == CL_PART_RRP) return CL_ERR_INVALID_ARG;  // windows of consecutive items need Eq. 3 or CP tasks
  if (!p->built) return CL_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  cl_status st;
  *h_total = 0;
  const long long slot = ring_edges / 2;  // edges per half of the ring
  const size_t esize = etype == CL_E_I32 ? 8 : 16;
  if ((st = cuda_ok(cudaMemsetAsync(d_offsets, 0, sizeof(int64_t), s)))) return st;
  if (p->n_items == 0) return cuda_ok(cudaStreamSynchronize(s));
  // windows of at most half the pool, at least 8, so that counting window w + 1 overlaps the
  // delivery of window w; a window's longest items run beside its other items
  Windows Wn{p, s, nullptr, d_counts, d_offsets, slot};
  if ((st = Wn.setup(8))) return st;
  const DevGraph* single = p->G == 1 ? &p->dg[0] : nullptr;
  const int grid_emit = etype == CL_E_I32 ? p->grid_emit32 : p->grid_emit64;
  cudaEvent_t evB[2] = {p->events[4], p->events[5]}, evC[2] = {p->events[6], p->events[7]};
  // a piece whose host copy is queued: handed to the sink once the copy is done
  struct Piece {
    int half;
    long long first, n, ib, ie;
  } pend{0, 0, 0, 0, 0};
  bool pending = false, stopped = false;
  long long delivered = 0, emitted = 0, k = 0;
  auto deliver = [&]() -> cl_status {
    pending = false;
    cl_status r = cuda_ok(cudaEventSynchronize(evC[pend.half]));
    if (r) return r;
    if (pend.n > 0 && sink(user, (const char*)h_ring + (size_t)pend.half * slot * esize, pend.first, pend.n, pend.ib,
                           pend.ie) != 0)
      stopped = true;
    delivered += pend.n;
    return CL_OK;
  };
  Wn.start();
  if ((st = Wn.count(0))) return Wn.fail(st);
  for (int w = 0; w < Wn.W && !stopped; ++w) {
    const long long ib = Wn.ib(w), ie = Wn.ie(w);
    if ((st = cuda_ok(cudaEventSynchronize(Wn.evCount[w & 1])))) return Wn.fail(st);
    // the window's pieces: end item and the offset there (first: the offset at ib)
    std::vector<long long> ends, ends_off;
    long long off_a = 0;
    auto read_pieces = [&](const long long* h) {
      const volatile long long* v = h;
      const long long kp = v[0];
      off_a = v[1];
      for (long long j = 0; j < kp; ++j) {
        ends.push_back((long long)v[2 + 2 * j]);
        ends_off.push_back((long long)v[3 + 2 * j]);
      }
      return kp;
    };
    read_pieces(Wn.h_pc[0]);
    if (w + 1 < Wn.W && (st = Wn.count(w + 1))) return Wn.fail(st);
    cudaStreamWaitEvent(s, Wn.evCount[w & 1], 0);  // this window's counts, offsets and staging
    const DevPlan V = Wn.view(w, false);
    long long a = ib;
    size_t next_end = 0;
    while (a < ie && !stopped) {
      if (next_end == ends.size()) {  // more pieces than computed at once: the next ones, on this stream
        launch_pieces((const long long*)d_offsets, a, ie, slot, Wn.d_pc[1], STREAM_MAX_PIECES, s);
        if ((st = last_ok())) return Wn.fail(st);
        if ((st = cuda_ok(cudaStreamSynchronize(s)))) return Wn.fail(st);
        const long long off_prev = off_a;
        if (read_pieces(Wn.h_pc[1]) == 0) return Wn.fail(CL_ERR_CAPACITY);  // one item holds more than half the ring
        off_a = off_prev;
      }
      const long long b = ends[next_end];
      const long long n_piece = ends_off[next_end] - (next_end ? ends_off[next_end - 1] : off_a);
      if (n_piece < 0 || n_piece > slot || b <= a || b > ie) return Wn.fail(CL_ERR_DEVICE);  // inconsistent pieces
      ++next_end;
      const int half = (int)(k & 1);
      void* d_half = (char*)d_ring + (size_t)half * slot * esize;
      launch_emit(V, single, (const long long*)d_offsets, SampleRange{a, b, (int)Wn.win[w], a}, etype, d_half, slot,
                  p->stage, p->block, grid_emit, 0, s);
      if ((st = last_ok())) return Wn.fail(st);
      cudaEventRecord(evB[half], s);
      cudaStreamWaitEvent(p->side, evB[half], 0);
      if (n_piece > 0 && (st = cuda_ok(cudaMemcpyAsync((char*)h_ring + (size_t)half * slot * esize, d_half,
                                                       (size_t)n_piece * esize, cudaMemcpyDeviceToHost, p->side))))
        return Wn.fail(st);
      cudaEventRecord(evC[half], p->side);
      if (pending && (st = deliver())) return Wn.fail(st);  // the previous piece, while this one travels
      pend = Piece{half, emitted, n_piece, a, b};
      pending = true;
      emitted += n_piece;
      a = b;
      ++k;
    }
    cudaEventRecord(Wn.evDone[w & 1], s);
  }
  if (pending && !stopped && (st = deliver())) return Wn.fail(st);
  if ((st = cuda_ok(cudaStreamSynchronize(p->side)))) return Wn.fail(st);
  if ((st = cuda_ok(cudaStreamSynchronize(Wn.cs)))) return Wn.fail(st);
  if ((st = cuda_ok(cudaStreamSynchronize(s)))) return st;
  p->staged = false;  // the pool now holds the last windows only
  *h_total = delivered;
  if (stopped) return CL_ERR_STOPPED;
  int err = 0;
  if ((st = cuda_ok(cudaMemcpy(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost)))) return st;
  return err ? (cl_status)err : CL_OK;
}

// cl_generate_host through a device buffer of the whole edge list: windows counted on the
// counting stream while the previous window is emitted at its final offsets and copied to host
// memory at the same place (copy engines, a second stream).
static cl_status host_windows(cl_plan* p, int32_t etype, void* h_edges, int64_t capacity, void* d_edges,
                              int32_t* d_counts, int64_t* d_offsets, int chunks, int64_t* h_total, cudaStream_t s) {
  cl_status st;
  const size_t esize = etype == CL_E_I32 ? 8 : 16;
  Windows Wn{p, s, nullptr, d_counts, d_offsets, std::numeric_limits<long long>::max()};
  if ((st = Wn.setup(chunks))) return st;
  const DevGraph* single = p->G == 1 ? &p->dg[0] : nullptr;
  const int grid_emit = etype == CL_E_I32 ? p->grid_emit32 : p->grid_emit64;
  bool over = false;
  long long total = 0;
  Wn.start();
  if ((st = Wn.count(0))) return Wn.fail(st);
  for (int w = 0; w < Wn.W; ++w) {
    if ((st = cuda_ok(cudaEventSynchronize(Wn.evCount[w & 1])))) return Wn.fail(st);
    const volatile long long* v = Wn.h_pc[0];
    const long long kp = v[0], off_b = v[1];
    const long long off_e = kp > 0 ? (long long)v[3 + 2 * (kp - 1)] : off_b;
    total = off_e;
    if (w + 1 < Wn.W && (st = Wn.count(w + 1))) return Wn.fail(st);
    if (off_e > capacity) over = true;  // the counts continue, to report m
    if (!over && off_e > off_b) {
      cudaStreamWaitEvent(s, Wn.evCount[w & 1], 0);  // this window's counts, offsets and staging
      launch_emit(Wn.view(w, false), single, (const long long*)d_offsets, SampleRange{Wn.ib(w), Wn.ie(w),
                  (int)Wn.win[w], 0}, etype, d_edges, capacity, p->stage, p->block, grid_emit, 0, s);
      if ((st = last_ok())) return Wn.fail(st);
      cudaEventRecord(p->events[4], s);
      cudaStreamWaitEvent(p->side, p->events[4], 0);
      if ((st = cuda_ok(cudaMemcpyAsync((char*)h_edges + (size_t)off_b * esize, (const char*)d_edges + off_b * esize,
                                        (size_t)(off_e - off_b) * esize, cudaMemcpyDeviceToHost, p->side))))
        return Wn.fail(st);
    }
    cudaStreamWaitEvent(s, Wn.evCount[w & 1], 0);
    cudaEventRecord(Wn.evDone[w & 1], s);
  }
  if ((st = cuda_ok(cudaStreamSynchronize(p->side)))) return Wn.fail(st);
  if ((st = cuda_ok(cudaStreamSynchronize(Wn.cs)))) return Wn.fail(st);
  if ((st = cuda_ok(cudaStreamSynchronize(s)))) return st;
  p->staged = false;
  *h_total = total;
  if (over) return CL_ERR_CAPACITY;
  int err = 0;
  if ((st = cuda_ok(cudaMemcpy(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost)))) return st;
  return err ? (cl_status)err : CL_OK;
}

cl_status cl_generate_host(cl_plan* p, int32_t etype, void* h_edges, int64_t capacity, void* d_edges,
                           int32_t* d_counts, int64_t* d_offsets, int32_t chunks, int32_t copy_sms, int64_t* h_total,
                           cl_stream_t stream) {
  if (!p || !d_offsets || !h_total || capacity < 0) return CL_ERR_INVALID_ARG;
  if (etype != CL_E_I32 && etype != CL_E_I64) return CL_ERR_INVALID_ARG;
  if (p->n_items > 0 && !d_counts) return CL_ERR_INVALID_ARG;
  if (capacity > 0 && !h_edges) return CL_ERR_INVALID_ARG;
  if (chunks < 0 || chunks > CL_HOST_MAX_CHUNKS || copy_sms < 0) return CL_ERR_INVALID_ARG;
  if (p->partition == CL_PART_RRP) return CL_ERR_INVALID_ARG;  // ranges of consecutive items need Eq. 3 or CP tasks
  if (!p->built) return CL_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  cl_status st;
  *h_total = 0;
  const bool mapped = d_edges == nullptr;  // kernels store into the host buffer itself
  void* k_edges = d_edges;                 // where the emitting kernels write
  if (mapped && capacity > 0 && cudaHostGetDevicePointer(&k_edges, h_edges, 0) != cudaSuccess) {
    cudaGetLastError();
    return CL_ERR_INVALID_ARG;  // host memory the device cannot address
  }
  if ((st = cuda_ok(cudaMemsetAsync(d_offsets, 0, sizeof(int64_t), s)))) return st;
  if (p->n_items == 0) return cuda_ok(cudaStreamSynchronize(s));
  if (!mapped)
    return host_windows(p, etype, h_edges, capacity, d_edges, d_counts, d_offsets, chunks == 0 ? 8 : chunks, h_total,
                        s);
  const int C = chunks == 0 ? 8 : (chunks > p->T ? p->T : chunks);
  long long* d_ends = nullptr;
  if ((st = host_pipe(p, C + 3, &d_ends))) return st;
  // chunk c: tasks [tc_c, tc_{c+1}) of Eq. 3 (equal cost), items [task_start[tc_c], task_start[tc_{c+1}])
  std::vector<int> tc(C + 1);
  std::vector<long long> ic(C + 1);
  for (int c = 0; c <= C; ++c) tc[c] = (int)((long long)p->T * c / C);
  for (int c = 0; c < C; ++c)
    if ((st = cuda_ok(cudaMemcpyAsync(&ic[c], p->d_task + tc[c], sizeof(long long), cudaMemcpyDeviceToHost, s))))
      return st;
  if ((st = cuda_ok(cudaStreamSynchronize(s)))) return st;
  ic[C] = p->n_items;
  const DevGraph* single = p->G == 1 ? &p->dg[0] : nullptr;
  // The first two ranges are counted side by side, each on half of the counting
  // grid: the heaviest items (the first segments of the heaviest rows) bound a
  // range's count from below by their serial length, and the first host copy
  // waits for them; counted one after the other, the second range's heavy items
  // would start only once the first range is done.  The second range (stream
  // aux) keeps its own task counter and regeneration list.
  const bool lead = C >= 2;
  DevPlan P = dev_plan(p);
  DevPlan Pa = P;
  if (lead) {
    Pa.task_ctr = P.task_ctr + 2;
    if (p->stage) {
      const unsigned half = P.ovf_cap / 2;
      Pa.ovf_count = P.ovf_count + 1;
      Pa.ovf_list = P.ovf_list + (P.ovf_cap - half);
      Pa.ovf_cap = half;
      P.ovf_cap -= half;
    }
  }
  const size_t esize = etype == CL_E_I32 ? 8 : 16;
  const int grid_emit = etype == CL_E_I32 ? p->grid_emit32 : p->grid_emit64;
  // zero-copy path: the counting launch leaves `reserve` SMs to the host stores
  int reserve = copy_sms == 0 ? (p->sms >= 32 ? 16 : p->sms / 2) : copy_sms;
  if (reserve >= p->sms) reserve = p->sms - 1;
  if (reserve < 1) reserve = 1;
  const int bps = p->grid_count / (p->sms > 0 ? p->sms : 1) > 0 ? p->grid_count / p->sms : 1;
  const int grid_count = mapped ? bps * (p->sms - reserve) : p->grid_count;
  const int grid_side = bps * reserve;
  cudaMemsetAsync(p->d_stats, 0, 4 * sizeof(unsigned long long), s);
  if (p->stage) {
    cudaMemsetAsync(P.overflow, 0, sizeof(int), s);
    cudaMemsetAsync(P.ovf_count, 0, 2 * sizeof(unsigned), s);
  }
  if (lead) {
    cudaEventRecord(p->events[C + 1], s);  // the resets above, before the aux stream's count
    cudaStreamWaitEvent(p->aux, p->events[C + 1], 0);
    const int gh = grid_count / 2 > 0 ? grid_count / 2 : 1;
    if (ic[0] < ic[1])
      launch_count_range(P, single, d_counts, p->stage, SampleRange{ic[0], ic[1], tc[0], ic[0]}, p->block, gh, s);
    if (ic[1] < ic[2])
      launch_count_range(Pa, single, d_counts, p->stage, SampleRange{ic[1], ic[2], tc[1], ic[1]}, p->block,
                         grid_count - gh, p->aux);
    cudaEventRecord(p->events[C + 2], p->aux);
  }
  bool over = false;
  // copy-engine path: once chunk c's edges are in device memory, its host copy is queued on the side stream
  auto queue_copy = [&](int c) -> cl_status {
    cl_status r;
    if ((r = cuda_ok(cudaEventSynchronize(p->events[c])))) return r;
    const long long start = c == 0 ? 0 : p->h_ends[c - 1], end = p->h_ends[c];
    if (end > capacity) over = true;
    if (over || end <= start) return CL_OK;
    return cuda_ok(cudaMemcpyAsync((char*)h_edges + start * esize, (const char*)d_edges + start * esize,
                                   (size_t)(end - start) * esize, cudaMemcpyDeviceToHost, p->side));
  };
  for (int c = 0; c < C; ++c) {
    const long long ib = ic[c], ie = ic[c + 1];
    if (lead && c == 1) cudaStreamWaitEvent(s, p->events[C + 2], 0);  // the aux stream's count
    // the plan view of this range's count and emit: its regeneration list
    DevPlan Pc = P;
    if (lead && c == 1) {
      Pc.ovf_list = Pa.ovf_list;
      Pc.ovf_count = Pa.ovf_count;
      Pc.ovf_cap = Pa.ovf_cap;
    }
    if (ie > ib) {
      if (!(lead && c < 2))
        launch_count_range(P, single, d_counts, p->stage, SampleRange{ib, ie, tc[c], ib}, p->block, grid_count, s);
      if (mapped && p->stage)  // the regeneration list as it stands after this chunk's count
        cudaMemcpyAsync(p->d_snap + c, Pc.ovf_count, sizeof(unsigned), cudaMemcpyDeviceToDevice, s);
      launch_count_scan(d_counts + ib, ie - ib, (long long*)d_offsets + ib, p->d_scan_part, s,
                        (const long long*)d_offsets + ib);
    }
    if ((st = last_ok())) return st;
    if (mapped) {
      // this chunk's edges go out over the host link while the next chunk is counted
      cudaEventRecord(p->events[c], s);
      if (ie == ib) continue;
      cudaStreamWaitEvent(p->side, p->events[c], 0);
      DevPlan Ps = Pc;
      Ps.task_ctr = P.task_ctr + 1;  // its own work counter
      Ps.ovf_count = p->d_snap + c;
      launch_emit(Ps, single, (const long long*)d_offsets, SampleRange{ib, ie, tc[c], 0}, etype, k_edges, capacity,
                  p->stage, p->block, grid_side, grid_side, p->side);
    } else {
      if (ie > ib)
        launch_emit(Pc, single, (const long long*)d_offsets, SampleRange{ib, ie, tc[c], 0}, etype, d_edges, capacity,
                    p->stage, p->block, grid_emit, 0, s);
      // the range's total, stored by a kernel into mapped host memory: a copy-engine
      // read here would wait behind the large host copies and stall this stream
      launch_copy_i64((const long long*)d_offsets + ie, d_ends + c, s);
      cudaEventRecord(p->events[c], s);
      // the previous chunk is complete on the device by now or soon: queue its host copy
      if (c > 0 && (st = queue_copy(c - 1))) return st;
    }
    if ((st = last_ok())) return st;
  }
  if (!mapped && (st = queue_copy(C - 1))) return st;
  p->staged = p->stage;
  cudaEventRecord(p->events[C], p->side);
  cudaStreamWaitEvent(s, p->events[C], 0);
  int err = 0;
  if ((st = cuda_ok(cudaMemcpyAsync(h_total, d_offsets + p->n_items, sizeof(int64_t), cudaMemcpyDeviceToHost, s))))
    return st;
  if ((st = cuda_ok(cudaMemcpyAsync(&err, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, s)))) return st;
  if ((st = cuda_ok(cudaStreamSynchronize(s)))) return st;
  if (*h_total > capacity) return CL_ERR_CAPACITY;
  return err ? (cl_status)err : CL_OK;
}

void cl_plan_destroy(cl_plan* p) {
  if (!p) return;
  if (p->side) {
    cudaStreamSynchronize(p->side);
    cudaStreamDestroy(p->side);
  }
  if (p->aux) {
    cudaStreamSynchronize(p->aux);
    cudaStreamDestroy(p->aux);
  }
  for (cudaEvent_t e : p->events) cudaEventDestroy(e);
  if (p->h_ends) cudaFreeHost(p->h_ends);
  if (p->h_sbuf) cudaFreeHost(p->h_sbuf);
  delete p;
}

}  // extern "C"
