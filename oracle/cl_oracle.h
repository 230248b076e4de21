/*
 * cl_oracle.h -- CPU oracle for the Chung-Lu edge-skipping generator.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this library: only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header, table or
 * constant generator with the CUDA library.
 *
 * What it computes (Alam & Khan, "Parallel Algorithms for Generating Random
 * Networks with Given Degree Sequences"):
 *   - the sequential skip algorithm, Algorithm 1 (Serial-CL / Create-Edges),
 *     for every item of the canonical item space, with the random stream made
 *     explicit (Philox4x32-10, counter = (draw, segment, u_lo, u_hi),
 *     key = seed);
 *   - the cost model of Eq. 1, Eq. 2 and Eq. 6 and the partition rule of
 *     Eq. 3 (uniform cost partitioning);
 *   - closed forms used as pins: expected edge count (Section 3, the pair
 *     probability min(1, w_i w_j / S)), its variance, capped expected
 *     degrees (Section 3 gives the uncapped case w_i - w_i^2/S) and the
 *     gradient of the calibration loss.
 *
 * Readings of the paper that this file takes (each is also listed in the
 * design notes): the loop of Algorithm 1 ends when the candidate falls past
 * the end of the row (otherwise it never ends); the skip is the floor of the
 * exact real log(r)/log(1-p); a draw is consumed per loop iteration even when
 * p = 1; the acceptance compares r < q/p strictly and exactly; the cap
 * min(., 1) is applied (the paper assumes max w^2 < S, the workloads do not).
 */
#ifndef CL_ORACLE_H
#define CL_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_W_I32 = 0, OR_W_F64 = 1 };

typedef struct {
  int64_t n;          /* number of nodes */
  int32_t wtype;      /* OR_W_I32 or OR_W_F64 */
  const void* w;      /* host array of n weights, sorted non-increasing */
  uint64_t seed;      /* Philox key */
  double heavy_w;     /* rows with w_u >= heavy_w are cut into 2^16-wide v-segments */
  double S_f64;       /* for OR_W_F64: the correctly rounded sum of w (caller computes it) */
} or_graph;

typedef struct {
  int64_t S_i64;      /* exact integer sum (OR_W_I32) */
  double S;           /* S as a double (exact for OR_W_I32 when < 2^53) */
  int64_t H;          /* number of heavy rows (a prefix, since w is sorted) */
  int64_t n_heavy_items;
  int64_t n_items;
  int32_t status;     /* 0 ok, 1 unsorted, 2 negative/non-finite, 3 range */
} or_info;

typedef struct {
  int64_t iterations;   /* loop iterations (one Philox block each) */
  int64_t fallbacks;    /* skips not decided by the double evaluation */
  int64_t unresolved;   /* skips not decided by the quad evaluation either */
} or_stats;

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), in place on ctr[4]. */
void or_philox4x32_10(uint32_t ctr[4], uint32_t k0, uint32_t k1);
/* r = (2*floor(X / 2^12) + 1) / 2^53 with X = hi*2^32 + lo: r in (0,1), exact in double. */
double or_uniform53(uint32_t lo, uint32_t hi);

/* Skip length of Algorithm 1: min(floor(ln r / ln(1 - Q/S)), R) for 0 < Q < S, R >= 1. */
int64_t or_skip(double r, double Q, double S, int64_t R, or_stats* st);
/* x = ln r / ln(1 - Q/S) evaluated in binary128, returned as hi + lo doubles. */
void or_skip_x_quad(double r, double Q, double S, double* hi, double* lo);
/* -ln(A/B) in binary128 for 0 < A <= B, returned as hi + lo doubles. */
/* -ln(1 - Q/S) for doubles 0 < Q < S, in binary128, as a pair of doubles. */
void or_neglog1m_quad(double Q, double S, double* hi, double* lo);
void or_neglog_ratio_quad(double A, double B, double* hi, double* lo);

int32_t or_analyze(const or_graph* g, or_info* info);
/* Bounds of item i: source row u, segment field (0xFFFFFFFF for light rows), [j0, end). */
int32_t or_item_bounds(const or_graph* g, const or_info* info, int64_t item,
                       int64_t* u, uint32_t* seg, int64_t* j0, int64_t* end);
/* Generates item i: writes up to cap destination nodes to v_out, returns the count. */
int64_t or_generate_item(const or_graph* g, const or_info* info, int64_t item,
                         int64_t* v_out, int64_t cap, or_stats* st);
/* Counts of every item in [ib, ie) (counts has ie - ib entries). */
void or_count_items(const or_graph* g, const or_info* info, int64_t ib, int64_t ie,
                    int32_t* counts, or_stats* st);
/* Edges of items [ib, ie) as (u, v) int64 pairs, canonical order; returns m or -1 on overflow. */
int64_t or_generate_items(const or_graph* g, const or_info* info, int64_t ib, int64_t ie,
                          int64_t* uv, int64_t cap, or_stats* st);

/* Item costs: c = 1 + (w_u / S) * sum_{v in [j0,end)} w_v  (Eq. 1-2; Eq. 6 for light rows). */
void or_item_costs(const or_graph* g, const or_info* info, double* c);
/* Uniform cost partition, Eq. 3: start[t] = first item with C >= t * Zbar, C inclusive prefix. */
void or_ucp_starts(const double* c, int64_t n_items, int64_t T, int64_t* start);
/* The paper's Calc-Cost (Algorithm 2) over P simulated processors: inclusive prefix C. */
void or_calc_cost(const double* c, int64_t n_items, int64_t P, double* C);

/* Integer weights: N = sum_{u<v} min(S, w_u w_v) as a 128-bit integer (hi, lo), so that
 * E[m] = N / S exactly.  Also Var[m] = sum p (1 - p) in extended precision. */
void or_expected_edges_i32(const int32_t* w, int64_t n, uint64_t* N_hi, uint64_t* N_lo,
                           int64_t* S, double* var);
void or_expected_edges_bruteforce_i32(const int32_t* w, int64_t n, uint64_t* N_hi, uint64_t* N_lo);

/* Capped expected degrees E_u = sum_{v != u} min(1, w_u w_v / S) for double weights sorted
 * non-increasing; the pair is capped iff fl(w_u * w_v) >= S. */
void or_expected_degree(const double* w, int64_t n, double S, double* E);
void or_expected_degree_bruteforce(const double* w, int64_t n, double S, double* E);
/* Gradient of L = sum_u gE_u * E_u with respect to w (S = sum w depends on w). */
void or_expected_degree_adjoint(const double* w, int64_t n, double S, const double* gE, double* gw);
void or_expected_degree_adjoint_bruteforce(const double* w, int64_t n, double S,
                                           const double* gE, double* gw);
/* The same gradient in O(n^2), summed pair by pair (no thresholds or suffix sums). */
void or_expected_degree_adjoint_pairwise(const double* w, int64_t n, double S, const double* gE, double* gw);

#ifdef __cplusplus
}
#endif
#endif
