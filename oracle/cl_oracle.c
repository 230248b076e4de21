/*
 * cl_oracle.c -- plain, single-threaded CPU oracle for the Chung-Lu skip
 * sampler.  TEST INFRASTRUCTURE ONLY: only the test suite, the smoke check
 * and the benchmark's CPU-baseline leg may load it; the product path never
 * does.  It shares no code with the CUDA library (its own Philox, its own
 * skip and acceptance arithmetic).
 *
 * Every function names the passage of Alam & Khan it follows.
 */
#include "cl_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* binary128 arithmetic: long double is binary128 on aarch64; on x86-64 */
/* long double is the 80-bit format, so __float128 + libquadmath is used */
#if defined(__x86_64__) || defined(__i386__)
#include <quadmath.h>
typedef __float128 hp_t;
#define HP_LOG(x) logq(x)
#define HP_LOG1P(x) log1pq(x)
#define HP_FLOOR(x) floorq(x)
#define HP_ROUND(x) roundq(x)
#define HP_LDEXP(x, e) ldexpq((x), (e))
#else
typedef long double hp_t;
#define HP_LOG(x) logl(x)
#define HP_LOG1P(x) log1pl(x)
#define HP_FLOOR(x) floorl(x)
#define HP_ROUND(x) roundl(x)
#define HP_LDEXP(x, e) ldexpl((x), (e))
#endif

/* ------------------------------------------------------------------ */
/* Philox4x32-10 from its published description (Salmon et al., SC'11): */
/* each round multiplies words 0 and 2 by the two round multipliers,    */
/* xors the high halves with the other words and the round key, and the */
/* key is bumped by the two Weyl constants between rounds.              */
void or_philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * c[0];
    uint64_t p1 = (uint64_t)M1 * c[2];
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c[0] = n0;
    c[1] = n1;
    c[2] = n2;
    c[3] = n3;
  }
}

/* The "random r in (0,1)" of Algorithm 1: 52 random bits k give
 * r = (2k+1)/2^53, never 0 or 1 and exact in double. */
static uint64_t grid52(uint32_t lo, uint32_t hi) { return (((uint64_t)hi << 32) | lo) >> 12; }

double or_uniform53(uint32_t lo, uint32_t hi) {
  return ldexp((double)(2 * grid52(lo, hi) + 1), -53);
}

/* ------------------------------------------------------------------ */
/* Skip length, Algorithm 1: delta = floor(log(r) / log(1 - p)) with     */
/* p = Q/S.  The floor is that of the exact real number.  A double      */
/* evaluation (relative error below 2^-50, far inside the 2^-44 window  */
/* used) decides it when x is not near an integer; otherwise binary128  */
/* decides it with a 2^-100 window; a case neither decides is counted   */
/* and takes the nearest integer (right when x is exactly an integer).  */

/* -ln(1 - Q/S) in double for 0 < Q < S. */
static double neglog1m_d(double Q, double S) {
  if (2.0 * Q <= S) return -log1p(-(Q / S));
  return -log((S - Q) / S); /* S - Q is exact here (S/2 < Q <= S) */
}
/* -ln r in double for r in (0, 1). */
static double neglog_r_d(double r) {
  if (r >= 0.5) return -log1p(-(1.0 - r)); /* 1 - r is exact for r in [1/2, 1) */
  return -log(r);
}
static hp_t neglog1m_q(double Q, double S) {
  hp_t q = (hp_t)Q, s = (hp_t)S;
  if (2.0 * Q <= S) return -HP_LOG1P(-(q / s));
  return -HP_LOG((s - q) / s);
}
static hp_t neglog_r_q(double r) {
  hp_t rq = (hp_t)r;
  if (r >= 0.5) return -HP_LOG1P(-((hp_t)1 - rq));
  return -HP_LOG(rq);
}

void or_skip_x_quad(double r, double Q, double S, double* hi, double* lo) {
  hp_t x = neglog_r_q(r) / neglog1m_q(Q, S);
  double h = (double)x;
  *hi = h;
  *lo = (double)(x - (hp_t)h);
}

void or_neglog1m_quad(double Q, double S, double* hi, double* lo) {
  hp_t y = neglog1m_q(Q, S);
  double h = (double)y;
  *hi = h;
  *lo = (double)(y - (hp_t)h);
}

void or_neglog_ratio_quad(double A, double B, double* hi, double* lo) {
  hp_t a = (hp_t)A, b = (hp_t)B, y;
  if (2.0 * A >= B)
    y = -HP_LOG1P(-((b - a) / b)); /* B - A exact: B/2 <= A <= B */
  else
    y = -HP_LOG(a / b);
  double h = (double)y;
  *hi = h;
  *lo = (double)(y - (hp_t)h);
}

int64_t or_skip(double r, double Q, double S, int64_t R, or_stats* st) {
  double x = neglog_r_d(r) / neglog1m_d(Q, S);
  const double tau = 0x1p-44;
  double xl = x * (1.0 - tau), xh = x * (1.0 + tau);
  if (xl >= (double)R) return R;
  if (xh < (double)R && floor(xl) == floor(xh)) return (int64_t)floor(x);
  if (st) st->fallbacks++;
  hp_t xq = neglog_r_q(r) / neglog1m_q(Q, S);
  const hp_t tq = HP_LDEXP((hp_t)1, -100);
  hp_t ql = xq * ((hp_t)1 - tq), qh = xq * ((hp_t)1 + tq);
  if (ql >= (hp_t)R) return R;
  if (qh < (hp_t)R && HP_FLOOR(ql) == HP_FLOOR(qh)) return (int64_t)HP_FLOOR(xq);
  if (st) st->unresolved++;
  hp_t k = HP_ROUND(xq);
  if (k >= (hp_t)R) return R;
  return (int64_t)k;
}

/* ------------------------------------------------------------------ */
/* Graph analysis: S = sum_k w_k (Algorithm 1, Serial-CL), validation of  */
/* the sorted, non-negative precondition (Section 3), heavy rows and the  */
/* item space.  Items, in canonical order: heavy rows u < H (w_u >= W_H)  */
/* cut at absolute multiples of 2^16 of v, then one item per light row.   */

#define SEG_LOG2 16

static double wval(const or_graph* g, int64_t i) {
  if (g->wtype == OR_W_I32) return (double)((const int32_t*)g->w)[i];
  return ((const double*)g->w)[i];
}


static int64_t heavy_base(int64_t U, int64_t n);

int32_t or_analyze(const or_graph* g, or_info* info) {
  memset(info, 0, sizeof(*info));
  int64_t n = g->n;
  if (n < 0) {
    info->status = 3;
    return 3;
  }
  if (g->wtype == OR_W_I32) {
    const int32_t* w = (const int32_t*)g->w;
    int64_t S = 0;
    for (int64_t i = 0; i < n; ++i) {
      if (w[i] < 0) info->status = 2;
      if (i + 1 < n && w[i] < w[i + 1] && info->status == 0) info->status = 1;
      S += w[i];
    }
    info->S_i64 = S;
    info->S = (double)S;
    if (info->status == 0 && S >= ((int64_t)1 << 53)) info->status = 3;
  } else {
    const double* w = (const double*)g->w;
    for (int64_t i = 0; i < n; ++i) {
      if (!(w[i] >= 0.0) || !isfinite(w[i])) info->status = 2;
      if (i + 1 < n && w[i] < w[i + 1] && info->status == 0) info->status = 1;
    }
    info->S = g->S_f64;
  }
  int64_t H = 0;
  while (H < n && wval(g, H) >= g->heavy_w) ++H; /* heavy rows form a prefix */
  info->H = H;
  int64_t Hh = H < n - 1 ? H : n - 1;
  int64_t nh = Hh > 0 ? heavy_base(Hh, n) : 0;
  info->n_heavy_items = nh;
  int64_t light = (n - 1) - H;
  info->n_items = nh + (light > 0 ? light : 0);
  return info->status;
}

/* Items before heavy row U: sum_{u<U} K_u with K_u = N1 - ((u+1) >> 16) + 1,
 * N1 = (n-1) >> 16, written with F(U) = sum_{x=0}^{U} floor(x / 2^16). */
static int64_t heavy_base(int64_t U, int64_t n) {
  const int64_t B = (int64_t)1 << SEG_LOG2;
  int64_t N1 = (n - 1) >> SEG_LOG2;
  int64_t q = U / B;
  int64_t F = B * q * (q - 1) / 2 + q * (U - q * B + 1);
  return U * (N1 + 1) - F;
}

int32_t or_item_bounds(const or_graph* g, const or_info* info, int64_t item, int64_t* u,
                       uint32_t* seg, int64_t* j0, int64_t* end) {
  int64_t n = g->n;
  if (item < 0 || item >= info->n_items) return -1;
  if (item >= info->n_heavy_items) {
    *u = info->H + (item - info->n_heavy_items);
    *seg = 0xFFFFFFFFu;
    *j0 = *u + 1;
    *end = n;
    return 0;
  }
  /* heavy row: the last r with heavy_base(r) <= item, by bisection */
  int64_t Hh = info->H < n - 1 ? info->H : n - 1;
  int64_t lo = 0, hi = Hh - 1;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo + 1) / 2;
    if (heavy_base(mid, n) <= item)
      lo = mid;
    else
      hi = mid - 1;
  }
  int64_t r = lo;
  int64_t k = ((r + 1) >> SEG_LOG2) + (item - heavy_base(r, n));
  int64_t s0 = k << SEG_LOG2, s1 = (k + 1) << SEG_LOG2;
  *u = r;
  *seg = (uint32_t)k;
  *j0 = s0 > r + 1 ? s0 : r + 1;
  *end = s1 < n ? s1 : n;
  return 0;
}

/* Q(u, v) = min(w_u w_v, S): S times the pair probability min(w_u w_v / S, 1)
 * of Section 3.  Integer weights: exact 64-bit product.  Double weights: the
 * rounded product, capped iff it is >= S. */
static double Qof(const or_graph* g, const or_info* info, int64_t u, int64_t v) {
  if (g->wtype == OR_W_I32) {
    const int32_t* w = (const int32_t*)g->w;
    int64_t q = (int64_t)w[u] * (int64_t)w[v];
    return q >= info->S_i64 ? (double)info->S_i64 : (double)q;
  }
  const double* w = (const double*)g->w;
  double q = w[u] * w[v];
  return q >= info->S ? info->S : q;
}

/* Acceptance of Algorithm 1: r < q/p, i.e. r * Q_prev < Q_v, decided exactly. */
static int accept(const or_graph* g, uint32_t lo, uint32_t hi, double Qprev, double Qv) {
  uint64_t k = grid52(lo, hi);
  if (g->wtype == OR_W_I32) {
    /* (2k+1) * Qprev < 2^53 * Qv in 128-bit integers */
    unsigned __int128 lhs = (unsigned __int128)(2 * k + 1) * (uint64_t)Qprev;
    unsigned __int128 rhs = (unsigned __int128)(uint64_t)Qv << 53;
    return lhs < rhs;
  }
  double r = ldexp((double)(2 * k + 1), -53);
  return fma(r, Qprev, -Qv) < 0.0; /* the sign of a fused multiply-add is exact */
}

/* One item of the skip sampler (Section 3, Algorithm 1).  In a
 * non-increasing weight sequence the pair probability of row u only falls as
 * v grows, so the probability p_ref = Q_ref / S of the last visited position
 * bounds every later one: the next candidate is found by a geometric skip
 * drawn at p_ref (Section 3's skip length), and a candidate v is kept with
 * probability Q(u, v) / Q_ref (thinning), which leaves every pair of the item
 * an edge with probability Q(u, v) / S, independently.  The reference then
 * moves to the candidate.  Reading of the paper: a skip that lands at or past
 * the end of the item closes it; p_ref = 0 closes it too (no later pair can
 * be an edge). */
int64_t or_generate_item(const or_graph* g, const or_info* info, int64_t item, int64_t* v_out,
                         int64_t cap, or_stats* st) {
  int64_t u, j0, end;
  uint32_t seg;
  if (or_item_bounds(g, info, item, &u, &seg, &j0, &end) != 0) return -1;
  const double S = info->S;
  const uint32_t k0 = (uint32_t)g->seed, k1 = (uint32_t)(g->seed >> 32);
  if (j0 >= end) return 0;
  double Q_ref = Qof(g, info, u, j0); /* the item's first position sets the first bound */
  int64_t pos = j0;                   /* first position the next skip can land on */
  uint32_t draw = 0;                  /* index of the item's next Philox block */
  int64_t count = 0;
  for (;;) {
    if (pos >= end || Q_ref <= 0.0) break;
    uint32_t b[4] = {draw, seg, (uint32_t)u, (uint32_t)((uint64_t)u >> 32)};
    or_philox4x32_10(b, k0, k1);
    ++draw;
    if (st) st->iterations++;
    const int64_t room = end - pos;
    /* p_ref = 1 (capped): every position is a candidate, no skip */
    const int64_t skip = Q_ref == S ? 0 : or_skip(or_uniform53(b[0], b[1]), Q_ref, S, room, st);
    if (skip >= room) break;
    const int64_t cand = pos + skip;
    const double Q_cand = Qof(g, info, u, cand);
    if (accept(g, b[2], b[3], Q_ref, Q_cand)) {
      if (count < cap && v_out) v_out[count] = cand;
      ++count;
    }
    Q_ref = Q_cand;
    pos = cand + 1;
  }
  return count;
}

void or_count_items(const or_graph* g, const or_info* info, int64_t ib, int64_t ie,
                    int32_t* counts, or_stats* st) {
  for (int64_t i = ib; i < ie; ++i) counts[i - ib] = (int32_t)or_generate_item(g, info, i, NULL, 0, st);
}

int64_t or_generate_items(const or_graph* g, const or_info* info, int64_t ib, int64_t ie,
                          int64_t* uv, int64_t cap, or_stats* st) {
  int64_t m = 0;
  int64_t tmp_cap = 1 << 16;
  int64_t* tmp = (int64_t*)malloc(sizeof(int64_t) * tmp_cap);
  for (int64_t i = ib; i < ie; ++i) {
    int64_t u, j0, end;
    uint32_t seg;
    or_item_bounds(g, info, i, &u, &seg, &j0, &end);
    int64_t c = or_generate_item(g, info, i, tmp, tmp_cap, st);
    if (c > tmp_cap) {
      tmp_cap = c;
      tmp = (int64_t*)realloc(tmp, sizeof(int64_t) * tmp_cap);
      c = or_generate_item(g, info, i, tmp, tmp_cap, NULL);
    }
    for (int64_t k = 0; k < c; ++k) {
      if (m < cap) {
        uv[2 * m] = u;
        uv[2 * m + 1] = tmp[k];
      }
      ++m;
    }
  }
  free(tmp);
  return m > cap ? -1 : m;
}

/* ------------------------------------------------------------------ */
/* Cost model, Eq. 1-2 (e_u = (w_u/S) sum_{v>u} w_v, c_u = e_u + 1) per  */
/* item; for a light row this is Eq. 6, (w_u/S)(S - sigma_u - w_u) + 1.  */
void or_item_costs(const or_graph* g, const or_info* info, double* c) {
  int64_t n = g->n;
  long double* sigma = (long double*)malloc(sizeof(long double) * (size_t)(n + 1));
  sigma[0] = 0;
  for (int64_t i = 0; i < n; ++i) sigma[i + 1] = sigma[i] + (long double)wval(g, i);
  long double S = sigma[n];
  for (int64_t it = 0; it < info->n_items; ++it) {
    int64_t u, j0, end;
    uint32_t seg;
    or_item_bounds(g, info, it, &u, &seg, &j0, &end);
    long double wu = (long double)wval(g, u);
    c[it] = (double)(wu / S * (sigma[end] - sigma[j0]) + 1.0L);
  }
  free(sigma);
}

/* Eq. 3: the lower boundary of partition t is the first item whose inclusive
 * cumulative cost reaches t * Zbar, Zbar = (total cost) / T. */
void or_ucp_starts(const double* c, int64_t n_items, int64_t T, int64_t* start) {
  double* C = (double*)malloc(sizeof(double) * (size_t)(n_items > 0 ? n_items : 1));
  double acc = 0;
  for (int64_t i = 0; i < n_items; ++i) {
    acc += c[i];
    C[i] = acc;
  }
  double Zbar = acc / (double)T;
  int64_t i = 0;
  for (int64_t t = 0; t <= T; ++t) {
    if (t == T) {
      start[t] = n_items;
      break;
    }
    double target = (double)t * Zbar;
    while (i < n_items && C[i] < target) ++i;
    start[t] = i;
  }
  free(C);
}

/* Calc-Cost of Algorithm 2 with P simulated processors: each computes the
 * local running sum of its block, an exclusive prefix over the block
 * totals is formed, and each block adds its prefix. */
void or_calc_cost(const double* c, int64_t n_items, int64_t P, double* C) {
  double* z = (double*)calloc((size_t)P, sizeof(double));
  for (int64_t p = 0; p < P; ++p) {
    int64_t lo = p * n_items / P, hi = (p + 1) * n_items / P;
    double acc = 0;
    for (int64_t i = lo; i < hi; ++i) {
      acc += c[i];
      C[i] = acc;
    }
    z[p] = acc;
  }
  double Z = 0;
  for (int64_t p = 0; p < P; ++p) {
    int64_t lo = p * n_items / P, hi = (p + 1) * n_items / P;
    for (int64_t i = lo; i < hi; ++i) C[i] += Z;
    Z += z[p];
  }
  free(z);
}

/* ------------------------------------------------------------------ */
/* Closed forms.  Section 3: edge (i, j) is present with probability      */
/* min(w_i w_j / S, 1) independently, so E[m] = sum_{i<j} min(S, w_i w_j)/S */

void or_expected_edges_i32(const int32_t* w, int64_t n, uint64_t* N_hi, uint64_t* N_lo,
                           int64_t* S_out, double* var) {
  int64_t S = 0;
  for (int64_t i = 0; i < n; ++i) S += w[i];
  /* suffix sums of w and w^2 */
  int64_t* suf = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  long double* suf2 = (long double*)malloc(sizeof(long double) * (size_t)(n + 1));
  suf[n] = 0;
  suf2[n] = 0;
  for (int64_t i = n - 1; i >= 0; --i) {
    suf[i] = suf[i + 1] + w[i];
    suf2[i] = suf2[i + 1] + (long double)w[i] * (long double)w[i];
  }
  unsigned __int128 N = 0;
  long double sp = 0, sp2 = 0;
  for (int64_t u = 0; u + 1 < n; ++u) {
    /* capped partners of u among v > u: a prefix [u+1, c) since w is sorted */
    int64_t lo = u + 1, hi = n;
    while (lo < hi) {
      int64_t mid = lo + (hi - lo) / 2;
      if ((int64_t)w[u] * w[mid] >= S)
        lo = mid + 1;
      else
        hi = mid;
    }
    int64_t c = lo;
    N += (unsigned __int128)(uint64_t)S * (uint64_t)(c - (u + 1));
    N += (unsigned __int128)(uint64_t)w[u] * (uint64_t)suf[c];
    long double wu = (long double)w[u];
    sp += wu * (long double)suf[c] / (long double)S;
    sp2 += wu * wu * suf2[c] / ((long double)S * (long double)S);
  }
  *N_hi = (uint64_t)(N >> 64);
  *N_lo = (uint64_t)N;
  *S_out = S;
  *var = (double)(sp - sp2); /* capped pairs have p(1-p) = 0 */
  free(suf);
  free(suf2);
}

void or_expected_edges_bruteforce_i32(const int32_t* w, int64_t n, uint64_t* N_hi, uint64_t* N_lo) {
  int64_t S = 0;
  for (int64_t i = 0; i < n; ++i) S += w[i];
  unsigned __int128 N = 0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i + 1; j < n; ++j) {
      int64_t q = (int64_t)w[i] * w[j];
      N += (unsigned __int128)(uint64_t)(q < S ? q : S);
    }
  *N_hi = (uint64_t)(N >> 64);
  *N_lo = (uint64_t)N;
}

/* Capped expected degree.  Section 3 gives E[d_i] = w_i - w_i^2/S when no
 * pair is capped; with the cap, E_u = sum_{v != u} min(1, w_u w_v / S).  For
 * sorted w the capped partners of u are a prefix [0, t_u), so
 *   E_u = (t_u - [u < t_u]) + (w_u / S) * (R_{t_u} - [u >= t_u] w_u),
 * R_k = sum_{v >= k} w_v. */
static int64_t cap_threshold(const double* w, int64_t n, double wu, double S) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (wu * w[mid] >= S)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

void or_expected_degree(const double* w, int64_t n, double S, double* E) {
  long double* R = (long double*)malloc(sizeof(long double) * (size_t)(n + 1));
  R[n] = 0;
  for (int64_t i = n - 1; i >= 0; --i) R[i] = R[i + 1] + (long double)w[i];
  for (int64_t u = 0; u < n; ++u) {
    int64_t t = cap_threshold(w, n, w[u], S);
    long double capped = (long double)(t - (u < t ? 1 : 0));
    long double A = R[t] - (u >= t ? (long double)w[u] : 0.0L);
    E[u] = (double)(capped + (long double)w[u] / (long double)S * A);
  }
  free(R);
}

void or_expected_degree_bruteforce(const double* w, int64_t n, double S, double* E) {
  for (int64_t u = 0; u < n; ++u) {
    long double acc = 0;
    for (int64_t v = 0; v < n; ++v) {
      if (v == u) continue;
      double q = w[u] * w[v];
      acc += (q >= S) ? 1.0L : (long double)w[u] * (long double)w[v] / (long double)S;
    }
    E[u] = (double)acc;
  }
}

/* Gradient of L = sum_u gE_u E_u(w), with S = sum w.  Differentiating
 * E_u = sum_{v != u, uncapped} w_u w_v / S (+ capped count):
 *   dL/dw_k = [gE_k A_k + sum_{u != k, (u,k) uncapped} gE_u w_u - K] / S,
 *   A_u = sum_{v != u, uncapped} w_v,  K = sum_u gE_u (w_u / S) A_u. */
void or_expected_degree_adjoint(const double* w, int64_t n, double S, const double* gE, double* gw) {
  long double* R = (long double*)malloc(sizeof(long double) * (size_t)(n + 1));
  long double* G = (long double*)malloc(sizeof(long double) * (size_t)(n + 1));
  int64_t* t = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  R[n] = 0;
  G[n] = 0;
  for (int64_t i = n - 1; i >= 0; --i) {
    R[i] = R[i + 1] + (long double)w[i];
    G[i] = G[i + 1] + (long double)gE[i] * (long double)w[i];
  }
  long double K = 0;
  for (int64_t u = 0; u < n; ++u) {
    t[u] = cap_threshold(w, n, w[u], S);
    long double A = R[t[u]] - (u >= t[u] ? (long double)w[u] : 0.0L);
    K += (long double)gE[u] * (long double)w[u] / (long double)S * A;
  }
  for (int64_t k = 0; k < n; ++k) {
    long double A = R[t[k]] - (k >= t[k] ? (long double)w[k] : 0.0L);
    long double B = G[t[k]] - (k >= t[k] ? (long double)gE[k] * (long double)w[k] : 0.0L);
    gw[k] = (double)(((long double)gE[k] * A + B - K) / (long double)S);
  }
  free(R);
  free(G);
  free(t);
}

void or_expected_degree_adjoint_bruteforce(const double* w, int64_t n, double S, const double* gE,
                                           double* gw) {
  /* dE_u/dw_k summed over u, term by term from the pairwise definition */
  long double Sl = (long double)S;
  for (int64_t k = 0; k < n; ++k) {
    long double acc = 0;
    for (int64_t u = 0; u < n; ++u) {
      for (int64_t v = 0; v < n; ++v) {
        if (v == u) continue;
        if (w[u] * w[v] >= S) continue; /* capped: derivative 0 */
        long double d = -(long double)w[u] * (long double)w[v] / (Sl * Sl);
        if (u == k) d += (long double)w[v] / Sl;
        if (v == k) d += (long double)w[u] / Sl;
        acc += (long double)gE[u] * d;
      }
    }
    gw[k] = (double)acc;
  }
}

/* The same gradient in O(n^2), every sum taken pair by pair from the pairwise
 * definition (no sorted thresholds, no suffix sums), for n in the thousands.
 * With f_uv = w_u w_v / S on an uncapped pair (fl(w_u w_v) < S) and a
 * constant 1 on a capped one (derivative 0), S = sum_k w_k:
 *   d f_uv / d w_k = ([u = k] w_v + [v = k] w_u) / S - w_u w_v / S^2,
 * and summing gE_u d f_uv / d w_k over ordered pairs u != v:
 *   dL/dw_k = (gE_k A_k + B_k - K) / S,
 *   A_u = sum_{v != u, (u,v) uncapped} w_v,
 *   B_k = sum_{u != k, (u,k) uncapped} gE_u w_u,
 *   K = sum_u gE_u w_u A_u / S. */
void or_expected_degree_adjoint_pairwise(const double* w, int64_t n, double S, const double* gE, double* gw) {
  long double* A = (long double*)calloc((size_t)(n > 0 ? n : 1), sizeof(long double));
  long double* B = (long double*)calloc((size_t)(n > 0 ? n : 1), sizeof(long double));
  for (int64_t u = 0; u < n; ++u)
    for (int64_t v = 0; v < n; ++v) {
      if (v == u || w[u] * w[v] >= S) continue;
      A[u] += (long double)w[v];
      B[u] += (long double)gE[v] * (long double)w[v];
    }
  long double K = 0;
  for (int64_t u = 0; u < n; ++u) K += (long double)gE[u] * (long double)w[u] * A[u] / (long double)S;
  for (int64_t k = 0; k < n; ++k) gw[k] = (double)(((long double)gE[k] * A[k] + B[k] - K) / (long double)S);
  free(A);
  free(B);
}
