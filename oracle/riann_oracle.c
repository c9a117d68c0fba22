/*
 * riann_oracle.c -- plain CPU oracle for RIANN's per-frame query step.
 *
 * TEST INFRASTRUCTURE ONLY: called by the tests, the smoke check and the CPU
 * baseline of the benchmark; never by the product path.  Plain C99 + OpenMP
 * over queries (queries are independent: Alg. 1 treats each query patch on its
 * own and the method uses no spatial propagation, Sec. 6).  No blocking, no
 * vectorisation tricks, no shared code with the CUDA library.
 *
 * Parity pins (tests/test_oracle_pins.py): brute force vs an independent numpy
 * argmin; alpha = 1 reduces RIANN to exact NN (triangle inequality); alpha = 0
 * special case; the membership test vs high-precision decimal square roots and
 * exact-boundary perfect squares; hand-worked constant-patch fixtures under
 * tests/golden/; definitional == indexed; key-point permutation invariance.
 * The other functions have pins of their own (tests/test_oracle_*.py): k-NN
 * lists vs sorted numpy brute force and hand-worked lists; the random-anchor
 * loop vs Philox known-answer vectors, its special cases and an independent
 * Python implementation; reconstruction vs a scatter formulation and closed
 * forms; clustering vs numpy medians and hand-worked trees; the unit-length
 * variant vs float64 and a hand-worked step on exactly representable
 * patches; 3-D volumes vs plain slicing.  tests/test_oracle_mutants.py plants
 * one mistake at a time in this file and checks that a pin fails.
 * The full alpha = 1/4 output has no external pin (the paper prints no values):
 * parity unpinned against the paper's own outputs.
 */
#include "riann_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PATCH 8

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* squared L2 distance of two D-byte vectors (the paper's dist, squared; Sec. 3.1) */
static uint32_t sqdist(const uint8_t* a, const uint8_t* b, int32_t D) {
  uint32_t s = 0;
  for (int32_t i = 0; i < D; ++i) {
    int32_t d = (int32_t)a[i] - (int32_t)b[i];
    s += (uint32_t)(d * d);
  }
  return s;
}

/* the 8x8xC query patch with top-left (y, x), in (dy, dx, c) order (Sec. 4) */
static void extract_query(const uint8_t* frame, int32_t W, int32_t C, int32_t y, int32_t x,
                          uint8_t* q) {
  int32_t k = 0;
  for (int32_t dy = 0; dy < PATCH; ++dy)
    for (int32_t dx = 0; dx < PATCH; ++dx)
      for (int32_t c = 0; c < C; ++c)
        q[k++] = frame[((int64_t)(y + dy) * W + (x + dx)) * C + c];
}

/*
 * Ring membership (Sec. 3.2: a ring of radius dist(anchor, q) and half-width
 * epsilon = alpha * dist(q, r_i); Alg. 1 candidate-set conditions
 * d - eps <= dist(anchor, r) <= d + eps).  With A = ||k - r||^2,
 * B = ||k - q||^2, C = ||q - r_p||^2 and alpha = p/q the condition is
 *     |sqrt(A) - sqrt(B)| <= (p/q) sqrt(C).
 * Squaring both (non-negative) sides:
 *     q^2 (A + B) - p^2 C <= 2 q^2 sqrt(A B).
 * Writing L for the left side, it holds when L <= 0, else iff L^2 <= 4 q^4 A B.
 * Evaluated in 128-bit integers, so there is no rounding anywhere.
 */
int oracle_ring_member(uint32_t A, uint32_t B, uint32_t C, int32_t p, int32_t q) {
  __int128 qq = (__int128)q * q;
  __int128 L = qq * ((__int128)A + (__int128)B) - (__int128)p * p * (__int128)C;
  if (L <= 0) return 1;
  unsigned __int128 lhs = (unsigned __int128)L * (unsigned __int128)L;
  unsigned __int128 rhs = (unsigned __int128)4 * (unsigned __int128)(qq * qq) *
                          (unsigned __int128)A * (unsigned __int128)B;
  return lhs <= rhs;
}

/* Distances from every reference to every key point (Sec. 3.3 pre-processing:
 * the distance lists, here only towards the K fixed anchors). */
void oracle_key_distances(const uint8_t* R, int32_t n, int32_t D,
                          const uint8_t* KP, int32_t K, uint32_t* P) {
#pragma omp parallel for schedule(static)
  for (int32_t r = 0; r < n; ++r)
    for (int32_t m = 0; m < K; ++m)
      P[(int64_t)r * K + m] = sqdist(KP + (int64_t)m * D, R + (int64_t)r * D, D);
}

typedef struct { uint32_t a; int32_t id; } entry_t;

static int cmp_entry(const void* x, const void* y) {
  const entry_t* u = (const entry_t*)x;
  const entry_t* v = (const entry_t*)y;
  if (u->a != v->a) return u->a < v->a ? -1 : 1;
  if (u->id != v->id) return u->id < v->id ? -1 : 1;
  return 0;
}

/* Sorted lists (Sec. 3.3 keeps, per anchor, its distances to the references
 * in sorted order; here one list per key point), ascending by (distance, index). */
void oracle_sort_tables(const uint32_t* P, int32_t n, int32_t K, uint32_t* TA, int32_t* Tid) {
#pragma omp parallel for schedule(static)
  for (int32_t m = 0; m < K; ++m) {
    entry_t* e = (entry_t*)malloc(sizeof(entry_t) * (size_t)n);
    for (int32_t r = 0; r < n; ++r) { e[r].a = P[(int64_t)r * K + m]; e[r].id = r; }
    qsort(e, (size_t)n, sizeof(entry_t), cmp_entry);
    for (int32_t j = 0; j < n; ++j) {
      TA[(int64_t)m * n + j] = e[j].a;
      Tid[(int64_t)m * n + j] = e[j].id;
    }
    free(e);
  }
}

/* argmin over all of R with the lower index winning ties (exact NN; used for
 * the frame-0 initialisation and for queries whose rings are too wide) */
static void brute_force(const uint8_t* q, const uint8_t* R, int32_t n, int32_t D,
                        int32_t* best_id, uint32_t* best_d) {
  int32_t bi = 0;
  uint32_t bd = sqdist(q, R, D);
  for (int32_t r = 1; r < n; ++r) {
    uint32_t d = sqdist(q, R + (int64_t)r * D, D);
    if (d < bd) { bd = d; bi = r; }
  }
  *best_id = bi;
  *best_d = bd;
}

static int64_t query_at(const int64_t* qidx, int64_t i) { return qidx ? qidx[i] : i; }

void oracle_exact_nn(const uint8_t* frame, int32_t H, int32_t W, int32_t C,
                     const uint8_t* R, int32_t n,
                     const int64_t* qidx, int64_t nq,
                     int32_t* annf, uint32_t* dist, uint32_t* count) {
  const int32_t D = PATCH * PATCH * C;
  const int32_t Wq = W - PATCH + 1;
  const int64_t Q = (int64_t)(H - PATCH + 1) * Wq;
  const int64_t N = qidx ? nq : Q;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < N; ++i) {
    uint8_t q[PATCH * PATCH * 3];
    int64_t qi = query_at(qidx, i);
    extract_query(frame, W, C, (int32_t)(qi / Wq), (int32_t)(qi % Wq), q);
    int32_t bi; uint32_t bd;
    brute_force(q, R, n, D, &bi, &bd);
    annf[i] = bi;
    if (dist) dist[i] = bd;
    if (count) count[i] = (uint32_t)n;
  }
}

/*
 * Definitional mode.  Alg. 1 for one query, in the paper's order:
 *   r_p = ANNF^(t-1)(x, y);  d = dist(q, r_p);  eps = alpha * d
 *   candidate set = references inside every ring (here the K key-point rings)
 *   ANNF^(t)(x, y) = argmin over the candidates (and r_p) of dist(q, s)
 * Every ring is evaluated over all references with the exact predicate.
 */
void oracle_riann_definitional(const uint8_t* frame, int32_t H, int32_t W, int32_t C,
                               const uint8_t* R, int32_t n,
                               const uint8_t* KP, int32_t K, const uint32_t* P,
                               const int32_t* prev, int32_t alpha_num, int32_t alpha_den,
                               int32_t ring_limit,
                               const int64_t* qidx, int64_t nq,
                               int32_t* annf, uint32_t* dist, uint32_t* count, uint32_t* nseed) {
  const int32_t D = PATCH * PATCH * C;
  const int32_t Wq = W - PATCH + 1;
  const int64_t Q = (int64_t)(H - PATCH + 1) * Wq;
  const int64_t N = qidx ? nq : Q;
#pragma omp parallel
  {
    uint8_t q[PATCH * PATCH * 3];
    uint32_t* B = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)K);
    uint32_t* ring_size = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)K);
    uint8_t* in_all = (uint8_t*)malloc((size_t)n);
#pragma omp for schedule(dynamic, 16)
    for (int64_t i = 0; i < N; ++i) {
      int64_t qi = query_at(qidx, i);
      extract_query(frame, W, C, (int32_t)(qi / Wq), (int32_t)(qi % Wq), q);
      if (!prev) {                                   /* frame 0: exact NN */
        int32_t bi; uint32_t bd;
        brute_force(q, R, n, D, &bi, &bd);
        annf[i] = bi;
        if (dist) dist[i] = bd;
        if (count) count[i] = (uint32_t)n;
        if (nseed) nseed[i] = 0;
        continue;
      }
      const int32_t rp = prev[qi];
      const uint32_t Cd = sqdist(q, R + (int64_t)rp * D, D);      /* dist(q, r_p)^2 */
      for (int32_t m = 0; m < K; ++m) B[m] = sqdist(q, KP + (int64_t)m * D, D);
      for (int32_t m = 0; m < K; ++m) ring_size[m] = 0;
      uint32_t s_size = 0;
      for (int32_t r = 0; r < n; ++r) {
        int inside = 1;
        for (int32_t m = 0; m < K; ++m) {
          int mem = oracle_ring_member(P[(int64_t)r * K + m], B[m], Cd, alpha_num, alpha_den);
          ring_size[m] += (uint32_t)mem;
          inside &= mem;
        }
        in_all[r] = (uint8_t)inside;
        s_size += (uint32_t)inside;
      }
      uint32_t ns = ring_size[0];
      for (int32_t m = 1; m < K; ++m) if (ring_size[m] < ns) ns = ring_size[m];
      if (nseed) nseed[i] = ns;
      if (ring_limit >= 0 && ns > (uint32_t)ring_limit) {   /* rings too wide: brute force */
        int32_t bi; uint32_t bd;
        brute_force(q, R, n, D, &bi, &bd);
        annf[i] = bi;
        if (dist) dist[i] = bd;
        if (count) count[i] = (uint32_t)n;
        continue;
      }
      int32_t bi = rp;                                /* r_p is always verified */
      uint32_t bd = Cd;
      for (int32_t r = 0; r < n; ++r) {
        if (!in_all[r]) continue;
        uint32_t d = sqdist(q, R + (int64_t)r * D, D);
        if (d < bd || (d == bd && r < bi)) { bd = d; bi = r; }
      }
      annf[i] = bi;
      if (dist) dist[i] = bd;
      if (count) count[i] = s_size;
    }
    free(B); free(ring_size); free(in_all);
  }
}

/*
 * k-NN output (Sec. 7: the method can return more than one match per
 * query).  The candidate set of a query is the set Alg. 1 takes its argmin
 * over, with the readings of oracle_riann_definitional: S u {r_p} (r_p once)
 * when some ring holds at most ring_limit references, otherwise (and for
 * frame 0) all of R.  The output is that set sorted by (distance, index),
 * cut to its first k entries.  Written as that definition: the ring test over
 * all references, every candidate's distance, one sort.
 */
typedef struct { uint32_t d; int32_t r; } cand_t;

static int cmp_cand(const void* x, const void* y) {
  const cand_t* a = (const cand_t*)x;
  const cand_t* b = (const cand_t*)y;
  if (a->d != b->d) return a->d < b->d ? -1 : 1;
  return (a->r > b->r) - (a->r < b->r);
}

void oracle_riann_knn(const uint8_t* frame, int32_t H, int32_t W, int32_t C,
                      const uint8_t* R, int32_t n,
                      const uint8_t* KP, int32_t K, const uint32_t* P,
                      const int32_t* prev, int32_t alpha_num, int32_t alpha_den,
                      int32_t ring_limit, int32_t k,
                      const int64_t* qidx, int64_t nq,
                      int32_t* knn, uint32_t* knn_dist, uint32_t* count) {
  const int32_t D = PATCH * PATCH * C;
  const int32_t Wq = W - PATCH + 1;
  const int64_t Q = (int64_t)(H - PATCH + 1) * Wq;
  const int64_t N = qidx ? nq : Q;
#pragma omp parallel
  {
    uint8_t q[PATCH * PATCH * 3];
    uint32_t* B = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)K);
    uint32_t* ring_size = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)K);
    uint8_t* in_s = (uint8_t*)malloc((size_t)n);
    cand_t* cand = (cand_t*)malloc(sizeof(cand_t) * (size_t)n);
#pragma omp for schedule(dynamic, 16)
    for (int64_t i = 0; i < N; ++i) {
      int64_t qi = query_at(qidx, i);
      extract_query(frame, W, C, (int32_t)(qi / Wq), (int32_t)(qi % Wq), q);
      int all = 1;                                   /* candidate set = all of R */
      int32_t rp = -1;
      uint32_t s_size = 0;
      if (prev) {
        rp = prev[qi];
        const uint32_t Cd = sqdist(q, R + (int64_t)rp * D, D);
        for (int32_t m = 0; m < K; ++m) {
          B[m] = sqdist(q, KP + (int64_t)m * D, D);
          ring_size[m] = 0;
        }
        for (int32_t r = 0; r < n; ++r) {
          int inside = 1;
          for (int32_t m = 0; m < K; ++m) {
            int mem = oracle_ring_member(P[(int64_t)r * K + m], B[m], Cd, alpha_num, alpha_den);
            ring_size[m] += (uint32_t)mem;
            inside &= mem;
          }
          in_s[r] = (uint8_t)inside;
          s_size += (uint32_t)inside;
        }
        uint32_t ns = ring_size[0];
        for (int32_t m = 1; m < K; ++m) if (ring_size[m] < ns) ns = ring_size[m];
        all = ring_limit >= 0 && ns > (uint32_t)ring_limit;
      }
      int32_t nc = 0;
      for (int32_t r = 0; r < n; ++r) {
        if (all || in_s[r] || r == rp) {
          cand[nc].d = sqdist(q, R + (int64_t)r * D, D);
          cand[nc].r = r;
          ++nc;
        }
      }
      qsort(cand, (size_t)nc, sizeof(cand_t), cmp_cand);
      for (int32_t j = 0; j < k; ++j) {
        knn[i * k + j] = j < nc ? cand[j].r : -1;
        if (knn_dist) knn_dist[i * k + j] = j < nc ? cand[j].d : 0xffffffffu;
      }
      if (count) count[i] = all ? (uint32_t)n : s_size;
    }
    free(B); free(ring_size); free(in_s); free(cand);
  }
}

/*
 * Reference-set construction (Sec. 3.4: the collected patches are clustered
 * with a high-dimensional regression tree and each cluster is represented by
 * its median).  Reading taken here, all in integers on the uint8 patches:
 *   a node with more than `leaf` patches splits on the coordinate of largest
 *   variance (cnt * sum x^2 - (sum x)^2, lowest coordinate on ties) at the
 *   lower median m of that coordinate (the value of rank (cnt-1)/2):
 *   left = {x <= m} when that leaves the right side non-empty, else
 *   left = {x < m}; both sides keep their input order;
 *   a node is a leaf when it holds at most `leaf` patches or no coordinate
 *   varies;
 *   the leaves, in the order of the final arrangement (left before right),
 *   are the clusters; a cluster's representative is its per-coordinate lower
 *   median.  (The paper also normalises representatives to unit length; the
 *   uint8 reading of the query step drops that.)
 * assign[i] = cluster of input patch i.  Returns the number of clusters.
 */
static int cmp_u8(const void* x, const void* y) {
  return (int)*(const uint8_t*)x - (int)*(const uint8_t*)y;
}

static uint8_t lower_median(uint8_t* v, int32_t cnt) {
  qsort(v, (size_t)cnt, 1, cmp_u8);
  return v[(cnt - 1) / 2];
}

int32_t oracle_cluster_references(const uint8_t* X, int32_t n, int32_t D, int32_t leaf,
                                  uint8_t* reps, int32_t* assign) {
  int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  uint8_t* vals = (uint8_t*)malloc((size_t)(n > 0 ? n : 1));
  int32_t* stack = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)(n + 1));
  for (int32_t i = 0; i < n; ++i) perm[i] = i;
  int32_t top = 0, nclusters = 0;
  if (n > 0) { stack[0] = 0; stack[1] = n; top = 1; }
  while (top > 0) {                               /* depth first, left child first */
    --top;
    const int32_t b = stack[2 * top], e = stack[2 * top + 1], cnt = e - b;
    int32_t best_d = -1;
    unsigned long long best_v = 0;
    if (cnt > leaf) {
      for (int32_t d = 0; d < D; ++d) {
        unsigned long long s = 0, s2 = 0;
        for (int32_t i = b; i < e; ++i) {
          const unsigned long long x = X[(int64_t)perm[i] * D + d];
          s += x; s2 += x * x;
        }
        const unsigned long long v = (unsigned long long)cnt * s2 - s * s;
        if (v > best_v) { best_v = v; best_d = d; }
      }
    }
    uint8_t m = 0;
    int strict = 0;
    int32_t nl = 0;
    if (best_d >= 0) {
      for (int32_t i = b; i < e; ++i) vals[i - b] = X[(int64_t)perm[i] * D + best_d];
      m = lower_median(vals, cnt);
      int32_t nle = 0;
      for (int32_t i = b; i < e; ++i) nle += X[(int64_t)perm[i] * D + best_d] <= m;
      strict = nle == cnt;                        /* everything <= m: split off the values below m */
      for (int32_t i = b; i < e; ++i) {
        const uint8_t x = X[(int64_t)perm[i] * D + best_d];
        nl += strict ? x < m : x <= m;
      }
      /* both sides are non-empty whenever the coordinate varies; a split that
       * would leave one empty is never made */
      if (nl == 0 || nl == cnt) best_d = -1;
    }
    if (best_d < 0) {                             /* a leaf: one cluster */
      for (int32_t d = 0; d < D; ++d) {
        for (int32_t i = b; i < e; ++i) vals[i - b] = X[(int64_t)perm[i] * D + d];
        reps[(int64_t)nclusters * D + d] = lower_median(vals, cnt);
      }
      for (int32_t i = b; i < e; ++i) if (assign) assign[perm[i]] = nclusters;
      ++nclusters;
      continue;
    }
    int32_t nw = 0;
    for (int32_t i = b; i < e; ++i) {
      const uint8_t x = X[(int64_t)perm[i] * D + best_d];
      if (strict ? x < m : x <= m) tmp[b + nw++] = perm[i];
    }
    int32_t nr = nl;
    for (int32_t i = b; i < e; ++i) {
      const uint8_t x = X[(int64_t)perm[i] * D + best_d];
      if (!(strict ? x < m : x <= m)) tmp[b + nr++] = perm[i];
    }
    for (int32_t i = b; i < e; ++i) perm[i] = tmp[i];
    stack[2 * top] = b + nl; stack[2 * top + 1] = e; ++top;     /* right, processed after left */
    stack[2 * top] = b; stack[2 * top + 1] = b + nl; ++top;
  }
  free(perm); free(tmp); free(vals); free(stack);
  return nclusters;
}

/*
 * Unit-normalised float variant (Sec. 3.4: references scaled to length 1;
 * Alg. 1: the query patch is normalised at run time).  Every step is an IEEE
 * single-precision operation in a fixed order (this file is compiled with
 * -ffp-contract=off, so nothing is fused unless written as fmaf):
 *   normalise  s = sum of v_i^2 (exact integer); v'_i = v_i / sqrtf(s)
 *              (the zero patch stays zero)
 *   distance   d(a, b) = sqrtf(acc), acc = fmaf(t_i, t_i, acc) over
 *              i = 0 .. D-1 in order, t_i = a_i - b_i, acc starting at 0
 *   ring m     |A - B| <= T with A = d(k'_m, r'), B = d(k'_m, q'),
 *              T = (p * C) / q, C = d(q', r'_p)
 *   then S, the routing test and the argmin as in the integer step, on
 *   these float distances (ties: lower index).
 */
static void unit_normalize(const uint8_t* v, int32_t D, float* out) {
  uint32_t s = 0;
  for (int32_t i = 0; i < D; ++i) s += (uint32_t)v[i] * v[i];
  if (s == 0) {
    for (int32_t i = 0; i < D; ++i) out[i] = 0.f;
    return;
  }
  const float nv = sqrtf((float)s);
  for (int32_t i = 0; i < D; ++i) out[i] = (float)v[i] / nv;
}

static float unit_dist(const float* a, const float* b, int32_t D) {
  float acc = 0.f;
  for (int32_t i = 0; i < D; ++i) {
    const float t = a[i] - b[i];
    acc = fmaf(t, t, acc);
  }
  return sqrtf(acc);
}

void oracle_unit_normalize(const uint8_t* X, int32_t n, int32_t D, float* out) {
  for (int32_t r = 0; r < n; ++r) unit_normalize(X + (int64_t)r * D, D, out + (int64_t)r * D);
}

float oracle_unit_dist(const float* a, const float* b, int32_t D) { return unit_dist(a, b, D); }

int oracle_unit_ring_member(float A, float B, float C, int32_t p, int32_t q) {
  const float T = ((float)p * C) / (float)q;
  return fabsf(A - B) <= T;
}

static void unit_brute_force(const float* qn, const float* Rf, int32_t n, int32_t D, int32_t* bi, float* bd) {
  *bi = 0;
  *bd = unit_dist(qn, Rf, D);
  for (int32_t r = 1; r < n; ++r) {
    const float d = unit_dist(qn, Rf + (int64_t)r * D, D);
    if (d < *bd) { *bd = d; *bi = r; }
  }
}

void oracle_riann_unit(const uint8_t* frame, int32_t H, int32_t W, int32_t C,
                       const uint8_t* R, int32_t n, const uint8_t* KP, int32_t K,
                       const int32_t* prev, int32_t alpha_num, int32_t alpha_den, int32_t ring_limit,
                       const int64_t* qidx, int64_t nq,
                       int32_t* annf, float* dist, uint32_t* count) {
  const int32_t D = PATCH * PATCH * C;
  const int32_t Wq = W - PATCH + 1;
  const int64_t Q = (int64_t)(H - PATCH + 1) * Wq;
  const int64_t N = qidx ? nq : Q;
  float* Rf = (float*)malloc(sizeof(float) * (size_t)n * D);
  float* Kf = (float*)malloc(sizeof(float) * (size_t)K * D);
  float* A = (float*)malloc(sizeof(float) * (size_t)n * K);
  oracle_unit_normalize(R, n, D, Rf);
  oracle_unit_normalize(KP, K, D, Kf);
  for (int32_t r = 0; r < n; ++r)
    for (int32_t m = 0; m < K; ++m) A[(int64_t)r * K + m] = unit_dist(Kf + (int64_t)m * D, Rf + (int64_t)r * D, D);
#pragma omp parallel
  {
    uint8_t q[PATCH * PATCH * 3];
    float qn[PATCH * PATCH * 3];
    float* B = (float*)malloc(sizeof(float) * (size_t)K);
    uint32_t* ring_size = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)K);
    uint8_t* in_s = (uint8_t*)malloc((size_t)n);
#pragma omp for schedule(dynamic, 16)
    for (int64_t i = 0; i < N; ++i) {
      const int64_t qi = query_at(qidx, i);
      extract_query(frame, W, C, (int32_t)(qi / Wq), (int32_t)(qi % Wq), q);
      unit_normalize(q, D, qn);
      int32_t bi;
      float bd;
      if (!prev) {
        unit_brute_force(qn, Rf, n, D, &bi, &bd);
        annf[i] = bi; if (dist) dist[i] = bd; if (count) count[i] = (uint32_t)n;
        continue;
      }
      const int32_t rp = prev[qi];
      const float Cd = unit_dist(qn, Rf + (int64_t)rp * D, D);
      for (int32_t m = 0; m < K; ++m) {
        B[m] = unit_dist(Kf + (int64_t)m * D, qn, D);
        ring_size[m] = 0;
      }
      uint32_t s_size = 0;
      for (int32_t r = 0; r < n; ++r) {
        int inside = 1;
        for (int32_t m = 0; m < K; ++m) {
          const int mem = oracle_unit_ring_member(A[(int64_t)r * K + m], B[m], Cd, alpha_num, alpha_den);
          ring_size[m] += (uint32_t)mem;
          inside &= mem;
        }
        in_s[r] = (uint8_t)inside;
        s_size += (uint32_t)inside;
      }
      uint32_t ns = ring_size[0];
      for (int32_t m = 1; m < K; ++m) if (ring_size[m] < ns) ns = ring_size[m];
      if (ring_limit >= 0 && ns > (uint32_t)ring_limit) {
        unit_brute_force(qn, Rf, n, D, &bi, &bd);
        annf[i] = bi; if (dist) dist[i] = bd; if (count) count[i] = (uint32_t)n;
        continue;
      }
      bi = rp;
      bd = Cd;
      for (int32_t r = 0; r < n; ++r) {
        if (!in_s[r]) continue;
        const float d = unit_dist(qn, Rf + (int64_t)r * D, D);
        if (d < bd || (d == bd && r < bi)) { bd = d; bi = r; }
      }
      annf[i] = bi; if (dist) dist[i] = bd; if (count) count[i] = s_size;
    }
    free(B); free(ring_size); free(in_s);
  }
  free(Rf); free(Kf); free(A);
}

/* A sorted list splits into three runs around a ring: references below it
 * (not members, A < B), the members, and references above it (not members,
 * A > B).  The members are one contiguous run because |sqrt(A) - sqrt(B)|
 * falls and then rises as A grows. */
typedef struct { const uint32_t* a; uint32_t B, C; int32_t p, q; int below; } ring_pred_t;

/* below == 1: "strictly below the ring";  below == 0: "not above the ring".
 * Either predicate is true on a prefix of the sorted list. */
static int in_prefix(const ring_pred_t* s, uint32_t A) {
  int mem = oracle_ring_member(A, s->B, s->C, s->p, s->q);
  if (s->below) return !mem && A < s->B;
  return mem || A <= s->B;
}

/* first j in [lo, hi) where the prefix predicate is false (binary search) */
static int32_t partition_point(const ring_pred_t* s, int32_t lo, int32_t hi) {
  while (lo < hi) {
    int32_t mid = lo + (hi - lo) / 2;
    if (in_prefix(s, s->a[mid])) lo = mid + 1; else hi = mid;
  }
  return lo;
}

/*
 * Indexed mode (Sec. 3.3): each ring is found with two binary searches in the
 * sorted list of its anchor; the candidates are the members of the smallest
 * ring that lie inside every other ring; then the argmin of Alg. 1.
 */
void oracle_riann_indexed(const uint8_t* frame, int32_t H, int32_t W, int32_t C,
                          const uint8_t* R, int32_t n,
                          const uint8_t* KP, int32_t K, const uint32_t* P,
                          const uint32_t* TA, const int32_t* Tid,
                          const int32_t* prev, int32_t alpha_num, int32_t alpha_den,
                          int32_t ring_limit,
                          const int64_t* qidx, int64_t nq,
                          int32_t* annf, uint32_t* dist, uint32_t* count, uint32_t* nseed) {
  const int32_t D = PATCH * PATCH * C;
  const int32_t Wq = W - PATCH + 1;
  const int64_t Q = (int64_t)(H - PATCH + 1) * Wq;
  const int64_t N = qidx ? nq : Q;
#pragma omp parallel
  {
    uint8_t q[PATCH * PATCH * 3];
    uint32_t* B = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)K);
    int32_t* lo = (int32_t*)malloc(sizeof(int32_t) * (size_t)K);
    int32_t* hi = (int32_t*)malloc(sizeof(int32_t) * (size_t)K);
#pragma omp for schedule(dynamic, 16)
    for (int64_t i = 0; i < N; ++i) {
      int64_t qi = query_at(qidx, i);
      extract_query(frame, W, C, (int32_t)(qi / Wq), (int32_t)(qi % Wq), q);
      if (!prev) {
        int32_t bi; uint32_t bd;
        brute_force(q, R, n, D, &bi, &bd);
        annf[i] = bi;
        if (dist) dist[i] = bd;
        if (count) count[i] = (uint32_t)n;
        if (nseed) nseed[i] = 0;
        continue;
      }
      const int32_t rp = prev[qi];
      const uint32_t Cd = sqdist(q, R + (int64_t)rp * D, D);
      int32_t seed = 0;
      for (int32_t m = 0; m < K; ++m) {
        B[m] = sqdist(q, KP + (int64_t)m * D, D);
        ring_pred_t s = { TA + (int64_t)m * n, B[m], Cd, alpha_num, alpha_den, 1 };
        lo[m] = partition_point(&s, 0, n);
        s.below = 0;
        hi[m] = partition_point(&s, lo[m], n);
        if (hi[m] - lo[m] < hi[seed] - lo[seed]) seed = m;
      }
      const uint32_t ns = (uint32_t)(hi[seed] - lo[seed]);
      if (nseed) nseed[i] = ns;
      if (ring_limit >= 0 && ns > (uint32_t)ring_limit) {
        int32_t bi; uint32_t bd;
        brute_force(q, R, n, D, &bi, &bd);
        annf[i] = bi;
        if (dist) dist[i] = bd;
        if (count) count[i] = (uint32_t)n;
        continue;
      }
      int32_t bi = rp;
      uint32_t bd = Cd, s_size = 0;
      for (int32_t j = lo[seed]; j < hi[seed]; ++j) {
        const int32_t r = Tid[(int64_t)seed * n + j];
        int inside = 1;
        for (int32_t m = 0; m < K && inside; ++m) {
          if (m == seed) continue;
          inside = oracle_ring_member(P[(int64_t)r * K + m], B[m], Cd, alpha_num, alpha_den);
        }
        if (!inside) continue;
        ++s_size;
        uint32_t d = sqdist(q, R + (int64_t)r * D, D);
        if (d < bd || (d == bd && r < bi)) { bd = d; bi = r; }
      }
      annf[i] = bi;
      if (dist) dist[i] = bd;
      if (count) count[i] = s_size;
    }
    free(B); free(lo); free(hi);
  }
}

/* Sec. 4 reconstruction, written as its definition: for every output pixel,
 * the query patches that cover it are those with top-left corner
 * y-7 <= py <= y and x-7 <= px <= x inside the query grid.  R is the table
 * the matched rows are read from: the references themselves (Sec. 4), or a
 * transformed copy T(R) for an effect by patch replacement (Sec. 5). */
void oracle_reconstruct(const uint8_t* R, int32_t n, int32_t C, const int32_t* annf, int32_t H, int32_t W,
                        const uint8_t* frame, uint8_t* out, unsigned long long* err2) {
  const int32_t Hq = H - 7, Wq = W - 7, D = 64 * C;
  unsigned long long e = 0, g = 0;
  for (int32_t y = 0; y < H; ++y) {
    for (int32_t x = 0; x < W; ++x) {
      for (int32_t c = 0; c < C; ++c) {
        uint64_t sum = 0, count = 0;
        for (int32_t py = (y - 7 > 0 ? y - 7 : 0); py <= y && py < Hq; ++py) {
          for (int32_t px = (x - 7 > 0 ? x - 7 : 0); px <= x && px < Wq; ++px) {
            const int32_t r = annf[(int64_t)py * Wq + px];
            if (r < 0 || r >= n) continue;
            sum += R[(int64_t)r * D + ((int64_t)(y - py) * 8 + (x - px)) * C + c];
            ++count;
          }
        }
        const uint32_t v = count ? (uint32_t)((2 * sum + count) / (2 * count)) : 0u;
        const int64_t o = ((int64_t)y * W + x) * C + c;
        if (out) out[o] = (uint8_t)v;
        if (frame) {
          const int64_t d = (int64_t)frame[o] - (int64_t)v;
          e += (unsigned long long)(d * d);
          g += (unsigned long long)frame[o] * frame[o];
        }
      }
    }
  }
  if (err2) {
    err2[0] = e;
    err2[1] = g;
  }
}

/* ---- Alg. 1 with random anchors ------------------------------------------ */

/* Philox4x32-10 as published: ten rounds of two 32x32->64-bit products with
 * the multipliers 0xD2511F53 and 0xCD9E8D57, the key bumped by the Weyl
 * constants 0x9E3779B9 and 0xBB67AE85 between rounds. */
void oracle_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static int cmp_u64(const void* x, const void* y) {
  const uint64_t u = *(const uint64_t*)x, v = *(const uint64_t*)y;
  return u < v ? -1 : (u > v ? 1 : 0);
}

/* Sec. 3.4: the pairwise distances, each row sorted. */
void oracle_full_tables(const uint8_t* R, int32_t n, int32_t D, uint64_t* T) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int32_t i = 0; i < n; ++i) {
    uint64_t* row = T + (int64_t)i * n;
    for (int32_t j = 0; j < n; ++j)
      row[j] = ((uint64_t)sqdist(R + (int64_t)i * D, R + (int64_t)j * D, D) << 32) | (uint32_t)j;
    qsort(row, (size_t)n, sizeof(uint64_t), cmp_u64);
  }
}

/* r in the ring of the anchor: (1 - a) d <= dist(anchor, r) <= (1 + a) d with
 * d = dist(q, anchor), a = p/q, squared: A = ||anchor - r||^2, B = ||q - anchor||^2 */
static int anchor_ring_member(uint32_t A, uint32_t B, int32_t p, int32_t q) {
  const uint64_t qq = (uint64_t)q * (uint64_t)q;
  if (p < q) {
    const uint64_t lo = (uint64_t)(q - p) * (uint64_t)(q - p);
    if (lo * B > qq * A) return 0;
  }
  const uint64_t hi = (uint64_t)(q + p) * (uint64_t)(q + p);
  return qq * A <= hi * B;
}

void oracle_riann_anchor(const uint8_t* frame, int32_t H, int32_t W, int32_t C,
                         const uint8_t* R, int32_t n, const uint64_t* T, const int32_t* prev,
                         int32_t alpha_num, int32_t alpha_den, int32_t L, int32_t max_rings,
                         uint64_t seed, uint32_t frame_id,
                         const int64_t* qidx, int64_t nq,
                         int32_t* annf, uint32_t* dist, uint32_t* count, uint32_t* rings) {
  const int32_t D = 64 * C, Wq = W - 7;
  const int64_t Q = (int64_t)(H - 7) * Wq;
  const int64_t NQ = qidx ? nq : Q;
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
#pragma omp parallel
  {
    uint8_t q[192];
    int32_t* S = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    int32_t* S2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
#pragma omp for schedule(dynamic, 16)
    for (int64_t i = 0; i < NQ; ++i) {
      const int64_t qi = query_at(qidx, i);
      extract_query(frame, W, C, (int32_t)(qi / Wq), (int32_t)(qi % Wq), q);
      if (!prev) {
        int32_t bi; uint32_t bd;
        brute_force(q, R, n, D, &bi, &bd);
        annf[i] = bi;
        if (dist) dist[i] = bd;
        if (count) count[i] = (uint32_t)n;
        if (rings) rings[i] = 0;
        continue;
      }
      const int32_t ri = prev[qi];
      const uint32_t Bi = sqdist(q, R + (int64_t)ri * D, D);
      int32_t bi = ri;                      /* best so far: r_i, then the anchors, then S */
      uint32_t bd = Bi;
      /* S_0: the ring of r_i, in row r_i of the sorted matrix */
      int32_t ns = 0;
      const uint64_t* row = T + (int64_t)ri * n;
      for (int32_t j = 0; j < n; ++j)
        if (anchor_ring_member((uint32_t)(row[j] >> 32), Bi, alpha_num, alpha_den)) S[ns++] = (int32_t)(uint32_t)row[j];
      uint32_t t = 0;
      while (ns >= L && (int32_t)t < max_rings) {
        const uint32_t ctr[4] = {(uint32_t)qi, t, frame_id, 0u};
        uint32_t x[4];
        oracle_philox4x32_10(ctr, key, x);
        const int32_t a = S[(int32_t)(((uint64_t)x[0] * (uint64_t)ns) >> 32)];
        const uint32_t Ba = sqdist(q, R + (int64_t)a * D, D);
        if (Ba < bd || (Ba == bd && a < bi)) { bd = Ba; bi = a; }
        int32_t m = 0;
        for (int32_t k = 0; k < ns; ++k) {
          const uint32_t A = sqdist(R + (int64_t)a * D, R + (int64_t)S[k] * D, D);
          if (anchor_ring_member(A, Ba, alpha_num, alpha_den)) S2[m++] = S[k];
        }
        int32_t* tmp = S; S = S2; S2 = tmp;
        ns = m;
        ++t;
      }
      for (int32_t k = 0; k < ns; ++k) {
        const uint32_t d = sqdist(q, R + (int64_t)S[k] * D, D);
        if (d < bd || (d == bd && S[k] < bi)) { bd = d; bi = S[k]; }
      }
      annf[i] = bi;
      if (dist) dist[i] = bd;
      if (count) count[i] = (uint32_t)ns;
      if (rings) rings[i] = t;
    }
    free(S); free(S2);
  }
}

void oracle_random_field(int32_t H, int32_t W, int32_t n, uint64_t seed, uint32_t frame_id, int32_t* annf) {
  const int64_t Q = (int64_t)(H - 7) * (W - 7);
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int64_t q = 0; q < Q; ++q) {
    const uint32_t ctr[4] = {(uint32_t)q, 0u, frame_id, 1u};
    uint32_t x[4];
    oracle_philox4x32_10(ctr, key, x);
    annf[q] = (int32_t)(((uint64_t)x[0] * (uint64_t)(uint32_t)n) >> 32);
  }
}
