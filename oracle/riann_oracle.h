/*
 * riann_oracle.h -- plain, slow, obviously-correct CPU oracle for RIANN's
 * per-frame query step (Ben-Zrihem & Zelnik-Manor, "Approximate Nearest
 * Neighbor Fields in Video", arXiv 1508.07953).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline of the benchmark call this code.  It shares no code with the CUDA
 * library and includes none of its headers.
 *
 * Conventions (all integer):
 *   patch      8x8xC uint8, vector order (dy, dx, c)  -- D = 64*C bytes
 *   frame      uint8 [H][W][C], row-major
 *   query q    top-left corner (y, x), 0 <= y < H-7, 0 <= x < W-7,
 *              query index = y*(W-7) + x                      (Sec. 4: all patches)
 *   dist       squared L2 over the D bytes, exact in uint32  (<= 192*255^2)
 *   ANN field  int32 [H-7][W-7] of 0-based reference indices  (Alg. 1 output)
 *
 * Reading of the method taken here (fixed key points, Sec. 3.2 rings):
 *   ring of key point k_m for query q, with previous match r_p:
 *       Ring_m = { r : | ||k_m - r|| - ||k_m - q|| | <= alpha * ||q - r_p|| }
 *   (rings of Sec. 3.2 / Alg. 1, with the anchors fixed to K key points and the
 *    half-width epsilon = alpha * dist(q, r_p) of Alg. 1's first ring for all rings)
 *   S = intersection of all K rings;  N_seed = min_m |Ring_m|
 *   if N_seed > ring_limit (ring_limit >= 0): brute force over all of R, count = n
 *   else ANNF(q) = argmin over S u {r_p} of dist(q, r), count = |S|
 *   with ties broken by the lower reference index.
 *   Frame 0 (no previous field): brute force, count = n.
 */
#ifndef RIANN_ORACLE_H
#define RIANN_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Exact ring membership |sqrt(A) - sqrt(B)| <= (p/q) sqrt(C) (Sec. 3.2). */
int oracle_ring_member(uint32_t A, uint32_t B, uint32_t C, int32_t p, int32_t q);

/* P[r*K + m] = ||k_m - R_r||^2 (Sec. 3.3 pre-processing, restricted to key points). */
void oracle_key_distances(const uint8_t* R, int32_t n, int32_t D,
                          const uint8_t* KP, int32_t K, uint32_t* P);

/* Per key point m, the references sorted ascending by (P[r][m], r):
 * TA[m*n + j] = distance, Tid[m*n + j] = reference index (Sec. 3.3 sorted lists). */
void oracle_sort_tables(const uint32_t* P, int32_t n, int32_t K, uint32_t* TA, int32_t* Tid);

/* Exact nearest neighbour by brute force (frame-0 initialisation).
 * qidx: optional list of nq query indices (NULL = all, nq ignored);
 * outputs are indexed by list position.  count[i] = n. */
void oracle_exact_nn(const uint8_t* frame, int32_t H, int32_t W, int32_t C,
                     const uint8_t* R, int32_t n,
                     const int64_t* qidx, int64_t nq,
                     int32_t* annf, uint32_t* dist, uint32_t* count);

/* RIANN query step, definitional mode: every ring is evaluated by the exact
 * predicate over all n references.  prev == NULL means frame 0 (brute force).
 * nseed (nullable) receives min_m |Ring_m| (0 for brute-forced frame-0 queries). */
void oracle_riann_definitional(const uint8_t* frame, int32_t H, int32_t W, int32_t C,
                               const uint8_t* R, int32_t n,
                               const uint8_t* KP, int32_t K, const uint32_t* P,
                               const int32_t* prev, int32_t alpha_num, int32_t alpha_den,
                               int32_t ring_limit,
                               const int64_t* qidx, int64_t nq,
                               int32_t* annf, uint32_t* dist, uint32_t* count, uint32_t* nseed);

/* RIANN query step, indexed mode: ring bounds by binary search on the sorted
 * per-key lists (Sec. 3.3: two binary searches per ring), candidates enumerated from
 * the smallest ring and filtered by the other rings. */
void oracle_riann_indexed(const uint8_t* frame, int32_t H, int32_t W, int32_t C,
                          const uint8_t* R, int32_t n,
                          const uint8_t* KP, int32_t K, const uint32_t* P,
                          const uint32_t* TA, const int32_t* Tid,
                          const int32_t* prev, int32_t alpha_num, int32_t alpha_den,
                          int32_t ring_limit,
                          const int64_t* qidx, int64_t nq,
                          int32_t* annf, uint32_t* dist, uint32_t* count, uint32_t* nseed);

/* k-NN output (Sec. 7: more than one match per query): the set the argmin of
 * oracle_riann_definitional ranges over -- S u {r_p} (r_p once), or all of R
 * for frame 0 / rings too wide -- sorted by (dist, index) and cut to its first
 * k entries: knn[i*k + j], knn_dist[i*k + j] (nullable); -1 / UINT32_MAX past
 * the size of the set.  count as oracle_riann_definitional. */
void oracle_riann_knn(const uint8_t* frame, int32_t H, int32_t W, int32_t C,
                      const uint8_t* R, int32_t n,
                      const uint8_t* KP, int32_t K, const uint32_t* P,
                      const int32_t* prev, int32_t alpha_num, int32_t alpha_den,
                      int32_t ring_limit, int32_t k,
                      const int64_t* qidx, int64_t nq,
                      int32_t* knn, uint32_t* knn_dist, uint32_t* count);

/* Reference-set construction (Sec. 3.4: regression-tree clusters, each
 * represented by its median).  X: n patches of D bytes.  A node with more
 * than `leaf` patches splits on its coordinate of largest variance (integer
 * cnt*sum(x^2) - sum(x)^2, lowest coordinate on ties) at that coordinate's
 * lower median m: {x <= m} go left unless that is every patch, then {x < m};
 * order is kept on both sides.  Leaves (at most `leaf` patches, or no
 * variance) in left-to-right order are the clusters; reps[c*D + d] = lower
 * median of coordinate d over cluster c; assign[i] (nullable) = cluster of
 * patch i.  Returns the number of clusters (reps must hold n rows). */
int32_t oracle_cluster_references(const uint8_t* X, int32_t n, int32_t D, int32_t leaf,
                                  uint8_t* reps, int32_t* assign);

/* ---- unit-normalised float variant (Sec. 3.4 / Alg. 1: unit-length patches) ----
 * IEEE single precision in a fixed order:
 *   normalise  v'_i = v_i / sqrtf(sum v_i^2) (the zero patch stays zero)
 *   distance   d(a, b) = sqrtf(acc), acc = fmaf(t_i, t_i, acc) for i = 0..D-1, t_i = a_i - b_i
 *   ring m     |A - B| <= (p * C) / q  (A = d(k'_m, r'), B = d(k'_m, q'), C = d(q', r'_p))
 * and S, routing and the argmin of oracle_riann_definitional on those
 * distances; dist receives the float distance of the answer. */
void oracle_unit_normalize(const uint8_t* X, int32_t n, int32_t D, float* out);
float oracle_unit_dist(const float* a, const float* b, int32_t D);
int oracle_unit_ring_member(float A, float B, float C, int32_t p, int32_t q);
void oracle_riann_unit(const uint8_t* frame, int32_t H, int32_t W, int32_t C,
                       const uint8_t* R, int32_t n, const uint8_t* KP, int32_t K,
                       const int32_t* prev, int32_t alpha_num, int32_t alpha_den, int32_t ring_limit,
                       const int64_t* qidx, int64_t nq,
                       int32_t* annf, float* dist, uint32_t* count);

/* Reconstruction by patch replacement (Sec. 4: every patch is replaced by
 * its match and the overlaps are averaged).  out[y][x][c] = rounded
 * average over the query patches (py, px) that cover (y, x) -- py <= y < py+8,
 * px <= x < px+8, inside the query grid, with annf[py][px] in [0, n) -- of
 * byte (y-py, x-px, c) of their matched reference patch.  Reading taken here:
 * the average is rounded half up to 8 bits, (2*sum + count) / (2*count) in
 * integers (0 where no valid patch covers the pixel).  frame / err2 nullable:
 * err2[0] = sum over all bytes of (frame - out)^2, err2[1] = sum of frame^2,
 * so that the paper's error E = ||f_GT - f_R|| / ||f_GT|| = sqrt(err2[0] / err2[1]). */
void oracle_reconstruct(const uint8_t* R, int32_t n, int32_t C, const int32_t* annf, int32_t H, int32_t W,
                        const uint8_t* frame, uint8_t* out, unsigned long long* err2);

/* ---- Alg. 1 with random anchors (the paper's own loop) ----------------- */

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11): counter ctr[4] and key key[2] -> out[4]. */
void oracle_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out);

/* Sec. 3.3 / Sec. 3.4, the sorted matrix of pairwise distances: T[i*n + j] = (A << 32) | id,
 * row i holding every reference sorted ascending by (A = ||r_i - r_id||^2, id). */
void oracle_full_tables(const uint8_t* R, int32_t n, int32_t D, uint64_t* T);

/* One frame of Alg. 1 for the queries of a frame with a previous field.
 * Readings taken here (alpha = p/q):
 *   ring of anchor a for query q: (1 - alpha) d_a <= dist(a, r) <= (1 + alpha) d_a
 *     with d_a = dist(q, a) (Alg. 1: eps = alpha * d), decided exactly in integers:
 *     (q - p)^2 ||q - a||^2 <= q^2 ||a - r||^2 (when p < q) and
 *     q^2 ||a - r||^2 <= (q + p)^2 ||q - a||^2;
 *   S_0 = ring of r_i = prev[q] (a range of row r_i of T), kept in that row's order;
 *   while |S| >= L and fewer than max_rings anchors were drawn:
 *     anchor = S[(x * |S|) >> 32], x the first word of Philox4x32-10 with
 *     counter (query index, ring number t = 0, 1, ..., frame_id, 0) and key
 *     (seed low word, seed high word);  S <- S n ring(anchor), order kept;
 *   answer = argmin of dist(q, r) over S u {r_i} u {anchors drawn}, lower index
 *     on ties (every one of them had its distance computed);
 *   count = |S| at the end, rings = anchors drawn.
 * prev == NULL: brute force (count = n, rings = 0). */
void oracle_riann_anchor(const uint8_t* frame, int32_t H, int32_t W, int32_t C,
                         const uint8_t* R, int32_t n, const uint64_t* T, const int32_t* prev,
                         int32_t alpha_num, int32_t alpha_den, int32_t L, int32_t max_rings,
                         uint64_t seed, uint32_t frame_id,
                         const int64_t* qidx, int64_t nq,
                         int32_t* annf, uint32_t* dist, uint32_t* count, uint32_t* rings);

/* Alg. 1's random initial field (each entry uniform over the references;
 * 0-based here): entry q =
 * (x * n) >> 32, x the first word of Philox4x32-10 with counter
 * (q, 0, frame_id, 1) and key (seed low, seed high). */
void oracle_random_field(int32_t H, int32_t W, int32_t n, uint64_t seed, uint32_t frame_id, int32_t* annf);

/* Number of OpenMP threads the oracle uses (1 when built without OpenMP). */
int oracle_num_threads(void);
void oracle_set_num_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
