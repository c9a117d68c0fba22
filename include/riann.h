/*
 * riann.h -- C ABI of the RIANN per-frame query engine for NVIDIA GB300
 * (sm_103a).  RIANN: Ben-Zrihem & Zelnik-Manor, "Approximate Nearest Neighbor
 * Fields in Video" (arXiv 1508.07953).
 *
 * Problem (Sec. 1, Fig. 1; Alg. 1 inputs/outputs): a fixed set R of n
 * reference patches, a stream of video frames, and for every frame a dense
 * ANN field: for each overlapping 8x8 patch of the frame, the index of a near
 * reference patch.
 *
 * Layouts (all integer, all row-major, no padding):
 *   patch      uint8 [8][8][C], element order (dy, dx, c); D = 64*C; C in {1, 3}
 *   frame      uint8 [H][W][C]
 *   ANN field  int32 [H-7][W-7]; entry (y, x) belongs to the patch whose
 *              top-left pixel is (y, x) (stride 1, valid region only)
 *   distance   squared L2 over the D bytes, uint32 (at most 192*255^2)
 *
 * Method as computed here (fixed key points k_0..k_{K-1}; Sec. 3.2, Alg. 1):
 *   eps(q)   = alpha * ||q - r_p||, r_p = previous field at the same position
 *   Ring_m   = { r : | ||k_m - r|| - ||k_m - q|| | <= eps(q) }   (closed, exact)
 *   S        = intersection of the K rings
 *   if min_m |Ring_m| > ring_limit (ring_limit >= 0): brute force over R,
 *       count = n
 *   else field(q) = argmin over S u {r_p} of ||q - r||^2, count = |S|
 *   ties go to the lower reference index.  With no previous field (frame 0,
 *   Alg. 1's initialisation step) every query is answered by brute force.
 * Membership is decided exactly in integers, so results are bit-reproducible.
 *
 * Memory ownership: the caller owns every buffer it passes in; the library
 * owns what it allocates (index tables, scratch) and frees it in the matching
 * destroy call.  Device pointers must point to memory of the current device.
 *
 * Execution: every call is asynchronous on the given stream unless its
 * comment says otherwise.  Calls that share an index share its scratch, so
 * they must be ordered on one stream (or use separate sessions).
 *
 * Errors: every int-returning call returns RIANN_OK (0) or one of the codes
 * below; argument errors are detected on the host before any work is queued.
 * Errors found by a kernel (e.g. a previous-field entry outside [0, n)) are
 * OR-ed into a per-index device status word read by riann_status().
 */
#ifndef RIANN_H
#define RIANN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL is the legacy default stream. */
struct CUstream_st;
typedef struct CUstream_st* riann_stream_t;

typedef struct riann_index_s* riann_index_t;

enum {
  RIANN_OK = 0,
  RIANN_ERR_INVALID_ARG = 1,  /* a size, pointer or parameter is out of range   */
  RIANN_ERR_OOM = 2,          /* a device or pinned-host allocation failed        */
  RIANN_ERR_UNSUPPORTED = 3,  /* device is not sm_103 / feature not built         */
  RIANN_ERR_CUDA = 4,         /* a CUDA runtime call failed                       */
  RIANN_ERR_TIMEOUT = 5,      /* a bounded device wait gave up                    */
  RIANN_ERR_ADMISSION = 6,    /* server: the stream does not fit the budget       */
  RIANN_ERR_DEVICE = 7,       /* a kernel reported bad input (see riann_status)   */
  RIANN_ERR_TOO_LARGE = 8     /* more queries than a fixed scratch or batch context holds */
};

/* Bits of the device status word. */
#define RIANN_DEV_BAD_PREV 0x1u   /* a previous-field entry was outside [0, n)  */
#define RIANN_DEV_BOUNDS 0x2u     /* checked build: a table index was out of range
                                     (the access was skipped)                    */
#define RIANN_DEV_TIMEOUT 0x4u    /* a bounded spin-wait in a kernel gave up      */

typedef struct {
  /* Ring half-width eps = (alpha_num / alpha_den) * dist(q, r_p)
   * (Sec. 3.2: the ring half-width is alpha times the distance from the query
   * to its previous match; the paper uses alpha = 0.25).
   * 1 <= alpha_den <= 8, 0 <= alpha_num <= 8 * alpha_den. */
  int32_t alpha_num;
  int32_t alpha_den;
  /* A query whose smallest ring holds more than ring_limit references is
   * answered by brute force over all of R (count = n).  -1: never. */
  int32_t ring_limit;
  /* Performance knob only; results never depend on it.  0 = the index's
   * tuned setting; 1..4 = number of 4-ring code groups the candidate scan
   * tests before it compacts survivors (see riann_autotune). */
  int32_t cap;
} riann_params;

/* alpha = 1/4 (Sec. 3.2), ring_limit = n/8, cap = 0. */
riann_params riann_default_params(int32_t n);

typedef struct {
  int32_t n, K, channels, dim;   /* dim = 64 * channels */
  size_t device_bytes;           /* bytes of device memory the index holds */
  int32_t unit;                  /* 1: unit-normalised float index (riann_build_unit_index) */
} riann_index_info_t;

/*
 * Pre-processing (Sec. 3.3: every anchor keeps its distances to the
 * references as a sorted list, computed once; Sec. 3.4: the reference model).
 * Copies the n reference patches and K key points, computes every
 * key-point-to-reference distance and, per key point, the references sorted by
 * (distance, index); also a bf16 copy of R for the brute-force path.
 *   d_patches   device uint8 [n][8][8][channels]; 1 <= n <= 2^24
 *   d_keypoints device uint8 [K][8][8][channels]; 1 <= K <= 64
 *   channels    1 or 3
 * Asynchronous on `stream`; inputs may be freed once the stream reaches the
 * end of the build.  *out receives the handle (NULL on error).
 */
int riann_build_reference_index(const uint8_t* d_patches, int32_t n, int32_t channels,
                                const uint8_t* d_keypoints, int32_t K,
                                riann_stream_t stream, riann_index_t* out);

/*
 * riann_build_reference_index with a choice of scan order (performance only:
 * every order gives identical results).  For each key point the index also
 * keeps the references in a "pair order": sorted by (7-bit bucket of the
 * distance to the key point, 7-bit bucket of the distance to a partner key
 * point), then as in the key's sorted list; a query whose seed ring is that
 * key's scans only the buckets where both rings' code ranges meet.
 *   scan_order  RIANN_SCAN_AUTO: RIANN_SCAN_PAIRS for n >= 16384, else
 *                 RIANN_SCAN_SINGLE (smaller buckets fragment the runs);
 *               RIANN_SCAN_PAIRS: partner = the farthest other key point;
 *               RIANN_SCAN_SINGLE: partner = the key itself (the pair order is
 *                 its sorted list; the scan visits the seed ring's exact run).
 * Errors as riann_build_reference_index, plus RIANN_ERR_INVALID_ARG for an
 * unknown scan_order.
 */
#define RIANN_SCAN_AUTO 0
#define RIANN_SCAN_PAIRS 1
#define RIANN_SCAN_SINGLE 2
int riann_build_reference_index_ex(const uint8_t* d_patches, int32_t n, int32_t channels,
                                   const uint8_t* d_keypoints, int32_t K, int32_t scan_order,
                                   riann_stream_t stream, riann_index_t* out);

/*
 * Unit-normalised float variant (Sec. 3.4: representatives scaled to length
 * 1; Alg. 1: the query normalised at run time).  Same arguments as
 * riann_build_reference_index.  Every distance of the method is then the L2
 * distance between unit-length patches, in IEEE single precision with a fixed
 * order of operations:
 *   normalise  v'_i = v_i / sqrt(sum v_i^2) (correctly rounded; the zero
 *              patch stays zero)
 *   distance   d(a, b) = sqrt(acc), acc = fma(t_i, t_i, acc) for
 *              i = 0 .. D-1 in (dy, dx, c) order, t_i = a_i - b_i, from 0
 *   ring m     |fl(A - B)| <= T, T = fl(fl(alpha_num * C) / alpha_den)
 *   answer     argmin of d over S u {r_p} (lower index on ties); routing and
 *              count as for the integer index
 * On such an index riann_annf_frame and riann_exact_nn write d as float32 bit
 * patterns into d_out_dist; sessions and riann_reconstruct work as usual.
 * k-NN, batch contexts, servers, the anchor loop and the allocation-free
 * brute force return RIANN_ERR_UNSUPPORTED.  Its brute force runs on the CUDA
 * cores (the fixed fp32 order has no tensor-core equivalent).
 */
int riann_build_unit_index(const uint8_t* d_patches, int32_t n, int32_t channels,
                           const uint8_t* d_keypoints, int32_t K,
                           riann_stream_t stream, riann_index_t* out);

/* Synchronises the device and frees the index and its scratch.  NULL is a no-op. */
void riann_index_destroy(riann_index_t idx);

int riann_index_info(riann_index_t idx, riann_index_info_t* out);

/*
 * Copies the pre-processed tables into caller buffers (device or host
 * pointers; each nullable), for inspection and testing (Sec. 3.3 lists):
 *   P    uint32 [n][K]  squared distance of reference r to key point m
 *   TA   uint32 [K][n]  per key point, those distances in ascending order
 *   Tid  int32  [K][n]  per key point, the reference index of each TA entry
 *                       (ties in distance ordered by index)
 * Synchronous (returns after the copies completed on `stream`).
 */
int riann_index_tables(riann_index_t idx, riann_stream_t stream,
                       uint32_t* P, uint32_t* TA, int32_t* Tid);

/*
 * One RIANN query step over a whole frame (Alg. 1, one iteration of the
 * frame loop: every query patch of the frame).
 *   d_frame       device uint8 [H][W][channels]; 8 <= H, W; (H-7)*(W-7) < 2^31
 *   d_prev_annf   device int32 [H-7][W-7], the previous field; NULL = frame 0
 *                 (every query answered by brute force, Alg. 1's initialisation)
 *   d_out_annf    device int32 [H-7][W-7] (required; may not alias d_prev_annf)
 *   d_out_dist    device uint32 [H-7][W-7], squared distance of the match (nullable)
 *   d_out_count   device uint32 [H-7][W-7], |S| or n for brute force (nullable)
 * Asynchronous on `stream`.  Uses the index's scratch (grown on first use of
 * a larger frame, which allocates and synchronises).
 */
int riann_annf_frame(riann_index_t idx, const riann_params* p, riann_stream_t stream,
                     const uint8_t* d_frame, int32_t H, int32_t W,
                     const int32_t* d_prev_annf, int32_t* d_out_annf,
                     uint32_t* d_out_dist, uint32_t* d_out_count);

/*
 * k-NN variant of riann_annf_frame (Sec. 7: the method can return more than
 * one match per query).  The candidate set of a query is the one the
 * argmin of riann_annf_frame ranges over -- S u {r_p} (r_p counted once) for a
 * ring-answered query, all n references for frame 0 and for queries routed to
 * brute force -- and the output is its k smallest entries in ascending
 * (distance, index) order:
 *   k               1 <= k <= RIANN_KNN_MAX
 *   d_out_annf      device int32 [H-7][W-7]: the first of them (required; the
 *                   field the next frame takes as d_prev_annf, equal to
 *                   riann_annf_frame's output)
 *   d_out_knn       device int32 [H-7][W-7][k] (required); entries past the
 *                   size of the candidate set are -1
 *   d_out_knn_dist  device uint32 [H-7][W-7][k], squared distances (nullable);
 *                   0xFFFFFFFF past the size of the candidate set
 *   d_out_count     as riann_annf_frame
 * Neither output may alias d_prev_annf.  The first call on a larger frame also
 * grows the brute-force path's k-NN scratch (128 bytes per query, at least
 * 10 MB; allocates and synchronises).  Single-frame form only (no session or batch
 * variant).
 */
#define RIANN_KNN_MAX 8
int riann_knn_frame(riann_index_t idx, const riann_params* p, riann_stream_t stream,
                    const uint8_t* d_frame, int32_t H, int32_t W,
                    const int32_t* d_prev_annf, int32_t k, int32_t* d_out_annf,
                    int32_t* d_out_knn, uint32_t* d_out_knn_dist, uint32_t* d_out_count);

/*
 * Reference-set construction (Sec. 3.4: the collected patches are clustered
 * with a high-dimensional regression tree, each cluster represented by its
 * median).  Integer reading on the uint8 patches: a node with more than
 * `leaf` patches splits on its coordinate of largest variance
 * (cnt * sum x^2 - (sum x)^2, lowest coordinate on ties) at that
 * coordinate's lower median m (the value of rank (cnt-1)/2): {x <= m} go
 * left, or {x < m} when that would be every patch; both sides keep their
 * order.  Leaves (at most `leaf` patches, or no varying coordinate) are the
 * clusters, numbered left to right; a cluster's representative is its
 * per-coordinate lower median.  (The paper also scales representatives to
 * unit length; the uint8 query path has no use for that.)
 *   d_patches     device uint8 [n][8][8][channels], 1 <= n, channels 1 or 3
 *   leaf          largest cluster that is not split further, >= 1
 *   d_out_reps    device uint8 [n][8][8][channels] (room for n clusters); rows
 *                 0 .. *out_count - 1 receive the representatives
 *   d_out_assign  device int32 [n], cluster of each input patch (nullable)
 *   out_count     host: number of clusters
 * Synchronous: takes its scratch from the stream-ordered memory pool (4 x 4 +
 * 1 bytes per patch plus two node lists), builds the tree level by level (one launch and one small
 * device-to-host read per level) and returns when the outputs are written.
 */
int riann_cluster_references(riann_stream_t stream, const uint8_t* d_patches, int32_t n, int32_t channels,
                             int32_t leaf, uint8_t* d_out_reps, int32_t* d_out_assign, int32_t* out_count);

/*
 * 3-D spatio-temporal patches (Sec. 1: the method extends from 2-D patches to
 * spatio-temporal ones).  A query becomes the 8 x 8 x 3 volume over three
 * consecutive gray frames, in (dy, dx, tau) order with tau = 0 the oldest.
 * riann_stack_frames interleaves the frames into one 3-channel frame,
 *   d_out[(y*W + x)*3 + tau] = d_f<tau>[y*W + x],
 * whose (dy, dx, c) patches are exactly those volumes; passed with a
 * 3-channel index of reference volumes ([n][8][8][3], the same order) to
 * riann_annf_frame (or riann_knn_frame, or a 3-channel session), it answers
 * the spatio-temporal query step.  A video's first two frames have no full
 * volume: a caller that wants fields for them repeats the earliest frame.
 *   d_f0, d_f1, d_f2  device uint8 [H][W], oldest first
 *   d_out             device uint8 [H][W][3]; may not alias an input
 * Asynchronous on `stream`.  Errors: RIANN_ERR_INVALID_ARG for null
 * pointers, aliasing or H, W < 1.
 */
int riann_stack_frames(riann_stream_t stream, const uint8_t* d_f0, const uint8_t* d_f1, const uint8_t* d_f2,
                       int32_t H, int32_t W, uint8_t* d_out);

/*
 * Brute-force exact nearest neighbour field (the dense tensor-core path on its
 * own; Alg. 1's initialisation replaced by exact NN).  Arguments as riann_annf_frame.
 */
int riann_exact_nn(riann_index_t idx, riann_stream_t stream,
                   const uint8_t* d_frame, int32_t H, int32_t W,
                   int32_t* d_out_annf, uint32_t* d_out_dist);

/* Work counters of the most recent riann_annf_frame / riann_exact_nn call on
 * this index (the work measure of Sec. 3.3 / Fig. 5: rings and candidates
 * grow with temporal change). */
typedef struct {
  uint64_t ring_queries;     /* queries answered by ring intersection           */
  uint64_t dense_queries;    /* queries answered by brute force (incl. frame 0)  */
  uint64_t sum_seed;         /* sum over ring queries of the entries the scan visits
                                (the seed ring's runs, see riann_build_reference_index_ex) */
  uint64_t sum_candidates;   /* sum over ring queries of |S|                    */
  uint64_t sum_filtered;     /* sum over ring queries of the entries that pass the scan's
                                code test (each gathers its row of every key's codes) */
  uint64_t sum_exact;        /* sum over ring queries of the entries that pass every
                                code range (each needs the exact test and its row)  */
} riann_frame_stats_t;

/*
 * Allocation-free brute force (the paper has no counterpart: this is a
 * deployment variant of riann_exact_nn).  For callers that may not allocate
 * device memory while running -- a real-time pipeline whose memory budget is
 * fixed at start-up, or a plug-in whose host application owns all
 * allocations.  Same arguments and results as riann_exact_nn, but its scratch
 * is a 16 MiB device array compiled into the library (held on every GPU that
 * loads the library until the process exits), so it calls no allocator.
 *   - Frames with more than riann_exact_nn_noalloc_max_queries(channels)
 *     queries ((H-7)*(W-7)) are rejected with RIANN_ERR_TOO_LARGE.
 *   - The first call on a device looks up the array's device address and
 *     builds its TMA descriptors; make that first call before any stream
 *     capture.  Until that set-up has succeeded on a device, a call made
 *     while `stream` is capturing is refused with RIANN_ERR_INVALID_ARG (the
 *     next call outside a capture retries the set-up).
 *   - All calls share the array: calls that overlap on the GPU (e.g. on two
 *     streams at once) race and must be serialised by the caller.
 *   - The current device must be the index's device.
 */
int riann_exact_nn_noalloc(riann_index_t idx, riann_stream_t stream,
                           const uint8_t* d_frame, int32_t H, int32_t W,
                           int32_t* d_out_annf, uint32_t* d_out_dist);

/* Largest query count (H-7)*(W-7) riann_exact_nn_noalloc accepts for 1 or 3
 * channels (0 for other values). */
int64_t riann_exact_nn_noalloc_max_queries(int32_t channels);

/*
 * Failure-detection check of the brute-force kernel's bounded waits (the paper
 * has no counterpart).  Runs riann_exact_nn on the frame with its TMA producer
 * withholding every reference tile, so that the MMA issuer's wait for the
 * first one -- a barrier that nothing will complete -- runs out after
 * `spin_cycles` clock cycles (1000 <= spin_cycles <= 2e9; about 1 s is the
 * limit every call of the library uses).  The kernel then sets
 * RIANN_DEV_TIMEOUT in the index's status word, releases its tensor memory and
 * returns; the device context stays usable and later calls on the index are
 * unaffected.  d_out_annf receives no defined values.  Asynchronous on
 * `stream`: read the bit with riann_status.  Errors as riann_exact_nn, plus
 * RIANN_ERR_INVALID_ARG for spin_cycles out of range and RIANN_ERR_UNSUPPORTED
 * on a unit-normalised index.
 */
int riann_test_wait_expiry(riann_index_t idx, riann_stream_t stream, const uint8_t* d_frame, int32_t H, int32_t W,
                           int32_t* d_out_annf, int64_t spin_cycles);

/*
 * Measurement utility (the paper has no counterpart): the sustained rate of
 * the integer instruction pair the key-point distances use -- per 4 bytes a
 * per-byte absolute difference and a 4-way dot product of it with itself --
 * over every SM of the current device, in integer operations per second
 * (8 per pair: 4 multiplies and 4 adds).  Synchronises `stream`; allocates a
 * small buffer from the stream-ordered pool.  Errors: RIANN_ERR_INVALID_ARG
 * for a null pointer, RIANN_ERR_OOM, RIANN_ERR_CUDA.
 */
int riann_measure_int_peak(riann_stream_t stream, double* ops_per_s);

/*
 * Check of the checked build (the paper has no counterpart).  Overwrites the
 * pair-order cell offsets of key point `key` from its second cell on with
 * n + extra, so that the first run of every query seeded by that key reaches
 * `extra` entries past the end of the key's rows.  The checked library
 * (libriann_checked.so) detects the bad run before any access, sets
 * RIANN_DEV_BOUNDS and skips it; the normal library reads those entries from
 * the next key's rows (they exist because key < K - 1) and gives wrong
 * results.  The index is unusable afterwards: destroy it.  Synchronous.
 * Errors: RIANN_ERR_INVALID_ARG unless 0 <= key < K - 1 and 1 <= extra <= 64;
 * RIANN_ERR_UNSUPPORTED unless the index scans in pair order
 * (RIANN_SCAN_PAIRS, or n >= 16384).
 */
int riann_test_corrupt_offsets(riann_index_t idx, int32_t key, int32_t extra);

/* Synchronises `stream` and reads the counters. */
int riann_frame_stats(riann_index_t idx, riann_stream_t stream, riann_frame_stats_t* out);

/*
 * Per-kernel timing.  When enabled, every kernel of a frame is bracketed by
 * CUDA events recorded on the frame's stream.  riann_profile_read
 * synchronises `stream` and writes, per slot, the duration in milliseconds of
 * that kernel's most recent launch (-1 if it did not run since the last read):
 *   slot 0  ring-intersection kernel (patch, key distances, rings, verification)
 *   slot 1  brute-force kernel (frame 0 and queries routed to it)
 *   slot 2  query-row preparation of the brute-force path
 */
#define RIANN_SLOT_RING 0
#define RIANN_SLOT_DENSE 1
#define RIANN_SLOT_PREP 2
int riann_profile_enable(riann_index_t idx, int on);
int riann_profile_read(riann_index_t idx, riann_stream_t stream, float* ms, int32_t nslots);

/* ------------------------------------------------------------------------
 * Sessions: one per video stream.  A session keeps the stream's previous ANN
 * field on the device between frames (Alg. 1: r_i = ANNF^(t-1)(x, y)), double
 * buffered, plus the scratch of one frame, so sessions on different CUDA
 * streams run concurrently.  The first frame of a session (and the first
 * after riann_session_reset, e.g. at a known scene cut) is answered by brute
 * force (Alg. 1's initialisation).  Results are identical to chaining
 * riann_annf_frame calls by hand.
 * ------------------------------------------------------------------------ */
typedef struct riann_session_s* riann_session_t;

typedef struct {
  int32_t H, W;
  int64_t frames;          /* frames processed so far                    */
  int32_t has_field;       /* 1 when a previous field is held            */
  size_t device_bytes;     /* device memory the session holds            */
} riann_session_info_t;

/* Allocates the session for frames of H x W x channels(idx).  The session
 * keeps a pointer to idx, which must outlive it. */
int riann_session_create(riann_index_t idx, int32_t H, int32_t W, riann_session_t* out);
/* Synchronises the device and frees the session.  NULL is a no-op. */
void riann_session_destroy(riann_session_t s);
/* Drops the previous field: the next frame is answered by brute force. */
int riann_session_reset(riann_session_t s);
int riann_session_info(riann_session_t s, riann_session_info_t* out);
/* Device bytes a session for H x W frames holds (the admission cost: two
 * fields, distances, counts and a frame buffer; scratch excluded). */
int64_t riann_session_state_bytes(riann_index_t idx, int32_t H, int32_t W);

/* One frame from device memory.  The field, distances and counts stay in the
 * session (riann_session_outputs); the d_out_* pointers (nullable) receive
 * copies.  Asynchronous on `stream`. */
int riann_session_frame(riann_session_t s, const riann_params* p, riann_stream_t stream,
                        const uint8_t* d_frame, int32_t* d_out_annf, uint32_t* d_out_dist,
                        uint32_t* d_out_count);
/* One frame from host memory: copies h_frame [H][W][C] to the device, runs
 * the step and copies the field (and, if not NULL, distances and counts) back
 * into host buffers.  Asynchronous on `stream` when the host buffers are
 * pinned; the caller synchronises the stream before reading them. */
int riann_session_frame_host(riann_session_t s, const riann_params* p, riann_stream_t stream,
                             const uint8_t* h_frame, int32_t* h_out_annf, uint32_t* h_out_dist,
                             uint32_t* h_out_count);
/* Checkpoint: copies the latest field (int32 [H-7][W-7]) to `out` (host or
 * device); synchronous.  RIANN_ERR_INVALID_ARG when the session holds none. */
int riann_session_field(riann_session_t s, riann_stream_t stream, int32_t* out);
/* Resume: makes `field` (host or device, int32 [H-7][W-7]) the previous field
 * of the next frame; synchronous. */
int riann_session_restore(riann_session_t s, riann_stream_t stream, const int32_t* field);
/* Device pointers of the latest field, distances and counts (owned by the
 * session; valid until its next frame). */
int riann_session_outputs(riann_session_t s, int32_t** d_annf, uint32_t** d_dist, uint32_t** d_count);
/* The session's device frame buffer (H x W x C bytes), for callers that
 * upload frames themselves. */
uint8_t* riann_session_frame_buffer(riann_session_t s);
/* Copies the latest field, distances and counts (each nullable; host or
 * device destinations) on `stream`, asynchronously. */
int riann_session_copy_outputs(riann_session_t s, riann_stream_t stream, int32_t* annf, uint32_t* dist,
                               uint32_t* count);

/* ------------------------------------------------------------------------
 * Batched form: the frames of many sessions (of one index, of any sizes)
 * answered by one ring-intersection launch per frame, spread over four
 * streams forked from and joined back to the caller's, followed by one
 * brute-force pass over the union of the queries they routed.  The launch
 * sequence is captured once as a CUDA graph and replayed every call (unless
 * created with RIANN_BATCH_NO_GRAPH); frame and field pointers travel in a
 * pinned descriptor table the graph copies in, and the graph is re-captured
 * only when a slot receives a larger frame than it has held (or the
 * parameters or tuning change).  Results are identical to running each
 * session alone.
 * ------------------------------------------------------------------------ */
typedef struct riann_batch_s* riann_batch_t;
#define RIANN_BATCH_NO_GRAPH 0x1

typedef struct {
  int32_t max_items;
  int64_t max_queries;
  int32_t uses_graph;
  int64_t runs, graph_builds;
  size_t device_bytes;
} riann_batch_info_t;

/* Scratch for up to max_items frames holding max_queries queries in total
 * (< 2^31).  The context keeps a pointer to idx. */
int riann_batch_create(riann_index_t idx, int32_t max_items, int64_t max_queries, int32_t flags,
                       riann_batch_t* out);
void riann_batch_destroy(riann_batch_t b);
/* One step for n distinct sessions of the context's index; d_frames[i] is the
 * device frame of sessions[i].  Asynchronous on `stream`; waits (host side)
 * for the context's previous step before reusing its descriptor table.
 * RIANN_ERR_TOO_LARGE when the frames exceed max_queries. */
int riann_batch_run(riann_batch_t b, const riann_params* p, riann_stream_t stream,
                    riann_session_t* sessions, const uint8_t* const* d_frames, int32_t n);
/* Work counters of the context's last step (synchronises `stream`). */
int riann_batch_stats(riann_batch_t b, riann_stream_t stream, riann_frame_stats_t* out);
int riann_batch_info(riann_batch_t b, riann_batch_info_t* out);

/* ------------------------------------------------------------------------
 * Autotuner: times the ring kernel's variants (query tile 4x32 or 8x16;
 * 1 to 4 code groups tested before compaction) on a sample frame and its
 * previous field, keeps the fastest in the index, and returns every timing.
 * The variants compute identical results.
 * ------------------------------------------------------------------------ */
typedef struct {
  int32_t tile_shape;   /* 0: 4 x 32 queries per CTA, 1: 8 x 16 */
  int32_t depth;        /* 1..4 */
  float ms;             /* mean time of one frame (riann_autotune), else -1 */
} riann_tuning_t;

int riann_autotune(riann_index_t idx, const riann_params* p, riann_stream_t stream,
                   const uint8_t* d_frame, int32_t H, int32_t W, const int32_t* d_prev_annf,
                   int32_t iters, riann_tuning_t* results, int32_t max_results, int32_t* n_results);
int riann_set_tuning(riann_index_t idx, const riann_tuning_t* t);
int riann_get_tuning(riann_index_t idx, riann_tuning_t* out);

/* ------------------------------------------------------------------------
 * Served form: continuous batching of many streams of different sizes and
 * channel counts.  Streams are admitted while their resident state
 * (riann_session_state_bytes) fits `budget_bytes`, their queries fit
 * `max_tick_queries` per index and, when `load_limit` > 0, the GPU time they
 * claim fits: every open stream with a declared frame rate claims
 * fps * (H-7) * (W-7) * t_q GPU seconds per second, t_q being the GPU time
 * per query measured on its index (CUDA events around each index's part of
 * every tick, exponentially averaged), and the claims may sum to at most
 * `load_limit` (e.g. 0.85).  Until an index has a measurement only one
 * rate-declaring stream of it is admitted.  Otherwise riann_server_open
 * returns RIANN_ERR_ADMISSION (the caller may retry later).  A
 * submitted frame is copied into one of the stream's two pinned input slots;
 * a newer frame replaces one not yet dispatched (counted as dropped).
 * riann_server_step completes the tick in flight (blocking only if `wait`)
 * and launches the next over every stream with a pending frame: copies in,
 * one batched step per index, fields copied back to pinned host memory.
 * Frames arriving while a tick runs join the next tick.  Results equal those
 * of each stream run alone.  All times are riann_server_clock() seconds.
 * ------------------------------------------------------------------------ */
typedef struct riann_server_s* riann_server_t;

typedef struct {
  int32_t stream_id;
  int64_t frame_id;
  double t_arrival;   /* as given to riann_server_submit            */
  double t_done;      /* when the host saw the frame's tick complete */
} riann_server_result_t;

typedef struct {
  int32_t open_streams;
  size_t budget_bytes, used_bytes;
  int64_t ticks, frames_done, queries_done, rejected, submitted, dropped;
  double load;              /* GPU seconds per second claimed by the open streams */
  double ns_per_query[2];   /* measured GPU time per query, [0] gray, [1] RGB; 0: none yet */
} riann_server_info_t;

#define RIANN_SERVER_PLAIN 0x1   /* run each frame of a tick by itself (comparison mode) */

double riann_server_clock(void);
/* gray / rgb: indexes for 1- and 3-channel streams (either may be NULL).
 * The server keeps pointers to them; they must outlive it.  load_limit <= 0:
 * no rate admission. */
int riann_server_create(riann_index_t gray, riann_index_t rgb, size_t budget_bytes, int64_t max_tick_queries,
                        int32_t max_streams, const riann_params* p, int32_t flags, double load_limit,
                        riann_server_t* out);
void riann_server_destroy(riann_server_t s);
/* fps: the stream's declared frame rate (<= 0: claims no GPU time). */
int riann_server_open(riann_server_t s, int32_t H, int32_t W, int32_t C, double fps, int32_t* stream_id);
int riann_server_close(riann_server_t s, int32_t stream_id);
/* h_frame: host uint8 [H][W][C]; copied before the call returns. */
int riann_server_submit(riann_server_t s, int32_t stream_id, const uint8_t* h_frame, int64_t frame_id,
                        double t_arrival);
/* *launched = number of frames in the newly launched tick (0: none, or the
 * previous tick is still running and wait == 0). */
int riann_server_step(riann_server_t s, riann_stream_t stream, int32_t wait, int32_t* launched);
/* Pops up to `max` completed frames. */
int riann_server_poll(riann_server_t s, riann_server_result_t* out, int32_t max, int32_t* n);
/* Latest completed field of a stream (int32 [H-7][W-7] host copy); valid
 * while the stream has no frame in flight. */
int riann_server_field(riann_server_t s, int32_t stream_id, int32_t* out);
int riann_server_info(riann_server_t s, riann_server_info_t* out);
int riann_server_stream_counts(riann_server_t s, int32_t stream_id, int64_t* submitted, int64_t* dropped,
                               int64_t* completed);

/* ------------------------------------------------------------------------
 * Reconstruction (Sec. 4: the video is rebuilt by replacing every patch with
 * its match and averaging where patches overlap; error
 * E = ||f_GT - f_R||_2 / ||f_GT||_2).
 *
 * d_annf: device int32 [H-7][W-7], a field over this index (entries outside
 *   [0, n) set RIANN_DEV_BAD_PREV and contribute nothing).
 * d_out (nullable): device uint8 [H][W][C], f_R: every pixel the average of the
 *   matched reference pixels of all query patches covering it, rounded half up
 *   to 8 bits, (2 * sum + count) / (2 * count) in integers.
 * d_frame (nullable): device uint8 [H][W][C], f_GT; with d_err2 it gives the
 *   error sums.
 * d_err2 (nullable, needs d_frame): device uint64 [2], written with
 *   sum (f_GT - f_R)^2 and sum f_GT^2 over all bytes, so that
 *   E = sqrt(err2[0] / err2[1]).
 * Asynchronous on `stream`; the caller owns every buffer.
 * ------------------------------------------------------------------------ */
int riann_reconstruct(riann_index_t idx, riann_stream_t stream, const int32_t* d_annf, int32_t H, int32_t W,
                      const uint8_t* d_frame, uint8_t* d_out, unsigned long long* d_err2);

/*
 * Effects by patch replacement (Sec. 5: an image operation such as
 * denoising, colouring or an artistic style is run once, offline, on the
 * reference patches; online, every query patch takes the processed copy of
 * the reference it matched and overlapping patches are averaged).  The same
 * reconstruction as riann_reconstruct, with the matched rows read from a
 * caller-supplied table instead of the index's references:
 *   d_payload  device uint8 [n][8][8][channels], row r = T(reference r)
 *              (n of this index), 16-byte aligned; owned by the caller and
 *              read during the call's kernel only
 *   channels   1 or 3, independent of the index's channel count (a gray
 *              index with an RGB payload colours a gray video)
 *   d_out, d_frame  uint8 [H][W][channels]; d_annf, d_err2 as
 *              riann_reconstruct (d_frame is then the target f_GT of the
 *              effect, e.g. the clean or coloured frame)
 * RIANN_ERR_INVALID_ARG for a null table, channels other than 1 or 3, a
 * table address that is not 16-byte aligned, or the riann_reconstruct cases.
 */
int riann_reconstruct_payload(riann_index_t idx, riann_stream_t stream, const uint8_t* d_payload, int32_t channels,
                              const int32_t* d_annf, int32_t H, int32_t W, const uint8_t* d_frame, uint8_t* d_out,
                              unsigned long long* d_err2);

/* ------------------------------------------------------------------------
 * Alg. 1 with random anchors, as the paper runs it (Sec. 3.2, 3.3, Alg. 1):
 * the candidate set starts as the ring around the previous match r_i
 * (radius d_i = dist(q, r_i), half-width alpha * d_i) and, while it holds L or
 * more references, is intersected with the ring around an anchor drawn at
 * random from it (radius and half-width from that anchor's distance to q);
 * the answer is the closest of the final candidates, r_i and the anchors.
 *
 * The rings come from the sorted distance matrix of Sec. 3.4 (every
 * reference's distances to all others, ascending): n^2 8-byte entries, built
 * once by riann_full_create (34 GB for n = 65536).  Ring test, in integers,
 * for anchor a and candidate r (alpha = p/q, B = ||q - a||^2):
 *   (q - p)^2 B <= q^2 ||a - r||^2 (when p < q)  and  q^2 ||a - r||^2 <= (q + p)^2 B.
 * The candidate set keeps the order of row r_i; the anchor of ring t is the
 * candidate at position (x * |S|) >> 32, x the first output word of
 * Philox4x32-10 with counter (query index, t, frame_id, 0) and key
 * (seed low 32 bits, seed high 32 bits).  Ties: lower reference index.
 * ------------------------------------------------------------------------ */
typedef struct riann_full_s* riann_full_t;

typedef struct {
  int32_t alpha_num, alpha_den;   /* ring half-width alpha = num/den (den 1..8, num 0..8*den) */
  int32_t L;                      /* stop below L candidates (the paper: 20); >= 1 */
  int32_t max_rings;              /* at most this many anchors per query (0..4096) */
  uint64_t seed;                  /* Philox key */
  uint32_t frame_id;              /* Philox counter word: distinct per frame */
} riann_anchor_params;

/* alpha = 1/4, L = 20, max_rings = 64, seed = 0, frame_id = 0. */
riann_anchor_params riann_default_anchor_params(void);

/* Builds the sorted distance matrix of the index's references (the index
 * must outlive the handle).  RIANN_ERR_OOM when it does not fit. */
int riann_full_create(riann_index_t idx, riann_stream_t stream, riann_full_t* out);
void riann_full_destroy(riann_full_t f);
/* Row-major copy of the matrix to host memory: n * n keys
 * (||r_i - r_id||^2 << 32) | id; synchronous. */
int riann_full_table(riann_full_t f, riann_stream_t stream, uint64_t* host_T);

/* One frame.  d_prev == NULL: brute force (count = n, rings = 0).  Outputs as
 * riann_annf_frame plus d_out_rings (nullable): anchors drawn per query.
 * Calls on one handle must not overlap on the GPU (they share its scratch). */
int riann_anchor_frame(riann_full_t f, const riann_anchor_params* p, riann_stream_t stream,
                       const uint8_t* d_frame, int32_t H, int32_t W, const int32_t* d_prev,
                       int32_t* d_out_annf, uint32_t* d_out_dist, uint32_t* d_out_count,
                       uint32_t* d_out_rings);

/* Alg. 1's random initial field (each entry uniform over the references;
 * 0-based here): writes the
 * int32 [H-7][W-7] field d_out_annf, entry q = (x * n) >> 32 with x the first
 * word of Philox4x32-10 at counter (q, 0, frame_id, 1), key (seed low, seed
 * high).  Asynchronous on `stream`. */
int riann_random_field(riann_stream_t stream, int32_t H, int32_t W, int32_t n, uint64_t seed, uint32_t frame_id,
                       int32_t* d_out_annf);

/* Work of the handle's last riann_anchor_frame (synchronises `stream`):
 * out3[0] = sum of |S_0| (first-ring sizes), out3[1] = candidate tests made by
 * the anchor rings, out3[2] = sum of the final |S|. */
int riann_anchor_work(riann_full_t f, riann_stream_t stream, uint64_t* out3);

/* Synchronises `stream`, then returns RIANN_OK if the device status word is
 * clear, RIANN_ERR_DEVICE otherwise (and clears it); *bits (nullable) receives
 * the word. */
int riann_status(riann_index_t idx, riann_stream_t stream, uint32_t* bits);

const char* riann_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* RIANN_H */
