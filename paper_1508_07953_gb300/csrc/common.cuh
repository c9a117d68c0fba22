// common.cuh -- internal declarations of the RIANN CUDA library (sm_103a).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <mutex>

#include "../../include/riann.h"

namespace riann {

constexpr int kPatch = 8;
constexpr int kMaxK = 64;
constexpr int kMaxDim = 192;
constexpr int kDenseTileN = 256;   // reference rows per tensor-core tile
constexpr int kDenseTileM = 128;   // query rows per tensor-core tile
constexpr int kBuckets = 256;      // quantile buckets per key point (8-bit codes)
constexpr int kPairCodes = 128;    // filter codes per key point (7-bit: code >> 1)
// Smallest reference set whose keys scan in pair order with a second key:
// below it a 7-bit bucket holds too few references for the partner's runs to
// pay for their fragmentation, and each key pairs with itself (measured: pair
// order 12-16 % faster at n = 16384, 24 % slower at n = 4096).
constexpr int kPairMinN = 16384;
constexpr int kKnnMax = 8;         // largest k of the k-NN output
static_assert(kKnnMax == RIANN_KNN_MAX, "k-NN list length");

// Work counters of the last frame or batch (riann_frame_stats).
enum StatSlot { kStatRingQueries = 0, kStatDenseQueries, kStatSumSeed, kStatSumS, kStatSumFiltered, kStatSumExact,
                kStats = 8 };

// Kernel slots of the per-kernel event profiler (riann_profile_*).
enum KernelSlot { kSlotSparse = 0, kSlotDense = 1, kSlotPrep = 2, kSlots = 4 };

// Ring-kernel variants the autotuner chooses between: query tile shape, and
// the number of code groups (1..kMaxScanDepth) the scan tests per chunk.
constexpr int kMaxScanDepth = 4;
enum TileShape { kTile4x32 = 0, kTile8x16 = 1, kTileShapes = 2 };

// Checked build (compiled with -DRIANN_CHECKED into libriann_checked.so):
// every index a kernel gathers from a table is tested against the table's
// extent before the access; a failed test sets RIANN_DEV_BOUNDS in the
// status word and the access is skipped.  In the normal build the test is
// compiled out (the tables are built by the library, so the indices are in
// range by construction).
#if defined(RIANN_CHECKED)
__device__ __forceinline__ bool checked_ok(bool ok, uint32_t* status) {
  if (!ok) atomicOr(status, RIANN_DEV_BOUNDS);
  return ok;
}
#define RIANN_IN_RANGE(cond, status) ::riann::checked_ok((cond), (status))
#else
#define RIANN_IN_RANGE(cond, status) true
#endif

// Largest possible squared distance between two patches of `dim` bytes.
__host__ __device__ constexpr uint32_t max_sqdist(int dim) { return (uint32_t)dim * 255u * 255u; }

// One frame of a launch: its pixels, its previous field (nullptr: every query
// is answered by brute force, Alg. 1's initialisation step), its outputs, and its place
// in the launch's tile and query numbering (a single-frame launch has one item
// with both offsets 0).  Global query id = query_begin + y * Wq + x.
struct FrameItem {
  const uint8_t* frame;
  const int32_t* prev;
  int32_t* out_annf;
  uint32_t* out_dist;     // nullable
  uint32_t* out_count;    // nullable
  int32_t H, W, Hq, Wq;
  int32_t tiles_x;        // ring-kernel tiles per row of queries
  int64_t query_begin;    // first global query id of this item
};

// Device header of a batched launch.
struct BatchHeader {
  int32_t n_items;
  int64_t total_queries;
};

// Scratch of one launch in flight (one frame or one batch).
struct Workspace {
  int64_t cap_q = 0;                    // queries it can hold
  int32_t* dense_list = nullptr;        // [cap_q] global query ids routed to brute force
  uint32_t* counters = nullptr;         // [4]: 0 brute-force list length
  unsigned long long* best = nullptr;   // [cap_q] packed (dist << 32 | index)
  __nv_bfloat16* Aq = nullptr;          // [cap_q padded to 128][D] bf16 query rows
  uint32_t* qnorm = nullptr;            // [cap_q padded] ||q||^2
  CUtensorMap tmAq;                     // Aq rows, box 64 x 128
  unsigned long long* knn_lists = nullptr;   // k-NN brute force: per-work-item best-8 lists
  int64_t knn_cap = 0;                  // entries of knn_lists
  size_t bytes = 0;
};

// Reference-tile split of the brute-force launch: with fewer than two query
// tiles per CTA, each query tile's reference tiles are shared among nsplit
// work items.  With balance (the argmin form), more query tiles are split too
// when that evens out the last wave: the split s of 1..4 with the fewest
// whole-tile passes per CTA, ceil(n_qt s / grid) / s, is taken if it saves
// more than 2 %.  (The k-NN form keeps one list per item and does not.)
__host__ __device__ inline int dense_nsplit(int64_t n_qt, int grid, int n_rt, bool balance = false) {
  int nsplit = 1;
  if (n_qt > 0 && n_qt < 2 * (int64_t)grid) {
    nsplit = (int)((2 * (int64_t)grid + n_qt - 1) / n_qt);
  } else if (balance && n_qt > 0) {
    double best = (double)((n_qt + grid - 1) / grid);
    for (int sp = 2; sp <= 4; ++sp) {
      const double w = (double)((n_qt * sp + grid - 1) / grid) / sp;
      if (w < 0.98 * best) {
        best = w;
        nsplit = sp;
      }
    }
  }
  if (nsplit > n_rt) nsplit = n_rt;
  return nsplit;
}

// Device-resident index (Sec. 3.3 pre-processing restricted to K key points).
struct Index {
  int device = 0;
  int n = 0, K = 0, C = 0, D = 0;
  int Kp = 0;                     // K rounded up to 4 (row stride of P)
  int n_pad = 0;                  // n rounded up to kDenseTileN
  uint8_t* R = nullptr;           // [n][D] reference patches
  uint8_t* KP = nullptr;          // [K][D] key points
  // Brute-force operands (exact in bf16 / fp32).  Gray: Rbf = -2r and RN =
  // ||r||^2 = h 2^16 + m 2^8 + l as the three terms (h 2^16, m 2^8, l) in
  // columns 0..2 of [n_pad][16] (pad rows 2^24), in the tensor core's
  // no-swizzle K-major order (per 8-row group 256 B: the 8 x 16-byte core
  // matrix of columns 0..7, then that of columns 8..15).  RGB: Rbf = r and
  // rnorm = ||r||^2 (pad rows +inf).  Pad rows of Rbf are zero.
  __nv_bfloat16* Rbf = nullptr;   // [n_pad][D]
  __nv_bfloat16* RN = nullptr;    // [n_pad][16] (gray)
  float* rnorm = nullptr;         // [n_pad] (RGB)
  uint32_t* P = nullptr;          // [n][Kp] ||k_m - r||^2 (rows padded to Kp = K rounded up to 4; pad 0)
  uint32_t* TA = nullptr;         // [K][n] per key: distances ascending
  int32_t* Tid = nullptr;         // [K][n] per key: reference index of each TA entry
  // 8-bit bucket codes: code_m(A) = max{b : E[m][b] <= A}, edges at every
  // ceil(n/256)-th rank of TA[m]; monotone in A, so a whole bucket strictly
  // inside a ring's code range lies inside the ring.
  uint32_t* E = nullptr;          // [K][kBuckets] bucket edges (UINT32_MAX past the end)
  uint32_t* RB = nullptr;         // [K][kBuckets + 1] first rank of each bucket in TA[m]; RB[m][256] = n
  // Pair order of key m: the references sorted by the cell (code7_m, code7_p)
  // of m and its partner p = partner[m] (code7 = code >> 1), then in the order
  // of key m's sorted list (TA, Tid), so that the references of one seed bucket
  // whose partner code lies in a range are contiguous.  A key paired with
  // itself (n < kPairMinN) keeps exactly its sorted list's order.
  bool pair_scan = false;         // partners are the farthest key points (else every key pairs with itself)
  int32_t* partner = nullptr;     // [K] scan partner of each key (the farthest key point, or itself)
  int32_t* Tid2 = nullptr;        // [K][n] reference id at each position of the pair order
  uint32_t* OFF = nullptr;        // [K][kPairCodes^2 + 1] first position of each cell (cell = cm * 128 + cp)
  uint32_t* CW = nullptr;         // [K][G][nw] in key m's pair order, filter codes of keys 4g..4g+3 (one
                                  // byte each: 0x80 | (code >> 1)); rows padded to nw = n rounded up to 4
                                  // (16-byte aligned rows)
  uint8_t* CE = nullptr;          // [K][n][Ke] in key m's pair order, the filter codes of every key of an
                                  // entry (the bytes of CW), rows of Ke = K rounded up to 16 bytes (pad 0x80)
  int Ke = 0;
  int G = 0;                      // ceil(K / 4) = Kp / 4
  int nw = 0;                     // n rounded up to 4
  uint32_t* status = nullptr;     // device status word (RIANN_DEV_* bits)
  unsigned long long* stats = nullptr;  // [kStats] counters of the last frame
  size_t device_bytes = 0;
  // unit-normalised float variant: patches scaled to length 1 (fp32, fixed
  // operation order); P, TA, E hold the bit patterns of the float distances
  bool unit = false;
  float* Rf = nullptr;            // [n][D] normalised references
  float* KPf = nullptr;           // [K][D] normalised key points

  // ring-kernel tuning (riann_autotune sets them; these are the defaults)
  int tile_shape = kTile4x32;
  int depth = 3;                  // scan depth (code groups tested before compaction, 1..kMaxScanDepth);
                                  // set at build: 4 for 16 or more groups, else 3

  // optional per-kernel timing with CUDA events recorded on the launch stream
  bool profile = false;
  bool prof_recorded[kSlots] = {};
  cudaEvent_t prof_ev[kSlots][2] = {};

  std::mutex mu;                  // guards ws and the profiler
  Workspace ws;                   // scratch of riann_annf_frame / riann_exact_nn

  // TMA descriptor of the brute-force B operand
  CUtensorMap tmRbf;              // Rbf rows, box 64 x (reference rows per tile)
  bool tm_ready = false;
};

// Arguments of the fused ring-intersection kernel (a1-a4).
struct SparseArgs {
  FrameItem one;                  // the frame of a single-frame launch
  const FrameItem* items;         // batched launch: device item array
  const BatchHeader* hdr;         // batched launch: device header
  int item;                       // batched launch: the entry of `items` this launch covers
  const uint8_t* R;
  const uint8_t* KP;
  const uint32_t* P;
  const uint32_t* TA;
  const int32_t* Tid;
  const uint32_t* E;
  const uint32_t* RB;
  const int32_t* partner;
  const int32_t* Tid2;
  const uint32_t* OFF;
  const uint32_t* CW;
  const uint8_t* CE;
  int n, K, Kp, G, nw, Ke;
  int alpha_num, alpha_den, ring_limit;
  int depth;                      // scan depth (1..kMaxScanDepth)
  int unit;                       // unit-normalised float variant (Rf, KPf below)
  const float* Rf;
  const float* KPf;
  int knn;                        // k of the k-NN variant (0: 1-NN path)
  int32_t* knn_idx;               // k-NN variant: [Q][knn] matches, ascending (dist, index); -1 past |S u {r_p}|
  uint32_t* knn_dist;             // k-NN variant: [Q][knn] their squared distances (nullable; ~0 past the end)
  int32_t* dense_list;
  uint32_t* counters;             // [0] brute-force list length
  uint32_t* status;
  unsigned long long* stats;      // nullable
};

// Arguments of the brute-force path (a5).
struct DenseArgs {
  FrameItem one;                  // single frame (items == nullptr)
  const FrameItem* items;         // batched launch: device item array
  const BatchHeader* hdr;
  int64_t Q;                      // queries of the single frame, or the list capacity
  const int32_t* list;            // nullptr: every query of `one` in order
  const uint32_t* list_count;     // device count of `list`
  const uint8_t* R;
  int n;
  unsigned long long* stats;      // nullable; a whole-frame launch records Q brute-force queries
  int knn;                        // k of the k-NN output (0: argmin only); single frame only
  int32_t* knn_idx;               // [Q][knn]
  uint32_t* knn_dist;             // [Q][knn], nullable
  long long spin_limit;           // bound of the kernel's waits in clock cycles (0: the default, about 1 s)
  int withhold;                   // test hook (riann_test_wait_expiry): no reference tile is loaded
};

// Record the start/end event of a profiled kernel slot (no-op when profiling is off).
void prof_begin(Index& ix, int slot, cudaStream_t s);
void prof_end(Index& ix, int slot, cudaStream_t s);

// 2-D SWIZZLE_128B tensor map over bf16 rows of D elements.
bool make_row_map(CUtensorMap* m, const void* base, uint64_t rows, int D, int box_rows);
int dense_ref_rows_per_tile(int C);
cudaError_t launch_dense_tc(const DenseArgs& a, Index& ix, Workspace& ws, cudaStream_t s);
// entries of Workspace::knn_lists a k-NN brute-force launch over up to Q queries needs
int64_t dense_knn_list_entries(int64_t Q);
int64_t noalloc_max_queries(int C);
cudaError_t launch_exact_nn_noalloc(const DenseArgs& a, Index& ix, cudaStream_t s);

// ring kernel: one frame (grid = its tiles), its descriptor in the launch
// parameters or (batched form) in a device array
int ring_tile_rows(int shape);
int ring_tile_cols(int shape);
// per-device launch set-up of the ring kernels for C channels (outside any capture)
cudaError_t ring_prepare(int C);
cudaError_t launch_sparse(const SparseArgs& a, int C, int shape, cudaStream_t s);
cudaError_t launch_sparse_item(const SparseArgs& a, int C, int shape, int tiles, cudaStream_t s);

cudaError_t launch_index_build(Index& ix, cudaStream_t s);

// unit.cu: unit-normalised float variant -- normalised tables and P (as
// float bits) for an index with ix.unit set, and its brute force
cudaError_t launch_unit_tables(Index& ix, cudaStream_t s);
cudaError_t launch_dense_unit(const DenseArgs& d, Index& ix, cudaStream_t s);

// cluster.cu: Sec. 3.4 reference-set construction (synchronises `s`)
cudaError_t cluster_references(const uint8_t* X, int n, int C, int leaf, uint8_t* reps, int32_t* assign,
                               int32_t* out_count, cudaStream_t s);

// stack.cu: out[p][tau] = f_tau[p] for the npix pixels of three gray frames
cudaError_t launch_stack3(const uint8_t* f0, const uint8_t* f1, const uint8_t* f2, int64_t npix, uint8_t* out,
                          cudaStream_t s);

// Workspace management (allocation synchronises the device).
int ensure_workspace(Workspace& ws, const Index& ix, int64_t Q);
int ensure_knn_lists(Workspace& ws, int64_t Q);
void free_workspace(Workspace& ws);

int sm_count();

}  // namespace riann
