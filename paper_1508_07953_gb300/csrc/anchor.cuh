// anchor.cuh -- Alg. 1 with random anchors over the Sec. 3.4 sorted distance
// matrix (declarations).
#pragma once

#include "common.cuh"

namespace riann {

constexpr int kAnchorWarps = 4;      // warps per CTA of the persistent anchor launch
constexpr int kAnchorCtasPerSm = 4;
constexpr int kAnchorBitmapN = 65536;   // references a warp's membership bitmap covers (8 KB)

struct AnchorArgs {
  const uint8_t* frame;
  int32_t H, W;
  const int32_t* prev;
  int32_t* out_annf;
  uint32_t* out_dist;             // nullable
  uint32_t* out_count;            // nullable
  uint32_t* out_rings;            // nullable
  const uint8_t* R;
  int n, NP;                      // references; row stride of T (n rounded up to a power of two >= 2048)
  const unsigned long long* T;    // [n][NP] (||r_i - r_id||^2 << 32) | id, rows ascending
  int alpha_num, alpha_den, L, max_rings;
  uint32_t key0, key1, frame_id;  // Philox4x32-10 key and the frame word of the counter
  int32_t* scratch;               // [resident warps][2][n] candidate lists
  uint32_t* counter;              // next query (zeroed before the launch)
  unsigned long long* work;       // [3] sum |S_0|, candidate tests of the anchor rings, final |S| (zeroed)
  uint32_t* status;
};

// Row stride of the sorted matrix for n references.
int full_table_stride(int n);
// T[i][j] for all i < n: keys of row i, then each row sorted ascending.
cudaError_t build_full_table(const Index& ix, unsigned long long* T, int NP, cudaStream_t s);
// Resident warps of the persistent launch (the scratch holds 2 n ids for each).
int anchor_resident_warps();
cudaError_t launch_anchor(const AnchorArgs& a, int C, cudaStream_t s);
cudaError_t launch_fill_u32(uint32_t* p, int64_t count, uint32_t value, cudaStream_t s);
cudaError_t launch_random_field(int64_t Q, int n, uint64_t seed, uint32_t frame_id, int32_t* out, cudaStream_t s);

// index_build.cu
cudaError_t sort_segments(unsigned long long* keys, int NP, int64_t nseg, cudaStream_t s);
int sort_chunk();

}  // namespace riann
