// index_build.cu -- pre-processing of the reference set (Sec. 3.3: distances
// from the anchors to every reference, sorted ascending per anchor; here the
// anchors are the K fixed key points).  Runs once per reference set.
#include "common.cuh"

namespace riann {
namespace {

// P[r][m] = ||k_m - R_r||^2 (row stride Kp, pad entries 0).  One thread per
// (r, m); words compared with per-byte absolute differences and a 4-way dot
// product of them with themselves.
__global__ void k_key_distances(const uint8_t* __restrict__ R, const uint8_t* __restrict__ KP,
                                int n, int K, int Kp, int D, uint32_t* __restrict__ P) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * Kp) return;
  int r = (int)(t / Kp), m = (int)(t % Kp);
  if (m >= K) {
    P[t] = 0;
    return;
  }
  const uint32_t* a = reinterpret_cast<const uint32_t*>(R + (int64_t)r * D);
  const uint32_t* b = reinterpret_cast<const uint32_t*>(KP + (int64_t)m * D);
  uint32_t s = 0;
  for (int w = 0; w < D / 4; ++w) {
    uint32_t d = __vabsdiffu4(a[w], b[w]);
    s = __dp4a(d, d, s);
  }
  P[t] = s;
}

// Brute-force operands (layouts in common.cuh).  Gray (D = 64): Rbf = -2r
// (even integers -510..0, exact in bf16) and RN = ||r||^2 split into three
// terms exact in bf16 (h 2^16 with h <= 63, m 2^8 and l with m, l <= 255), so
// one extra K = 16 MMA against a ones row adds ||r||^2 to -2 q.r in the fp32
// accumulator.  RGB: Rbf = r and rnorm = ||r||^2 (exact in fp32: < 2^24).
// Rows n..n_pad-1: zero vector, norm term 2^24 (gray) or +inf (RGB), above
// every real score.
__global__ void k_prep_refs(const uint8_t* __restrict__ R, int n, int n_pad, int D,
                            __nv_bfloat16* __restrict__ Rbf, __nv_bfloat16* __restrict__ RN,
                            float* __restrict__ rnorm) {
  int r = blockIdx.x;
  if (r >= n_pad) return;
  const bool fold = D == 64;
  uint32_t s = 0;
  for (int i = threadIdx.x; i < D; i += blockDim.x) {
    uint32_t v = r < n ? R[(int64_t)r * D + i] : 0u;
    Rbf[(int64_t)r * D + i] = __float2bfloat16_rn(fold ? -2.f * (float)v : (float)v);
    s += v * v;
  }
  __shared__ uint32_t red[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 16) {
    uint32_t tot = 0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) tot += red[w];
    const int k = threadIdx.x;
    float t = 0.f;
    if (r >= n) t = k == 0 ? 16777216.f : 0.f;
    else if (k == 0) t = (float)((tot >> 16) << 16);
    else if (k == 1) t = (float)(((tot >> 8) & 255u) << 8);
    else if (k == 2) t = (float)(tot & 255u);
    // core-matrix order: group r / 8 (256 B), column half k / 8 (128 B), row r % 8 (16 B)
    RN[(int64_t)(r >> 3) * 128 + (k >> 3) * 64 + (r & 7) * 8 + (k & 7)] = __float2bfloat16_rn(t);
    if (k == 0) rnorm[r] = r < n ? (float)tot : __int_as_float(0x7f800000);
  }
}

// keys[m][j] = (P[j][m] << 32) | j for j < n, all-ones padding up to NP.
__global__ void k_make_keys(const uint32_t* __restrict__ P, int n, int Kp, int NP,
                            unsigned long long* __restrict__ keys) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int m = blockIdx.y;
  if (j >= NP) return;
  keys[(int64_t)m * NP + j] =
      j < n ? (((unsigned long long)P[(int64_t)j * Kp + m]) << 32) | (unsigned)j : ~0ull;
}

constexpr int kChunk = 2048;   // elements sorted in shared memory by one block

__device__ __forceinline__ void cmp_swap(unsigned long long& a, unsigned long long& b, bool up) {
  if ((a > b) == up) {
    unsigned long long t = a;
    a = b;
    b = t;
  }
}

// Bitonic sort of each kChunk-aligned chunk for stages k <= kChunk, or (merge
// mode) the j < kChunk steps of stage k.  Direction follows the global index so
// the chunks compose into the full network.  1024 threads, 2 elements each.
__global__ void k_bitonic_shared(unsigned long long* keys, int NP, int k_only) {
  __shared__ unsigned long long s[kChunk];
  unsigned long long* seg = keys + (int64_t)blockIdx.y * NP;
  const int base = blockIdx.x * kChunk;
  for (int i = threadIdx.x; i < kChunk; i += blockDim.x) s[i] = seg[base + i];
  __syncthreads();
  const int k_lo = k_only ? k_only : 2;
  const int k_hi = k_only ? k_only : kChunk;
  for (int k = k_lo; k <= k_hi; k <<= 1) {
    for (int j = (k_only ? kChunk : k) >> 1; j > 0; j >>= 1) {
      int t = threadIdx.x;                        // pair index
      int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
      bool up = ((base + i) & k) == 0;
      cmp_swap(s[i], s[i + j], up);
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < kChunk; i += blockDim.x) seg[base + i] = s[i];
}

// One global step (k, j) with j >= kChunk: thread per compared pair.
__global__ void k_bitonic_global(unsigned long long* keys, int NP, int k, int j) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NP / 2) return;
  unsigned long long* seg = keys + (int64_t)blockIdx.y * NP;
  int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
  bool up = (i & k) == 0;
  unsigned long long a = seg[i], b = seg[i + j];
  if ((a > b) == up) {
    seg[i] = b;
    seg[i + j] = a;
  }
}

__global__ void k_split_keys(const unsigned long long* __restrict__ keys, int n, int NP,
                             uint32_t* __restrict__ TA, int32_t* __restrict__ Tid) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  int m = blockIdx.y;
  if (j >= n) return;
  unsigned long long v = keys[(int64_t)m * NP + j];
  TA[(int64_t)m * n + j] = (uint32_t)(v >> 32);
  Tid[(int64_t)m * n + j] = (int32_t)(v & 0xffffffffu);
}

// Bucket edges and the first rank of each bucket, per key point.
__global__ void k_bucket_edges(const uint32_t* __restrict__ TA, int n, int K, uint32_t* __restrict__ E,
                               uint32_t* __restrict__ RB) {
  const int m = blockIdx.x, b = threadIdx.x;   // blockDim = kBuckets
  const int bs = (n + kBuckets - 1) / kBuckets;
  const uint32_t* t = TA + (int64_t)m * n;
  const int64_t rank = (int64_t)b * bs;
  const uint32_t e = rank < n ? t[rank] : 0xffffffffu;
  E[m * kBuckets + b] = e;
  int lo = 0, len = n;                         // first rank with t[j] >= e
  while (len > 0) {
    const int half = len >> 1;
    if (t[lo + half] < e) { lo += half + 1; len -= half + 1; } else { len = half; }
  }
  RB[m * (kBuckets + 1) + b] = (uint32_t)lo;
  if (b == 0) RB[m * (kBuckets + 1) + kBuckets] = (uint32_t)n;
}

// code[r][m] = number of edges of key m that are <= P[r][m], minus one.
__global__ void k_codes(const uint32_t* __restrict__ P, const uint32_t* __restrict__ E, int n, int K, int Kp,
                        uint8_t* __restrict__ code) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * K) return;
  const int m = (int)(t % K);
  const uint32_t a = P[(t / K) * Kp + m];
  const uint32_t* e = E + m * kBuckets;
  int lo = 0, len = kBuckets;                  // first edge > a
  while (len > 0) {
    const int half = len >> 1;
    if (e[lo + half] <= a) { lo += half + 1; len -= half + 1; } else { len = half; }
  }
  code[t] = (uint8_t)(lo - 1);                 // lo >= 1: e[0] is the smallest distance
}

// CW[m][g][j]: the filter codes of keys 4g..4g+3 of reference Tid[m][j], one
// byte each (byte i = key 4g+i): 0x80 | (code >> 1), the 7-bit code of 128
// buckets (every other edge of E) with bit 7 set, so that the ring kernel
// tests four keys with two subtractions and no borrow between bytes.  Keys
// past K read as 0x80 (code 0).
__global__ void k_pack_codes(const int32_t* __restrict__ Tid, const uint8_t* __restrict__ code, int n, int K,
                             int G, int nw, uint32_t* __restrict__ CW) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (j >= n) return;
  const int r = Tid[(int64_t)m * n + j];
  const uint8_t* c = code + (int64_t)r * K;
  for (int g = 0; g < G; ++g) {
    uint32_t w = 0;
    for (int i = 0; i < 4; ++i) {
      const int k = 4 * g + i;
      w |= (0x80u | (k < K ? (uint32_t)(c[k] >> 1) : 0u)) << (8 * i);
    }
    CW[((int64_t)m * G + g) * nw + j] = w;
  }
}

// CE[m][j][k]: the filter code of key k of reference Tid[m][j] (the same byte
// as in CW), every key of an entry in one row of Ke bytes (K rounded up to 16,
// padding bytes 0x80), so that one 16-byte load per lane reads 16 keys of a
// gathered entry.
__global__ void k_pack_entry_codes(const int32_t* __restrict__ Tid, const uint8_t* __restrict__ code, int n,
                                   int K, int Ke, uint8_t* __restrict__ CE) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;   // (j, k) of key blockIdx.y's rows
  const int m = blockIdx.y;
  if (t >= (int64_t)n * Ke) return;
  const int j = (int)(t / Ke), k = (int)(t % Ke);
  const int r = Tid[(int64_t)m * n + j];
  CE[((int64_t)m * n + j) * Ke + k] = (uint8_t)(0x80u | (k < K ? (uint32_t)(code[(int64_t)r * K + k] >> 1) : 0u));
}

// Scan partner of each key point (performance only): the key point farthest
// from it (largest ||k_m - k_p||^2, lowest index on ties), or the key itself
// (self = 1, and always when K = 1), whose pair order is then its sorted list.
__global__ void k_partners(const uint8_t* __restrict__ KP, int K, int D, int self, int32_t* __restrict__ partner) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= K) return;
  if (self) {
    partner[m] = m;
    return;
  }
  const uint32_t* a = reinterpret_cast<const uint32_t*>(KP + (int64_t)m * D);
  uint32_t best = 0;
  int bp = m;
  for (int p = 0; p < K; ++p) {
    if (p == m) continue;
    const uint32_t* b = reinterpret_cast<const uint32_t*>(KP + (int64_t)p * D);
    uint32_t s = 0;
    for (int w = 0; w < D / 4; ++w) {
      const uint32_t d = __vabsdiffu4(a[w], b[w]);
      s = __dp4a(d, d, s);
    }
    if (s > best || (s == best && bp == m)) {
      best = s;
      bp = p;
    }
  }
  partner[m] = bp;
}

// keys[m][t] = (cell << 32) | t for the reference r = Tid[m][t] at rank t of
// key m's sorted list, cell = code7_m(r) * 128 + code7_p(r) with p the partner
// of m and code7 = code >> 1; all-ones padding up to NP.  Sorted, a cell's
// references keep the sorted list's order (distance to k_m, then index).
__global__ void k_make_pair_keys(const uint8_t* __restrict__ code, const int32_t* __restrict__ Tid,
                                 const int32_t* __restrict__ partner, int n, int K, int NP,
                                 unsigned long long* __restrict__ keys) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (t >= NP) return;
  unsigned long long v = ~0ull;
  if (t < n) {
    const int r = Tid[(int64_t)m * n + t];
    const uint32_t cm = code[(int64_t)r * K + m] >> 1, cp = code[(int64_t)r * K + partner[m]] >> 1;
    v = ((unsigned long long)(cm * kPairCodes + cp) << 32) | (unsigned)t;
  }
  keys[(int64_t)m * NP + t] = v;
}

__global__ void k_pair_split(const unsigned long long* __restrict__ keys, const int32_t* __restrict__ Tid, int n,
                             int NP, int32_t* __restrict__ Tid2) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (j >= n) return;
  const int t = (int)(keys[(int64_t)m * NP + j] & 0xffffffffu);
  Tid2[(int64_t)m * n + j] = Tid[(int64_t)m * n + t];
}

// OFF[m][v] = first position j of key m's pair order whose cell is >= v, for
// v = 0 .. kPairCodes^2 (the last entry is n).
__global__ void k_pair_offsets(const unsigned long long* __restrict__ keys, int n, int NP, uint32_t* __restrict__ OFF) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  constexpr int kCells = kPairCodes * kPairCodes;
  if (v > kCells) return;
  const unsigned long long* t = keys + (int64_t)m * NP;
  int lo = 0, len = n;
  while (len > 0) {
    const int half = len >> 1;
    if ((uint32_t)(t[lo + half] >> 32) < (uint32_t)v) { lo += half + 1; len -= half + 1; } else { len = half; }
  }
  OFF[(int64_t)m * (kCells + 1) + v] = (uint32_t)lo;
}

}  // namespace

// Ascending sort of nseg segments of NP keys each (NP a power of two >= 2048),
// in batches of at most 32768 segments (the grid's y extent).
cudaError_t sort_segments(unsigned long long* keys, int NP, int64_t nseg, cudaStream_t s) {
  for (int64_t b0 = 0; b0 < nseg; b0 += 32768) {
    const int nb = (int)(nseg - b0 < 32768 ? nseg - b0 : 32768);
    unsigned long long* k0 = keys + b0 * NP;
    k_bitonic_shared<<<dim3(NP / kChunk, nb), kChunk / 2, 0, s>>>(k0, NP, 0);
    for (int k = 2 * kChunk; k <= NP; k <<= 1) {
      for (int j = k >> 1; j >= kChunk; j >>= 1)
        k_bitonic_global<<<dim3((NP / 2 + 255) / 256, nb), 256, 0, s>>>(k0, NP, k, j);
      k_bitonic_shared<<<dim3(NP / kChunk, nb), kChunk / 2, 0, s>>>(k0, NP, k);
    }
  }
  return cudaGetLastError();
}

int sort_chunk() { return kChunk; }

cudaError_t launch_index_build(Index& ix, cudaStream_t s) {
  const int n = ix.n, K = ix.K, D = ix.D;
  if (ix.unit) {   // unit-normalised float variant: P holds float bits
    const cudaError_t e0 = launch_unit_tables(ix, s);
    if (e0 != cudaSuccess) return e0;
  } else {
    int64_t tot = (int64_t)n * ix.Kp;
    k_key_distances<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(ix.R, ix.KP, n, K, ix.Kp, D, ix.P);
  }
  k_prep_refs<<<ix.n_pad, 64, 0, s>>>(ix.R, n, ix.n_pad, D, ix.Rbf, ix.RN, ix.rnorm);
  int NP = kChunk;
  while (NP < n) NP <<= 1;
  unsigned long long* keys = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&keys, sizeof(unsigned long long) * (size_t)NP * K, s);
  if (e != cudaSuccess) return e;
  k_make_keys<<<dim3((NP + 255) / 256, K), 256, 0, s>>>(ix.P, n, ix.Kp, NP, keys);
  k_bitonic_shared<<<dim3(NP / kChunk, K), kChunk / 2, 0, s>>>(keys, NP, 0);
  for (int k = 2 * kChunk; k <= NP; k <<= 1) {
    for (int j = k >> 1; j >= kChunk; j >>= 1)
      k_bitonic_global<<<dim3((NP / 2 + 255) / 256, K), 256, 0, s>>>(keys, NP, k, j);
    k_bitonic_shared<<<dim3(NP / kChunk, K), kChunk / 2, 0, s>>>(keys, NP, k);
  }
  k_split_keys<<<dim3((n + 255) / 256, K), 256, 0, s>>>(keys, n, NP, ix.TA, ix.Tid);
  e = cudaFreeAsync(keys, s);
  if (e != cudaSuccess) return e;

  k_bucket_edges<<<K, kBuckets, 0, s>>>(ix.TA, n, K, ix.E, ix.RB);
  uint8_t* code = nullptr;
  e = cudaMallocAsync((void**)&code, (size_t)n * K, s);
  if (e != cudaSuccess) return e;
  {
    const int64_t tot = (int64_t)n * K;
    k_codes<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(ix.P, ix.E, n, K, ix.Kp, code);
  }
  // the pair order of every key (Sec. 3.3's sorted lists refined by a second
  // key's bucket code): its reference ids, cell offsets and filter codes
  k_partners<<<(K + 63) / 64, 64, 0, s>>>(ix.KP, K, D, ix.pair_scan ? 0 : 1, ix.partner);
  e = cudaMallocAsync((void**)&keys, sizeof(unsigned long long) * (size_t)NP * K, s);
  if (e != cudaSuccess) return e;
  k_make_pair_keys<<<dim3((NP + 255) / 256, K), 256, 0, s>>>(code, ix.Tid, ix.partner, n, K, NP, keys);
  e = sort_segments(keys, NP, K, s);
  if (e != cudaSuccess) return e;
  k_pair_split<<<dim3((n + 255) / 256, K), 256, 0, s>>>(keys, ix.Tid, n, NP, ix.Tid2);
  k_pair_offsets<<<dim3((kPairCodes * kPairCodes + 1 + 255) / 256, K), 256, 0, s>>>(keys, n, NP, ix.OFF);
  e = cudaFreeAsync(keys, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(ix.CW, 0, sizeof(uint32_t) * (size_t)K * ix.G * ix.nw, s);
  if (e != cudaSuccess) return e;
  k_pack_codes<<<dim3((n + 255) / 256, K), 256, 0, s>>>(ix.Tid2, code, n, K, ix.G, ix.nw, ix.CW);
  k_pack_entry_codes<<<dim3((unsigned)(((int64_t)n * ix.Ke + 255) / 256), K), 256, 0, s>>>(ix.Tid2, code, n, K,
                                                                                          ix.Ke, ix.CE);
  e = cudaFreeAsync(code, s);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace riann
