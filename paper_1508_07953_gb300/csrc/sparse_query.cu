// sparse_query.cu -- the per-query RIANN step for frames with a previous field
// (Alg. 1 loop body): previous match and temporal change, ring bounds in the
// sorted per-key lists (Sec. 3.3), intersection of the rings, verification of
// the survivors (Alg. 1 final argmin).
//
// One warp per query.  A CTA owns a TY x TX tile of query positions, stages
// the (TY+7) x (TX+7) pixels they read plus all key points in shared memory,
// and hands queries to its warps through a shared counter (candidate counts
// vary by orders of magnitude between queries, Sec. 3.3 / Fig. 5).
//
// Ring sizes and the first filter of the intersection work on 8-bit bucket
// codes (see common.cuh): a reference whose code for key m lies outside the
// code range of the exact ring bounds is not a member of ring m.  The
// references that pass the filter are then tested exactly against every ring
// from their row of key-point distances in P (16 MB for n = 65536, K = 64:
// it stays in L2).
#include <algorithm>

#include "unit.cuh"

namespace riann {
namespace {

constexpr int kWarps = 8;
constexpr int kCtasPerSm = 3;   // register budget 80 per thread
constexpr unsigned kFull = 0xffffffffu;
constexpr int kCarveDevices = 64;          // devices whose carveout preference has been set
constexpr int kSmemPerCtaReserved = 1024;  // shared memory the hardware reserves per resident CTA

// Exact ring membership |sqrt(A) - sqrt(B)| <= (p/q) sqrt(C) for A, B <= 192*255^2:
// q^2 (A + B) - p^2 C <= 2 q^2 sqrt(A B)  <=>  L <= 0  or  L^2 <= 4 q^4 A B.
// A positive L is below q^2 (A + B) <= 64 * 2 * 192 * 255^2 < 2^31, so L^2 and
// A B are 32 x 32 -> 64-bit products, and 4 q^4 A B < 2^14 * 2^48 fits 64 bits.
__device__ __forceinline__ bool in_ring(uint32_t A, uint32_t B, uint32_t C, uint32_t p2,
                                        uint32_t q2) {
  const int64_t L = (int64_t)q2 * ((int64_t)A + (int64_t)B) - (int64_t)p2 * (int64_t)C;
  if (L <= 0) return true;
  const uint32_t l = (uint32_t)L;
  const unsigned long long ll = (unsigned long long)l * l;
  const unsigned long long ab = (unsigned long long)A * B;
  const unsigned long long k = 4u * q2 * q2;
  return ll <= ab * k;
}

// Farthest member of the ring from B on one side: the smallest member in
// [0, B] (up = false) or the largest in [B, Amax] (up = true).  The ring is an
// interval holding B, so in the offset t = |A - B| membership is true up to
// some t* and false beyond.  The float estimate (usually exact or off by one)
// is probed first and then its neighbour; otherwise the search gallops on
// with doubling steps -- away from B from a member, towards B from a
// non-member -- until it brackets t*, then bisects.  An estimate error only
// costs iterations; one membership test per iteration.
__device__ uint32_t ring_edge(uint32_t B, uint32_t C, uint32_t p2, uint32_t q2, float est, bool up,
                              uint32_t Amax) {
  uint32_t t;                                      // offset of the estimate
  if (up) t = (est <= (float)B ? B : (est >= (float)Amax ? Amax : (uint32_t)est)) - B;
  else t = B - (est <= 0.f ? 0u : (est >= (float)B ? B : (uint32_t)ceilf(est)));
  uint32_t good = 0, bad = (up ? Amax - B : B) + 1;   // a member at offset good, none at bad
  uint32_t step = 1;
  int mode = 2;                                    // 2: the estimate, +1 / -1: galloping, 0: bisecting
#pragma unroll 1
  for (;;) {
    if (mode == 1) {
      if (step >= bad - good) mode = 0; else t = good + step;
    } else if (mode == -1) {
      if (step >= bad - good) mode = 0; else t = bad - step;
    }
    if (mode == 0) t = good + (bad - good) / 2;
    const bool in = in_ring(up ? B + t : B - t, B, C, p2, q2);
    if (in) good = t; else bad = t;
    if (bad - good <= 1) return up ? B + good : B - good;
    if (mode == 2) mode = in ? 1 : -1;
    else if (mode == (in ? -1 : 1)) mode = 0;      // bracketed
    else step <<= 1;
  }
}

// Sum of squared byte differences of two 16-byte vectors, added to acc.
__device__ __forceinline__ uint32_t sq4(const uint32_t* q, uint4 u, uint32_t acc) {
  const uint4 a = *reinterpret_cast<const uint4*>(q);
  uint32_t d;
  d = __vabsdiffu4(a.x, u.x); acc = __dp4a(d, d, acc);
  d = __vabsdiffu4(a.y, u.y); acc = __dp4a(d, d, acc);
  d = __vabsdiffu4(a.z, u.z); acc = __dp4a(d, d, acc);
  d = __vabsdiffu4(a.w, u.w); acc = __dp4a(d, d, acc);
  return acc;
}

// code(x) = (number of bucket edges <= x) - 1, in [-1, 255].  Two levels:
// every 8th edge in shared memory (32 per key), then the 8 edges of one
// 32-byte segment from global memory.
__device__ __forceinline__ int bucket_code(const uint32_t* __restrict__ coarse, const uint32_t* __restrict__ e,
                                           uint32_t x) {
  int c = 0;   // coarse edges <= x
#pragma unroll
  for (int half = 16; half > 0; half >>= 1)
    if (coarse[c + half - 1] <= x) c += half;
  if (c == 31 && coarse[31] <= x) c = 32;
  if (c == 0) return -1;
  const uint4* s = reinterpret_cast<const uint4*>(e + 8 * (c - 1));
  const uint4 u = __ldg(s), v = __ldg(s + 1);
  return 8 * (c - 1) + (u.x <= x) + (u.y <= x) + (u.z <= x) + (u.w <= x) + (v.x <= x) + (v.y <= x) +
         (v.z <= x) + (v.w <= x) - 1;
}

// Number of entries of the sorted range t[lo, hi) below v (le: at most v),
// counted by the whole warp with coalesced loads; every lane gets the result.
__device__ __forceinline__ int warp_count_below(const uint32_t* __restrict__ t, int lo, int hi, uint32_t v,
                                                bool le, int lane) {
  int c = 0;
#pragma unroll 1
  for (int base = lo; base < hi; base += 256) {
    uint32_t x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int j = base + 32 * i + lane;
      x[i] = j < hi ? __ldg(t + j) : 0xffffffffu;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int j = base + 32 * i + lane;
      c += __popc(__ballot_sync(kFull, j < hi && (le ? x[i] <= v : x[i] < v)));
    }
  }
  return c;
}

// Rank range [first >= lo, first > hi) of the exact ring [lo, hi] in TA[m]:
// the first end lies in bucket clo's rank range, the second in bucket chi's.
__device__ __forceinline__ int2 ring_run(const uint32_t* __restrict__ ta, const uint32_t* __restrict__ rb,
                                         int clo, int chi, uint32_t lo, uint32_t hi, int lane,
                                         uint32_t* status) {
  const int a0 = clo < 0 ? 0 : (int)__ldg(rb + clo), a1 = (int)__ldg(rb + clo + 1);
  const int b0 = chi < 0 ? 0 : (int)__ldg(rb + chi), b1 = (int)__ldg(rb + chi + 1);
#if defined(RIANN_CHECKED)
  // the sorted list holds rb[kBuckets] entries: its counted ranges end there
  if (!(a0 <= a1 && b0 <= b1 && a1 <= (int)__ldg(rb + kBuckets) && b1 <= (int)__ldg(rb + kBuckets))) {
    if (lane == 0) atomicOr(status, RIANN_DEV_BOUNDS);
    return make_int2(0, 0);
  }
#endif
  const int a = a0 + warp_count_below(ta, a0, a1, lo, false, lane);
  const int b = b0 + warp_count_below(ta, b0, b1, hi, true, lane);
  return make_int2(a, b > a ? b : a);
}

// Filter codes are bytes 0x80 | c with c < 128, and range bounds bytes l <= 127
// and h1 = hi + 1 <= 128, so each byte of w - lo and w - h1 stays in [0, 255]
// (no borrow into the next byte): bit 7 of the first is [c >= l], of the
// second [c > hi].  A word passes when every byte has c in [l, hi].
constexpr uint32_t kHi = 0x80808080u;

// k-NN variant: the warp's best keys so far, lane j < k holding the j-th
// smallest (dist << 32 | index), the other lanes ~0.  Each lane offers one
// key (~0: none); offers are merged smallest first while they beat the k-th.
__device__ __forceinline__ void knn_merge(unsigned long long& list, unsigned long long offer, int k, int lane) {
  unsigned long long kth = __shfl_sync(kFull, list, k - 1);
  bool pend = offer < kth;
  while (__any_sync(kFull, pend)) {
    unsigned long long m = pend ? offer : ~0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long v = __shfl_xor_sync(kFull, m, o);
      m = v < m ? v : m;
    }
    if (offer == m) pend = false;                  // keys are distinct (distinct indices)
    const int pos = __popc(__ballot_sync(kFull, list < m));
    const unsigned long long up = __shfl_up_sync(kFull, list, 1);
    if (lane < k) list = lane < pos ? list : (lane == pos ? m : up);
    kth = __shfl_sync(kFull, list, k - 1);
    pend = pend && offer < kth;
  }
}

constexpr int kQueueA = 256;  // per-warp ring buffers of the filter cascade (powers of two)
constexpr int kQueueC = 64;
constexpr int kMaxRuns = kPairCodes;   // runs of one query: one per 7-bit seed bucket

// One CTA per tile of TY x TX query positions; the grid is one frame's tiles.
// Single-frame launch (BATCH = false): the frame's descriptor is a kernel
// parameter.  Batched form (BATCH = true): one launch per frame of the batch,
// the descriptor read from the device item array (entry a.item), so a
// captured graph of the launches stays valid while the descriptors change
// from one step to the next.  (A persistent launch taking the tiles of all
// frames from an atomic counter measured 8 % slower.)  KNN: the k-NN output
// (the k best of S u {r_p} instead of the argmin), single-frame launches only.
// UNIT: the unit-normalised float variant (unit.cuh) -- normalised query,
// float distances and ring bounds as float bit patterns; single-frame only.
template <int C, int SHAPE, bool BATCH, bool KNN, bool UNIT>
__global__ void __launch_bounds__(kWarps * 32, kCtasPerSm) k_sparse(const __grid_constant__ SparseArgs a) {
  constexpr int TY = SHAPE == kTile4x32 ? 4 : 8;
  constexpr int TX = SHAPE == kTile4x32 ? 32 : 16;
  constexpr int D = 64 * C, NW = D / 4;
  constexpr int TROW = (TX + 7) * C;              // tile row bytes
  constexpr int TROWP = ((TROW + 8) + 3) & ~3;    // + room for the 8-byte funnel reads
  constexpr int KPW = NW + 1;                     // key-point row stride in words (odd: no bank conflicts)
  constexpr int kMaxG = kMaxK / 4;
  __shared__ __align__(16) uint8_t s_tile[(TY + 7) * TROWP];
  __shared__ uint32_t s_kp[kMaxK * KPW];
  __shared__ uint32_t s_coarse[kMaxK][33];        // every 8th bucket edge per key (padded: no bank conflicts)
  // exact ring bounds [lo, hi] on A as (lo, hi - lo) per key; padding keys (0, ~0)
  __shared__ __align__(16) uint32_t s_lw[kWarps][2 * kMaxK];
  __shared__ int16_t s_clo[kWarps][kMaxK];        // their bucket codes (-1..255)
  __shared__ int16_t s_chi[kWarps][kMaxK];
  __shared__ uint32_t s_ub[kWarps][kMaxK];        // buckets each ring touches
  // per group in filter order: (offset of its code row in CW, packed 7-bit
  // lo, packed hi + 1, unused)
  __shared__ uint4 s_gd[kWarps][kMaxScanDepth];
  __shared__ __align__(16) uint32_t s_klo[kWarps][kMaxG];   // the same ranges in key order
  __shared__ __align__(16) uint32_t s_khi[kWarps][kMaxG];
  __shared__ __align__(16) uint32_t s_kil[kWarps][kMaxG];   // interiors: packed lo + 1 and hi
  __shared__ __align__(16) uint32_t s_kih[kWarps][kMaxG];
  __shared__ int32_t s_partner[kMaxK];            // scan partner of each key
  __shared__ uint32_t s_rs[kWarps][kMaxRuns];     // the query's runs in the seed's pair order: first position,
  __shared__ uint32_t s_rl[kWarps][kMaxRuns];     // and length
  __shared__ int32_t s_qa[kWarps][kQueueA];       // filter queues: run positions after stage A,
  __shared__ int32_t s_qc[kWarps][kQueueC];       // reference ids after stage B,
  __shared__ uint16_t s_qm[kWarps][kQueueC];      // and the words of their boundary codes
  __shared__ uint16_t s_pr[kWarps][32 * kMaxG];   // stage D: (entry, word) pairs of a batch
  __shared__ uint32_t s_fail[kWarps];             // stage D: entries with a failed word
  __shared__ __align__(16) uint32_t s_q[kWarps][NW];   // the warp's query patch
  __shared__ int32_t s_dense[TY * TX];
  __shared__ __align__(16) float s_qf[UNIT ? kWarps : 1][UNIT ? D : 4];   // UNIT: the normalised query
  __shared__ int s_next, s_ndense, s_dense_base;
  __shared__ FrameItem s_item;                    // batched launch: this launch's frame
  __shared__ unsigned long long s_stat[5];        // ring-answered queries, scanned entries, |S|, B and D entries

  const int K = a.K, n = a.n, G = a.G;
  {
    const uint32_t* kp = reinterpret_cast<const uint32_t*>(a.KP);
    for (int i = threadIdx.x; i < K * NW; i += blockDim.x) s_kp[(i / NW) * KPW + (i % NW)] = kp[i];
    for (int i = threadIdx.x; i < K * 32; i += blockDim.x) s_coarse[i >> 5][i & 31] = __ldg(a.E + (i >> 5) * kBuckets + 8 * (i & 31));
    for (int i = threadIdx.x; i < K; i += blockDim.x) s_partner[i] = __ldg(a.partner + i);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;          // lanes below this one
  const uint32_t p2 = (uint32_t)(a.alpha_num * a.alpha_num);
  const uint32_t q2 = (uint32_t)(a.alpha_den * a.alpha_den);
  const float alpha = (float)a.alpha_num / (float)a.alpha_den;
  const uint32_t Amax = max_sqdist(D);

  {
  // ---- this CTA's tile and its frame (kept in shared memory or read from
  // the kernel parameters, not copied into registers) ----
  if (BATCH) {
    if (threadIdx.x == 0) s_item = a.items[a.item];
    __syncthreads();
  }
  const FrameItem& it = BATCH ? s_item : a.one;
  const int tile = (int)blockIdx.x;
  // a batched launch is sized for the largest frame its slot has held
  // (an empty slot has tiles_x = 0): CTAs past this frame's tiles leave
  if (BATCH && tile >= it.tiles_x * ((it.Hq + TY - 1) / TY)) return;
  const int ty0 = (tile / it.tiles_x) * TY;
  const int tx0 = (tile % it.tiles_x) * TX;
  {
    const int64_t rowb = (int64_t)it.W * C;
#pragma unroll 1
    for (int i = threadIdx.x; i < (TY + 7) * TROWP; i += blockDim.x) {
      const int r = i / TROWP, c = i % TROWP;
      const int y = ty0 + r;
      const int64_t xb = (int64_t)tx0 * C + c;
      s_tile[i] = (c < TROW && y < it.H && xb < rowb) ? it.frame[(int64_t)y * rowb + xb] : (uint8_t)0;
    }
    if (threadIdx.x == 0) { s_next = 0; s_ndense = 0; s_stat[0] = s_stat[1] = s_stat[2] = s_stat[3] = s_stat[4] = 0; }
  }
  __syncthreads();

  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(&s_next, 1);
    t = __shfl_sync(kFull, t, 0);
    if (t >= TY * TX) break;
    const int ly = t / TX, lx = t % TX;
    const int y = ty0 + ly, x = tx0 + lx;
    if (y >= it.Hq || x >= it.Wq) continue;
    const int64_t qi = (int64_t)y * it.Wq + x;
    if (!it.prev) {   // no previous field: brute force (Alg. 1's initialisation step)
      if (lane == 0) s_dense[atomicAdd(&s_ndense, 1)] = (int32_t)(it.query_begin + qi);
      continue;
    }

    // a1: the query patch, 4 bytes per word, (dy, dx, c) order, kept in shared
    // memory for the whole query (registers go to the scan)
    uint32_t* q = s_q[warp];
    for (int w = lane; w < NW; w += 32) {
      const int dy = w / (2 * C), j = w % (2 * C);
      const int off = (ly + dy) * TROWP + lx * C + 4 * j;
      const int al = off & ~3;
      const uint32_t lo = *reinterpret_cast<const uint32_t*>(s_tile + al);
      const uint32_t hi = *reinterpret_cast<const uint32_t*>(s_tile + al + 4);
      q[w] = __funnelshift_r(lo, hi, (off & 3) * 8);
    }
    __syncwarp();

    // previous match r_p and temporal change C = ||q - r_p||^2 (Alg. 1: r_i, d_i)
    const int rp = __ldg(it.prev + qi);
    if ((unsigned)rp >= (unsigned)n) {
      if (lane == 0) {
        atomicOr(a.status, RIANN_DEV_BAD_PREV);
        it.out_annf[qi] = -1;
        if (it.out_dist) it.out_dist[qi] = 0xffffffffu;
        if (it.out_count) it.out_count[qi] = 0u;
      }
      if (KNN && lane < a.knn) {
        a.knn_idx[qi * a.knn + lane] = -1;
        if (a.knn_dist) a.knn_dist[qi * a.knn + lane] = 0xffffffffu;
      }
      continue;
    }
    uint32_t Cd = 0;
    float Cf = 0.f, Tf = 0.f;                       // UNIT: C and the ring half-width T
    float* qf = s_qf[UNIT ? warp : 0];
    if (UNIT) {
      // q' = q / ||q|| (exact integer sum of squares), then C = d(q', r'_p)
      uint32_t ss = 0;
      for (int w = lane; w < NW; w += 32) ss = __dp4a(q[w], q[w], ss);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(kFull, ss, o);
      const float nv = unit_scale(ss);
      for (int w = lane; w < NW; w += 32) {
        const uint32_t v = q[w];
#pragma unroll
        for (int j = 0; j < 4; ++j) qf[4 * w + j] = unit_coord((v >> (8 * j)) & 0xffu, ss, nv);
      }
      __syncwarp();
      Cf = unit_dist<D>(qf, a.Rf + (int64_t)rp * D);
      Tf = unit_width(a.alpha_num, a.alpha_den, Cf);
      Cd = __float_as_uint(Cf);
    } else {
      const uint4* r4 = reinterpret_cast<const uint4*>(a.R + (int64_t)rp * D);
#pragma unroll
      for (int v = 0; v < NW / 4; ++v) Cd = sq4(q + 4 * v, __ldg(r4 + v), Cd);
    }

    // a2: per ring m (lane m and m+32): B_m, exact bounds [lo, hi] on A, their
    // bucket codes, and bucket-granular bounds lb <= |Ring_m| <= ub.
    const float sC = (float)Cd;
    uint32_t seedkey = 0xffffffffu;                // (bucket width << 6) | m, width <= 256
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      const int m = lane + 32 * h;
      if (m < K) {
        uint32_t lo, hi;
        if (UNIT) {
          const float Bf = unit_dist<D>(a.KPf + (int64_t)m * D, qf);
          lo = unit_ring_low(Bf, Tf);
          hi = unit_ring_high(Bf, Tf);
        } else {
          const uint32_t* kp = s_kp + m * KPW;
          uint32_t B = 0;
#pragma unroll
          for (int w = 0; w < NW; ++w) {
            const uint32_t d = __vabsdiffu4(q[w], kp[w]);
            B = __dp4a(d, d, B);
          }
          const float cross = 2.f * alpha * sqrtf((float)B * sC);
          const float base = (float)B + alpha * alpha * sC;
          lo = ring_edge(B, Cd, p2, q2, base - cross, false, Amax);
          hi = ring_edge(B, Cd, p2, q2, base + cross, true, Amax);
        }
        const uint32_t* e = a.E + m * kBuckets;
        const int clo = bucket_code(s_coarse[m], e, lo);
        const int chi = bucket_code(s_coarse[m], e, hi);
        // buckets the ring touches: picks the seed and orders the filter
        // groups (performance only; the result does not depend on them)
        const uint32_t width = chi < 0 ? 0u : (uint32_t)(chi - (clo < 0 ? 0 : clo) + 1);
        s_lw[warp][2 * m] = lo;
        s_lw[warp][2 * m + 1] = hi - lo;
        s_clo[warp][m] = (int16_t)clo;
        s_chi[warp][m] = (int16_t)chi;
        s_ub[warp][m] = width;
        const uint32_t key = (width << 6) | (uint32_t)m;
        seedkey = key < seedkey ? key : seedkey;
      } else if (m < a.Kp) {   // padding key of a distance row: always passes
        s_lw[warp][2 * m] = 0u;
        s_lw[warp][2 * m + 1] = 0xffffffffu;
      }
    }
    int ms = (int)(__reduce_min_sync(kFull, seedkey) & 63u);
    __syncwarp();

    // routing: brute force iff every ring holds more than ring_limit
    // references.  Settled at once when the seed's bucket-granular upper bound
    // (first ranks of the buckets, RB) is within the limit; else by the seed
    // ring's exact size (its run in TA, counted by the whole warp), then by
    // the bounds of every ring and exact sizes of the rings whose bounds
    // straddle the limit -- the ring that settles it becomes the seed.
    if (a.ring_limit >= 0) {
      const int sclo = s_clo[warp][ms], schi = s_chi[warp][ms];
      const uint32_t* rbs = a.RB + ms * (kBuckets + 1);
      const uint32_t ubs = __ldg(rbs + schi + 1) - (sclo < 0 ? 0u : __ldg(rbs + sclo));
      bool found = ubs <= (uint32_t)a.ring_limit;
      // rings counted exactly, in order: the seed, then (unless some ring is
      // certainly within the limit) every ring whose bounds straddle it
      int cand = found ? -1 : ms;
      bool first = true;
      unsigned todo0 = 0u, todo1 = 0u;
      while (cand >= 0) {
        const int2 rr = ring_run(a.TA + (int64_t)cand * n, a.RB + cand * (kBuckets + 1), s_clo[warp][cand],
                                 s_chi[warp][cand], s_lw[warp][2 * cand],
                                 s_lw[warp][2 * cand] + s_lw[warp][2 * cand + 1], lane, a.status);
        if ((uint32_t)(rr.y - rr.x) <= (uint32_t)a.ring_limit) {
          found = true;
          ms = cand;
          break;
        }
        if (first) {
          first = false;
          uint32_t ubkey = 0xffffffffu;              // (smallest upper bound over the other rings << 6) | ring
#pragma unroll 1
          for (int h = 0; h < 2; ++h) {
            const int m = lane + 32 * h;
            bool mine = false;
            if (m < K && m != ms) {
              const int clo = s_clo[warp][m], chi = s_chi[warp][m];
              const uint32_t* rb = a.RB + m * (kBuckets + 1);
              const uint32_t ub = __ldg(rb + chi + 1) - (clo < 0 ? 0u : __ldg(rb + clo));
              const uint32_t lb = chi > clo + 1 ? __ldg(rb + chi) - __ldg(rb + clo + 1) : 0u;
              const uint32_t k2 = (ub << 6) | (uint32_t)m;   // ub <= n <= 2^24
              ubkey = k2 < ubkey ? k2 : ubkey;
              mine = ub > (uint32_t)a.ring_limit && lb <= (uint32_t)a.ring_limit;
            }
            const unsigned bal = __ballot_sync(kFull, mine);
            if (h == 0) todo0 = bal; else todo1 = bal;
          }
          ubkey = __reduce_min_sync(kFull, ubkey);
          if (ubkey != 0xffffffffu && (ubkey >> 6) <= (uint32_t)a.ring_limit) {   // a ring certainly within the limit
            ms = (int)(ubkey & 63u);
            found = true;
            break;
          }
        }
        cand = todo0 ? __ffs(todo0) - 1 : (todo1 ? __ffs(todo1) - 1 + 32 : -1);
        if (todo0) todo0 &= todo0 - 1; else todo1 &= todo1 - 1;
      }
      if (!found) {
        if (lane == 0) s_dense[atomicAdd(&s_ndense, 1)] = (int32_t)(it.query_begin + qi);
        continue;
      }
    }

    // a3: the runs the scan visits.  In the pair order of the seed ms (its
    // references sorted by the cells (code7_ms, code7_pm), pm its partner key,
    // each cell in the order of the seed's sorted list), every seed bucket b
    // of the seed ring's 7-bit code range holds one contiguous run of the
    // references whose partner code lies in the partner ring's range: run b =
    // [OFF(b, cl), OFF(b, ch + 1)); adjacent runs are merged.  The runs cover
    // every member of both rings (and more: the code ranges are supersets).
    // A seed paired with itself keeps its sorted list's order, and the scan
    // visits the seed ring's exact run in it.  An empty ring leaves no run:
    // S is empty.
    const int pm = s_partner[ms];
    int nruns = 0;
    uint32_t scanned = 0;
    {
      const int sclo = s_clo[warp][ms], schi = s_chi[warp][ms];
      const int pclo = s_clo[warp][pm], pchi = s_chi[warp][pm];
      if (pm == ms) {
        const int2 run = ring_run(a.TA + (int64_t)ms * n, a.RB + ms * (kBuckets + 1), sclo, schi,
                                  s_lw[warp][2 * ms], s_lw[warp][2 * ms] + s_lw[warp][2 * ms + 1], lane, a.status);
        if (run.y > run.x) {
          nruns = 1;
          scanned = (uint32_t)(run.y - run.x);
          if (lane == 0) {
            s_rs[warp][0] = (uint32_t)run.x;
            s_rl[warp][0] = scanned;
          }
        }
      } else if (schi >= 0 && pchi >= 0) {
        const int bl = (sclo < 0 ? 0 : sclo) >> 1, bh = schi >> 1;
        const int cl = (pclo < 0 ? 0 : pclo) >> 1, ch = pchi >> 1;
        const int nb = bh - bl + 1;
        const uint32_t* off = a.OFF + (int64_t)ms * (kPairCodes * kPairCodes + 1);
#pragma unroll 1
        for (int b0 = 0; b0 < nb; b0 += 32) {
          // one bucket per lane; a run that starts where the lower lane's
          // ends continues it, and a head's run ends with the last lane
          // below the next head
          const bool v = b0 + lane < nb;
          uint32_t st = 0, en = 0;
          if (v) {
            const uint32_t* ob = off + (bl + b0 + lane) * kPairCodes;
            st = __ldg(ob + cl);
            en = __ldg(ob + ch + 1);
            if (!RIANN_IN_RANGE(st <= en && en <= (uint32_t)n, a.status)) st = en = 0u;
          }
          const uint32_t pen = __shfl_up_sync(kFull, en, 1);
          const bool head = v && (lane == 0 || st != pen);
          const unsigned hm = __ballot_sync(kFull, head), vm = __ballot_sync(kFull, v);
          const unsigned above = hm & ~((2u << lane) - 1u);
          const int last = above ? __ffs(above) - 2 : 31 - __clz(vm);
          const uint32_t send = __shfl_sync(kFull, en, last);
          if (head) {
            const int k = nruns + __popc(hm & lt);
            s_rs[warp][k] = st;
            s_rl[warp][k] = send - st;
          }
          nruns += __popc(hm);
          scanned += v ? en - st : 0u;
        }
        scanned = __reduce_add_sync(kFull, scanned);
      }
    }
    // per group of 4 keys: the 7-bit code ranges of its rings (filter codes
    // are 0x80 | code7 with code7 = code >> 1, see index_build.cu), packed one
    // byte per key as lo and hi + 1 (keys that always pass -- the seed and its
    // partner, whose ranges the runs already meet, and padding -- take [0, 127];
    // an empty ring takes lo = hi + 1 = 1, which no code meets), and an
    // estimate of the fraction of references passing
    // (product over its keys of the fraction of buckets each ring touches)
    float est = 2.f;
    uint32_t glo = 0, ghi = 0;                     // the scan's ranges (seed and partner always pass)
    uint32_t elo = 0, ehi = 0, ilo = 0, ihi = 0;   // every ring's range, and its interior (see below)
    if (lane < G) {
      est = 1.f;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int k = 4 * lane + i;
        uint32_t l = 0, h1 = 128, l1 = 0, h0 = 128;
        if (k < K) {
          const int clo = s_clo[warp][k], chi = s_chi[warp][k];
          if (chi < 0) {
            l = h1 = 1;
          } else {
            l = (uint32_t)(clo < 0 ? 0 : clo) >> 1;
            h1 = ((uint32_t)chi >> 1) + 1;
            l1 = l + 1;
            h0 = h1 - 1;
          }
        }
        // a code strictly inside its ring's code range (l < c < hi) lies in
        // a bucket entirely inside the ring: only the others need the exact test
        elo |= l << (8 * i);
        ehi |= h1 << (8 * i);
        ilo |= l1 << (8 * i);
        ihi |= h0 << (8 * i);
        if (k < K && k != ms && k != pm) {
          est *= (float)s_ub[warp][k] * (1.f / kBuckets);   // fraction of buckets the ring touches
          glo |= l << (8 * i);
          ghi |= h1 << (8 * i);
        } else {
          ghi |= 128u << (8 * i);
        }
      }
    }
    {
      // the scan's groups: the ns1 smallest estimates (ties: lower group),
      // each found by a warp minimum over (estimate bits, group) -- the
      // estimates are non-negative floats, whose bits order like them
      const int nsel = min(min(G, a.depth), kMaxScanDepth);
      uint32_t ekey = (__float_as_uint(est) & ~31u) | (uint32_t)lane;
      for (int i = 0; i < nsel; ++i) {
        const uint32_t mn = __reduce_min_sync(kFull, ekey);
        if ((uint32_t)lane == (mn & 31u)) {
          s_gd[warp][i] = make_uint4((uint32_t)(lane * a.nw), glo, ghi, 0u);
          ekey = 0xffffffffu;
        }
      }
      // in key order for the entry rows (padding groups of a row always pass
      // and are interior)
      if (lane < (a.Ke >> 2)) {
        s_klo[warp][lane] = lane < G ? elo : 0u;
        s_khi[warp][lane] = lane < G ? ehi : kHi;
        s_kil[warp][lane] = lane < G ? ilo : 0u;
        s_kih[warp][lane] = lane < G ? ihi : kHi;
      }
    }
    __syncwarp();

    // a3 + a4, a cascade of filters over the runs; each stage compacts its
    // survivors into a per-warp queue (warp ballots), so that the next,
    // costlier stage runs on full batches of 32:
    //   A  32 words of 4 run positions per step (one per lane; a step that
    //      reaches the end of a run continues in the next one), against
    //      the codes of the ns1 most selective groups (rows of CW: one 16-byte
    //      load per group);
    //   B  one queued position per lane: its reference id (Tid2) and the
    //      codes of every key (its row of CE, one 16-byte load per 16 keys);
    //   D  one queued reference per lane: the exact test, lo_m <= A_m <= hi_m
    //      as one unsigned compare (A_m - lo_m <= hi_m - lo_m), of the keys
    //      whose codes B found on a boundary of their range (a 4-key word of
    //      the distance row each, spread over the warp's lanes), and
    //      verification of the members against the query.
    // A code range is a superset of its ring, so only D decides membership.
    // A deeper stage runs first whenever it holds a full batch, which bounds
    // the queues (A: < 32 + 128 entries, C: < 64).
    // (k-NN: the same start -- r_p on lane 0 -- is the warp's best-k list)
    unsigned long long best = lane == 0 ? (((unsigned long long)Cd << 32) | (unsigned)rp) : ~0ull;
    uint32_t cnt = 0;
    const uint32_t* cw = a.CW + (int64_t)ms * G * a.nw;
    const int32_t* tid = a.Tid2 + (int64_t)ms * n;
    const uint8_t* ce = a.CE + (int64_t)ms * n * a.Ke;
    const int kc = a.Ke >> 4;                      // 16-byte words per entry row of CE
    const int ns1 = min(min(G, a.depth), kMaxScanDepth);
    const uint4* gd = s_gd[warp];
    const uint4* prow = reinterpret_cast<const uint4*>(a.P);
    const int kq = a.Kp >> 2;                      // 16-byte words per distance row
    const uint4* lw4 = reinterpret_cast<const uint4*>(s_lw[warp]);
    const uint4* klo4 = reinterpret_cast<const uint4*>(s_klo[warp]);
    const uint4* khi4 = reinterpret_cast<const uint4*>(s_khi[warp]);
    const uint4* kil4 = reinterpret_cast<const uint4*>(s_kil[warp]);
    const uint4* kih4 = reinterpret_cast<const uint4*>(s_kih[warp]);
    const uint32_t* rs = s_rs[warp];
    const uint32_t* rl = s_rl[warp];
    int32_t* qa = s_qa[warp];
    int32_t* qc = s_qc[warp];
    uint16_t* qm = s_qm[warp];
    int ha = 0, na = 0, hc = 0, nc = 0;            // queue heads and lengths
    uint32_t nfilt = 0, nexact = 0;                // entries through B and through D (statistics)

    // scan position (warp-uniform): run ri, 4-aligned chunk start base in it.
    // A chunk's codes are loaded when its step runs: holding the next chunk
    // in registers through the other stages measured slower (it costs the
    // compiler 12 registers everywhere in the loop)
    int ri = 0;
    while (ri < nruns && rl[ri] == 0u) ++ri;
    int base = ri < nruns ? (int)(rs[ri] & ~3u) : 0;
    for (;;) {
      const bool done = ri >= nruns;
      if (nc >= 32 || (done && nc > 0)) {
        // ---- D: exact test of the boundary words, and verification ----
        // Entry e (lane e) needs the exact key distances only of the words
        // in its mask.  The warp spreads its (entry, word) pairs over the
        // lanes -- a lane's pairs after the sum of the lower lanes' counts,
        // from ballots of the counts' five bits -- loads each pair's 16-byte
        // word of the distance row and records a failed word in s_fail.
        const int take = nc < 32 ? nc : 32;
        bool alive = lane < take;
        const int slot = (hc + lane) & (kQueueC - 1);
        const int r = alive ? qc[slot] : 0;
        uint32_t mk = alive ? (uint32_t)qm[slot] : 0u;
        hc = (hc + take) & (kQueueC - 1);
        nexact += take;
        nc -= take;
        const uint32_t pc = (uint32_t)__popc(mk);
        int ppos = 0, ptot = 0;
#pragma unroll
        for (int bt = 0; bt < 5; ++bt) {
          const unsigned bb = __ballot_sync(kFull, (pc >> bt) & 1u);
          ppos += __popc(bb & lt) << bt;
          ptot += __popc(bb) << bt;
        }
        uint16_t* pr = s_pr[warp];
        while (mk) {
          pr[ppos++] = (uint16_t)((lane << 4) | (__ffs(mk) - 1));
          mk &= mk - 1;
        }
        if (lane == 0) s_fail[warp] = 0u;
        __syncwarp();
        for (int p0 = 0; p0 < ptot; p0 += 32) {
          const int k1 = p0 + lane;
          const uint32_t e1 = k1 < ptot ? pr[k1] : 0u;
          const int r1 = __shfl_sync(kFull, r, (int)(e1 >> 4));
          if (k1 < ptot && RIANN_IN_RANGE((int)(e1 & 15u) < kq, a.status)) {
            const uint4 v1 = __ldg(prow + (int64_t)r1 * kq + (e1 & 15u));
            const uint4 l0 = lw4[2 * (e1 & 15u)], l1 = lw4[2 * (e1 & 15u) + 1];
            const bool okw = (v1.x - l0.x <= l0.y) && (v1.y - l0.z <= l0.w) && (v1.z - l1.x <= l1.y) &&
                             (v1.w - l1.z <= l1.w);
            if (!okw) atomicOr(&s_fail[warp], 1u << (e1 >> 4));
          }
        }
        __syncwarp();
        alive = alive && ((s_fail[warp] >> lane) & 1u) == 0u;
        __syncwarp();
        unsigned long long key = ~0ull;
        if (alive) {
          ++cnt;
          uint32_t d = 0;
          if (UNIT) {
            d = __float_as_uint(unit_dist<D>(qf, a.Rf + (int64_t)r * D));
          } else {
            const uint4* r4 = reinterpret_cast<const uint4*>(a.R + (int64_t)r * D);
#pragma unroll
            for (int v = 0; v < NW / 4; ++v) d = sq4(q + 4 * v, __ldg(r4 + v), d);
          }
          key = ((unsigned long long)d << 32) | (unsigned)r;
          if (!KNN) best = key < best ? key : best;
        }
        // k-NN: r_p is on the list already (S u {r_p} is a set)
        if (KNN) knn_merge(best, alive && r != rp ? key : ~0ull, a.knn, lane);
        continue;
      }
      if (na >= 32 || (done && na > 0)) {
        // ---- B: the codes of every key of the entry, and its reference id ----
        const int take = na < 32 ? na : 32;
        const bool on = lane < take;
        const int j = on ? qa[(ha + lane) & (kQueueA - 1)] : 0;
        ha = (ha + take) & (kQueueA - 1);
        nfilt += take;
        na -= take;
        const int r = on ? __ldg(tid + j) : 0;
        const bool rok = !on || RIANN_IN_RANGE((unsigned)r < (unsigned)n, a.status);
        const uint4* er = reinterpret_cast<const uint4*>(ce + (int64_t)j * a.Ke);
        uint32_t pass = kHi, bmask = 0;            // bmask: words of the entry with a boundary code
#pragma unroll
        for (int c = 0; c < kMaxK / 16; ++c) {
          if (c < kc) {
            const uint4 w = on ? __ldg(er + c) : make_uint4(kHi, kHi, kHi, kHi);
            const uint4 l = klo4[c], h = khi4[c], il = kil4[c], ih = kih4[c];
            pass &= (w.x - l.x) & ~(w.x - h.x) & (w.y - l.y) & ~(w.y - h.y);
            pass &= (w.z - l.z) & ~(w.z - h.z) & (w.w - l.w) & ~(w.w - h.w);
            bmask |= ((((w.x - il.x) & ~(w.x - ih.x) & kHi) != kHi) ? 1u : 0u) << (4 * c);
            bmask |= ((((w.y - il.y) & ~(w.y - ih.y) & kHi) != kHi) ? 2u : 0u) << (4 * c);
            bmask |= ((((w.z - il.z) & ~(w.z - ih.z) & kHi) != kHi) ? 4u : 0u) << (4 * c);
            bmask |= ((((w.w - il.w) & ~(w.w - ih.w) & kHi) != kHi) ? 8u : 0u) << (4 * c);
          }
        }
        const bool ok = on && rok && (pass & kHi) == kHi;
        const unsigned m = __ballot_sync(kFull, ok);
        if (ok) {
          const int slot = (hc + nc + __popc(m & lt)) & (kQueueC - 1);
          qc[slot] = r;
          qm[slot] = (uint16_t)bmask;
        }
        nc += __popc(m);
        continue;
      }
      if (done) break;
      // ---- A: 32 words (4 positions each) from word base of run ri; when run
      // ri ends inside them, the rest come from the next non-empty run ----
      const int st = (int)rs[ri], en = st + (int)rl[ri];
      const int left = ((en - 1) >> 2) - (base >> 2) + 1;   // words of run ri from base on (>= 1)
      int ri2 = ri, base2 = base + 128;
      int j0 = base + 4 * lane, lst = st, len = en;        // this lane's word and its run
      bool lin = lane < left;
      const bool edge = base < st || left <= 32;           // a run boundary inside the chunk
      if (left <= 32) {
        ++ri2;
        while (ri2 < nruns && rl[ri2] == 0u) ++ri2;
        base2 = 0;
        if (ri2 < nruns) {
          const int st2 = (int)rs[ri2], en2 = st2 + (int)rl[ri2];
          const int w2 = ((en2 - 1) >> 2) - (st2 >> 2) + 1;      // words of run ri2
          const int take2 = 32 - left;
          if (lane >= left) {
            j0 = (st2 & ~3) + 4 * (lane - left);
            lst = st2;
            len = en2;
            lin = lane - left < w2;
          }
          if (w2 > take2) {
            base2 = (st2 & ~3) + 4 * take2;                       // run ri2 continues
          } else {
            ++ri2;
            while (ri2 < nruns && rl[ri2] == 0u) ++ri2;
            base2 = ri2 < nruns ? (int)(rs[ri2] & ~3u) : 0;
          }
        }
      }
      uint4 av[kMaxScanDepth];
#pragma unroll
      for (int g = 0; g < kMaxScanDepth; ++g) {
        av[g] = make_uint4(0, 0, 0, 0);
        if (g < ns1 && lin) av[g] = __ldg(reinterpret_cast<const uint4*>(cw + gd[g].x) + (j0 >> 2));
      }
      uint32_t p[4] = {kHi, kHi, kHi, kHi};
#pragma unroll
      for (int g = 0; g < kMaxScanDepth; ++g) {
        if (g < ns1) {
          const uint32_t lo = gd[g].y, h1 = gd[g].z;
          p[0] &= (av[g].x - lo) & ~(av[g].x - h1);
          p[1] &= (av[g].y - lo) & ~(av[g].y - h1);
          p[2] &= (av[g].z - lo) & ~(av[g].z - h1);
          p[3] &= (av[g].w - lo) & ~(av[g].w - h1);
        }
      }
      unsigned bits = 0;
#pragma unroll
      for (int u = 0; u < 4; ++u) bits |= ((p[u] & kHi) == kHi ? 1u : 0u) << u;
      // only chunks with a run boundary hold positions outside their runs (a
      // warp-uniform test: the chunks inside a run skip the range check)
      if (edge) {
        unsigned inr = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) inr |= (lin && j0 + u >= lst && j0 + u < len ? 1u : 0u) << u;
        bits &= inr;
      }
      ri = ri2;
      base = base2;
      // append the survivors to queue A: a lane's offset is the sum of the
      // survivor counts (0..4) of the lanes below it, from ballots of the
      // counts' three bits
      const unsigned c = (unsigned)__popc(bits);
      const unsigned c0 = __ballot_sync(kFull, c & 1u), c1 = __ballot_sync(kFull, c & 2u),
                     c2 = __ballot_sync(kFull, c & 4u);
      const int pre = __popc(c0 & lt) + 2 * __popc(c1 & lt) + 4 * __popc(c2 & lt);
      const int tot = __popc(c0) + 2 * __popc(c1) + 4 * __popc(c2);
      int slot = ha + na + pre;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if ((bits >> u) & 1u) qa[(slot++) & (kQueueA - 1)] = j0 + u;
      na += tot;
    }
    if (KNN) {
      if (lane < a.knn) {
        a.knn_idx[qi * a.knn + lane] = best == ~0ull ? -1 : (int32_t)(best & 0xffffffffu);
        if (a.knn_dist) a.knn_dist[qi * a.knn + lane] = (uint32_t)(best >> 32);
      }
      best = __shfl_sync(kFull, best, 0);
    }
    cnt = __reduce_add_sync(kFull, cnt);
    if (!KNN) {   // the (dist, index) minimum: the least distance, then the least index holding it
      const uint32_t dmin = __reduce_min_sync(kFull, (uint32_t)(best >> 32));
      const uint32_t imin = __reduce_min_sync(kFull, (uint32_t)(best >> 32) == dmin ? (uint32_t)best : 0xffffffffu);
      best = ((unsigned long long)dmin << 32) | imin;
    }
    if (lane == 0) {
      it.out_annf[qi] = (int32_t)(best & 0xffffffffu);
      if (it.out_dist) it.out_dist[qi] = (uint32_t)(best >> 32);
      if (it.out_count) it.out_count[qi] = cnt;
      if (a.stats) {
        atomicAdd(&s_stat[0], 1ull);
        atomicAdd(&s_stat[1], (unsigned long long)scanned);
        atomicAdd(&s_stat[2], (unsigned long long)cnt);
        atomicAdd(&s_stat[3], (unsigned long long)nfilt);
        atomicAdd(&s_stat[4], (unsigned long long)nexact);
      }
    }
    __syncwarp();
  }

  // hand the brute-force queries of this tile to the dense path
  __syncthreads();
  if (threadIdx.x == 0 && s_ndense > 0) s_dense_base = (int)atomicAdd(a.counters, (uint32_t)s_ndense);
  if (threadIdx.x == 0 && a.stats) {
    atomicAdd(&a.stats[kStatRingQueries], s_stat[0]);
    atomicAdd(&a.stats[kStatDenseQueries], (unsigned long long)s_ndense);
    atomicAdd(&a.stats[kStatSumSeed], s_stat[1]);
    atomicAdd(&a.stats[kStatSumS], s_stat[2]);
    atomicAdd(&a.stats[kStatSumFiltered], s_stat[3]);
    atomicAdd(&a.stats[kStatSumExact], s_stat[4]);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < s_ndense; i += blockDim.x) a.dense_list[s_dense_base + i] = s_dense[i];
  }
}

// The smallest shared-memory carveout that holds kCtasPerSm CTAs leaves the
// rest of the SM's 256 KB to L1 (the scan's gathers).  Set once per device
// for the four kernels of a (C, SHAPE), under a lock; index building calls it
// (never inside a stream capture), the launches only check the flag.
template <int C, int SHAPE>
cudaError_t carve_ring() {
  static std::mutex mu;
  static bool carved[kCarveDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kCarveDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (carved[dev]) return cudaSuccess;
  const void* fs[4] = {(const void*)k_sparse<C, SHAPE, true, false, false>,
                       (const void*)k_sparse<C, SHAPE, false, false, true>,
                       (const void*)k_sparse<C, SHAPE, false, true, false>,
                       (const void*)k_sparse<C, SHAPE, false, false, false>};
  int smem_max = 0;
  e = cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e != cudaSuccess) return e;
  for (const void* f : fs) {
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return e;
    const int64_t need = (int64_t)kCtasPerSm * ((int64_t)fa.sharedSizeBytes + kSmemPerCtaReserved);
    const int pct = (int)std::min<int64_t>(100, (100 * need + smem_max - 1) / smem_max);
    e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
    if (e != cudaSuccess) return e;
  }
  carved[dev] = true;
  return cudaSuccess;
}

template <int C, int SHAPE>
cudaError_t launch_ring(const SparseArgs& a, bool batch, int grid, cudaStream_t s) {
  cudaError_t e = carve_ring<C, SHAPE>();
  if (e != cudaSuccess) return e;
  if (batch) k_sparse<C, SHAPE, true, false, false><<<grid, kWarps * 32, 0, s>>>(a);
  else if (a.unit) k_sparse<C, SHAPE, false, false, true><<<grid, kWarps * 32, 0, s>>>(a);
  else if (a.knn > 0) k_sparse<C, SHAPE, false, true, false><<<grid, kWarps * 32, 0, s>>>(a);
  else k_sparse<C, SHAPE, false, false, false><<<grid, kWarps * 32, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_any(const SparseArgs& a, int C, int shape, bool batch, int grid, cudaStream_t s) {
  if (C == 1) return shape == kTile8x16 ? launch_ring<1, kTile8x16>(a, batch, grid, s)
                                        : launch_ring<1, kTile4x32>(a, batch, grid, s);
  return shape == kTile8x16 ? launch_ring<3, kTile8x16>(a, batch, grid, s)
                            : launch_ring<3, kTile4x32>(a, batch, grid, s);
}

}  // namespace

cudaError_t ring_prepare(int C) {
  cudaError_t e = C == 1 ? carve_ring<1, kTile4x32>() : carve_ring<3, kTile4x32>();
  if (e == cudaSuccess) e = C == 1 ? carve_ring<1, kTile8x16>() : carve_ring<3, kTile8x16>();
  return e;
}

int ring_tile_rows(int shape) { return shape == kTile8x16 ? 8 : 4; }
int ring_tile_cols(int shape) { return shape == kTile8x16 ? 16 : 32; }

cudaError_t launch_sparse(const SparseArgs& a, int C, int shape, cudaStream_t s) {
  const int tiles = a.one.tiles_x * ((a.one.Hq + ring_tile_rows(shape) - 1) / ring_tile_rows(shape));
  if (tiles <= 0) return cudaSuccess;
  return launch_any(a, C, shape, false, tiles, s);
}

// One frame of a batch: `tiles` CTAs, the frame's descriptor at a.items[a.item].
cudaError_t launch_sparse_item(const SparseArgs& a, int C, int shape, int tiles, cudaStream_t s) {
  if (tiles <= 0) return cudaSuccess;
  return launch_any(a, C, shape, true, tiles, s);
}

}  // namespace riann
