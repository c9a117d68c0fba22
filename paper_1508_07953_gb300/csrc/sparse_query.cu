// sparse_query.cu -- the per-query RIANN step for frames with a previous field
// (Alg. 1 loop body): previous match and temporal change, ring bounds by
// binary search in the sorted per-key lists (Sec. 3.3), intersection of the
// rings, verification of the survivors (Alg. 1 final argmin).
//
// One warp per query.  A CTA owns a TY x TX tile of query positions, stages
// the (TY+7) x (TX+7) pixels they read plus all key points in shared memory,
// and hands queries to its warps through a shared counter (candidate counts
// vary by orders of magnitude between queries, Sec. 3.3 / Fig. 5).
#include "common.cuh"

namespace riann {
namespace {

constexpr int TY = 4, TX = 32;
constexpr int kWarps = 8;
constexpr unsigned kFull = 0xffffffffu;

// Exact ring membership |sqrt(A) - sqrt(B)| <= (p/q) sqrt(C) for A, B <= 192*255^2:
// q^2 (A + B) - p^2 C <= 2 q^2 sqrt(A B)  <=>  L <= 0  or  L^2 <= 4 q^4 A B.
// All terms fit 64-bit integers: L < 64 * 2^25, 4 q^4 A B < 2^14 * 2^48.
__device__ __forceinline__ bool in_ring(uint32_t A, uint32_t B, uint32_t C, uint32_t p2,
                                        uint32_t q2) {
  const int64_t L = (int64_t)q2 * ((int64_t)A + (int64_t)B) - (int64_t)p2 * (int64_t)C;
  if (L <= 0) return true;
  const uint64_t l = (uint64_t)L;
  return l * l <= (4ull * q2 * q2) * (uint64_t)A * (uint64_t)B;
}

// Smallest member A in [0, B] (B itself is always a member: |sqrt B - sqrt B| = 0).
// Membership is false..false true..true on [0, B]; gallop from the estimate,
// then bisect, so any estimate error only costs iterations.
__device__ uint32_t ring_low(uint32_t B, uint32_t C, uint32_t p2, uint32_t q2, float est) {
  if (in_ring(0u, B, C, p2, q2)) return 0u;
  uint32_t a = est <= 0.f ? 0u : (est >= (float)B ? B : (uint32_t)est);
  uint32_t good, bad;   // in_ring(good), !in_ring(bad), bad < good
  if (in_ring(a, B, C, p2, q2)) {
    good = a;
    for (uint32_t step = 1;; step <<= 1) {
      uint32_t c = good > step ? good - step : 0u;
      if (!in_ring(c, B, C, p2, q2)) { bad = c; break; }
      good = c;
    }
  } else {
    bad = a;
    for (uint32_t step = 1;; step <<= 1) {
      uint32_t c = (B - bad > step) ? bad + step : B;
      if (in_ring(c, B, C, p2, q2)) { good = c; break; }
      bad = c;
    }
  }
  while (good - bad > 1) {
    uint32_t mid = bad + (good - bad) / 2;
    if (in_ring(mid, B, C, p2, q2)) good = mid; else bad = mid;
  }
  return good;
}

// Largest member A in [B, Amax]; membership is true..true false..false there.
__device__ uint32_t ring_high(uint32_t B, uint32_t C, uint32_t p2, uint32_t q2, float est,
                              uint32_t Amax) {
  if (in_ring(Amax, B, C, p2, q2)) return Amax;
  uint32_t a = est <= (float)B ? B : (est >= (float)Amax ? Amax : (uint32_t)est);
  uint32_t good, bad;   // in_ring(good), !in_ring(bad), good < bad
  if (in_ring(a, B, C, p2, q2)) {
    good = a;
    for (uint32_t step = 1;; step <<= 1) {
      uint32_t c = (Amax - good > step) ? good + step : Amax;
      if (!in_ring(c, B, C, p2, q2)) { bad = c; break; }
      good = c;
    }
  } else {
    bad = a;
    for (uint32_t step = 1;; step <<= 1) {
      uint32_t c = (bad - B > step) ? bad - step : B;
      if (in_ring(c, B, C, p2, q2)) { good = c; break; }
      bad = c;
    }
  }
  while (bad - good > 1) {
    uint32_t mid = good + (bad - good) / 2;
    if (in_ring(mid, B, C, p2, q2)) good = mid; else bad = mid;
  }
  return good;
}

// first j in [0, n) with t[j] >= v  /  first j with t[j] > v
__device__ __forceinline__ int lower_bound_u32(const uint32_t* __restrict__ t, int n, uint32_t v) {
  int lo = 0, len = n;
  while (len > 0) {
    int half = len >> 1;
    if (__ldg(t + lo + half) < v) { lo += half + 1; len -= half + 1; } else { len = half; }
  }
  return lo;
}
__device__ __forceinline__ int upper_bound_u32(const uint32_t* __restrict__ t, int n, uint32_t v) {
  int lo = 0, len = n;
  while (len > 0) {
    int half = len >> 1;
    if (__ldg(t + lo + half) <= v) { lo += half + 1; len -= half + 1; } else { len = half; }
  }
  return lo;
}

// Sum of squared byte differences of 4 words of q against one 16-byte vector.
__device__ __forceinline__ uint32_t sq4(const uint32_t* q, uint4 u, uint32_t acc) {
  uint32_t d;
  d = __vabsdiffu4(q[0], u.x); acc = __dp4a(d, d, acc);
  d = __vabsdiffu4(q[1], u.y); acc = __dp4a(d, d, acc);
  d = __vabsdiffu4(q[2], u.z); acc = __dp4a(d, d, acc);
  d = __vabsdiffu4(q[3], u.w); acc = __dp4a(d, d, acc);
  return acc;
}

template <int C>
__global__ void __launch_bounds__(kWarps * 32) k_sparse(SparseArgs a) {
  constexpr int D = 64 * C, NW = D / 4;
  constexpr int TROW = (TX + 7) * C;              // tile row bytes
  constexpr int TROWP = ((TROW + 8) + 3) & ~3;    // + room for the 8-byte funnel reads
  constexpr int KPW = NW + 1;                     // key-point row stride in words (odd: no bank conflicts)
  __shared__ __align__(16) uint8_t s_tile[(TY + 7) * TROWP];
  __shared__ uint32_t s_kp[kMaxK * KPW];
  __shared__ uint32_t s_lo[kWarps][kMaxK];
  __shared__ uint32_t s_hi[kWarps][kMaxK];
  __shared__ int32_t s_dense[TY * TX];
  __shared__ int s_next, s_ndense, s_dense_base;
  __shared__ unsigned long long s_stat[3];   // ring-answered queries, sum of seed sizes, sum of |S|

  const int K = a.K, n = a.n;
  const int tiles_x = (a.Wq + TX - 1) / TX;
  const int ty0 = (blockIdx.x / tiles_x) * TY;
  const int tx0 = (blockIdx.x % tiles_x) * TX;

  {
    const uint32_t* kp = reinterpret_cast<const uint32_t*>(a.KP);
    for (int i = threadIdx.x; i < K * NW; i += blockDim.x) s_kp[(i / NW) * KPW + (i % NW)] = kp[i];
    const int64_t rowb = (int64_t)a.W * C;
    for (int i = threadIdx.x; i < (TY + 7) * TROWP; i += blockDim.x) {
      const int r = i / TROWP, c = i % TROWP;
      const int y = ty0 + r;
      const int64_t xb = (int64_t)tx0 * C + c;
      s_tile[i] = (c < TROW && y < a.H && xb < rowb) ? a.frame[(int64_t)y * rowb + xb] : (uint8_t)0;
    }
    if (threadIdx.x == 0) { s_next = 0; s_ndense = 0; s_stat[0] = s_stat[1] = s_stat[2] = 0; }
  }
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t p2 = (uint32_t)(a.alpha_num * a.alpha_num);
  const uint32_t q2 = (uint32_t)(a.alpha_den * a.alpha_den);
  const float alpha = (float)a.alpha_num / (float)a.alpha_den;
  const uint32_t Amax = max_sqdist(D);

  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(&s_next, 1);
    t = __shfl_sync(kFull, t, 0);
    if (t >= TY * TX) break;
    const int ly = t / TX, lx = t % TX;
    const int y = ty0 + ly, x = tx0 + lx;
    if (y >= a.Hq || x >= a.Wq) continue;
    const int64_t qi = (int64_t)y * a.Wq + x;

    // a1: the query patch, 4 bytes per register, (dy, dx, c) order
    uint32_t q[NW];
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      const int dy = w / (2 * C), j = w % (2 * C);
      const int off = (ly + dy) * TROWP + lx * C + 4 * j;
      const int al = off & ~3;
      const uint32_t lo = *reinterpret_cast<const uint32_t*>(s_tile + al);
      const uint32_t hi = *reinterpret_cast<const uint32_t*>(s_tile + al + 4);
      q[w] = __funnelshift_r(lo, hi, (off & 3) * 8);
    }

    // previous match r_p and temporal change C = ||q - r_p||^2 (Alg. 1: r_i, d_i)
    const int rp = __ldg(a.prev + qi);
    if ((unsigned)rp >= (unsigned)n) {
      if (lane == 0) {
        atomicOr(a.status, RIANN_DEV_BAD_PREV);
        a.out_annf[qi] = -1;
        if (a.out_dist) a.out_dist[qi] = 0xffffffffu;
        if (a.out_count) a.out_count[qi] = 0u;
      }
      continue;
    }
    uint32_t Cd = 0;
    {
      const uint4* r4 = reinterpret_cast<const uint4*>(a.R + (int64_t)rp * D);
#pragma unroll
      for (int v = 0; v < NW / 4; ++v) Cd = sq4(q + 4 * v, __ldg(r4 + v), Cd);
    }

    // a2: per ring, B_m = ||q - k_m||^2, exact bounds [lo, hi] on A, and the
    // ring's run [jl, jh) in the sorted list of key m (two binary searches).
    unsigned long long seedkey = ~0ull;
    int jl[2] = {0, 0}, jh[2] = {0, 0};
    const float sC = (float)Cd;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int m = lane + 32 * h;
      if (m < K) {
        const uint32_t* kp = s_kp + m * KPW;
        uint32_t B = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          const uint32_t d = __vabsdiffu4(q[w], kp[w]);
          B = __dp4a(d, d, B);
        }
        const float cross = 2.f * alpha * sqrtf((float)B * sC);
        const float base = (float)B + alpha * alpha * sC;
        const uint32_t lo = ring_low(B, Cd, p2, q2, base - cross);
        const uint32_t hi = ring_high(B, Cd, p2, q2, base + cross, Amax);
        s_lo[warp][m] = lo;
        s_hi[warp][m] = hi;
        const uint32_t* ta = a.TA + (int64_t)m * n;
        jl[h] = lower_bound_u32(ta, n, lo);
        jh[h] = upper_bound_u32(ta, n, hi);
        const unsigned long long key =
            ((unsigned long long)(uint32_t)(jh[h] - jl[h]) << 32) | (unsigned)m;
        seedkey = key < seedkey ? key : seedkey;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long v = __shfl_xor_sync(kFull, seedkey, o);
      seedkey = v < seedkey ? v : seedkey;
    }
    const uint32_t nseed = (uint32_t)(seedkey >> 32);
    const int ms = (int)(seedkey & 0xffffffffu);
    const int jlo = __shfl_sync(kFull, (ms >> 5) ? jl[1] : jl[0], ms & 31);
    const int jhi = __shfl_sync(kFull, (ms >> 5) ? jh[1] : jh[0], ms & 31);
    __syncwarp();

    if (a.ring_limit >= 0 && nseed > (uint32_t)a.ring_limit) {
      // rings too wide: brute force over R, done by the dense path afterwards
      if (lane == 0) s_dense[atomicAdd(&s_ndense, 1)] = (int32_t)qi;
      continue;
    }

    // a3 + a4: enumerate the seed ring, keep references inside every other
    // ring, verify survivors by full distance; r_p is always a candidate.
    unsigned long long best = lane == 0 ? (((unsigned long long)Cd << 32) | (unsigned)rp) : ~0ull;
    uint32_t cnt = 0;
    const int32_t* tid = a.Tid + (int64_t)ms * n;
    for (int j = jlo + lane; j < jhi; j += 32) {
      const int r = __ldg(tid + j);
      const uint32_t* pr = a.P + (int64_t)r * K;
      bool ok = true;
      for (int m = 0; m < K; ++m) {
        if (m == ms) continue;
        const uint32_t v = __ldg(pr + m);
        if (v < s_lo[warp][m] || v > s_hi[warp][m]) { ok = false; break; }
      }
      if (ok) {
        ++cnt;
        const uint4* r4 = reinterpret_cast<const uint4*>(a.R + (int64_t)r * D);
        uint32_t d = 0;
#pragma unroll
        for (int v = 0; v < NW / 4; ++v) d = sq4(q + 4 * v, __ldg(r4 + v), d);
        const unsigned long long key = ((unsigned long long)d << 32) | (unsigned)r;
        best = key < best ? key : best;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long v = __shfl_xor_sync(kFull, best, o);
      best = v < best ? v : best;
      cnt += __shfl_xor_sync(kFull, cnt, o);
    }
    if (lane == 0) {
      a.out_annf[qi] = (int32_t)(best & 0xffffffffu);
      if (a.out_dist) a.out_dist[qi] = (uint32_t)(best >> 32);
      if (a.out_count) a.out_count[qi] = cnt;
      if (a.stats) {
        atomicAdd(&s_stat[0], 1ull);
        atomicAdd(&s_stat[1], (unsigned long long)nseed);
        atomicAdd(&s_stat[2], (unsigned long long)cnt);
      }
    }
    __syncwarp();
  }

  // hand the brute-force queries of this tile to the dense path
  __syncthreads();
  if (threadIdx.x == 0 && s_ndense > 0) s_dense_base = (int)atomicAdd(a.dense_count, (uint32_t)s_ndense);
  if (threadIdx.x == 0 && a.stats) {
    atomicAdd(&a.stats[kStatRingQueries], s_stat[0]);
    atomicAdd(&a.stats[kStatDenseQueries], (unsigned long long)s_ndense);
    atomicAdd(&a.stats[kStatSumSeed], s_stat[1]);
    atomicAdd(&a.stats[kStatSumS], s_stat[2]);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < s_ndense; i += blockDim.x) a.dense_list[s_dense_base + i] = s_dense[i];
}

}  // namespace

cudaError_t launch_sparse(const SparseArgs& a, int C, cudaStream_t s) {
  const int tiles = ((a.Hq + TY - 1) / TY) * ((a.Wq + TX - 1) / TX);
  if (C == 1) k_sparse<1><<<tiles, kWarps * 32, 0, s>>>(a);
  else k_sparse<3><<<tiles, kWarps * 32, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace riann
