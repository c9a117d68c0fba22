// anchor.cu -- Alg. 1 as the paper writes it: a first ring around the previous
// match r_i, then rings around anchors drawn at random from the candidate set,
// until fewer than L candidates remain (Sec. 3.2, Alg. 1), with the rings read
// from the sorted distance matrix of Sec. 3.3 / 3.4.
//
// The matrix: row i holds every reference as a 64-bit key
// (||r_i - r_id||^2 << 32) | id, ascending, so a ring around r_i is one
// contiguous range of row i, found by two searches.  Later rings are tested on
// the candidates, which leaves the order of the candidate list unchanged:
// either by one distance each or, when the anchor's own ring (a range of its
// row) holds no more references than there are candidates and n <= 65536, by
// marking that range in a per-warp bitmap and testing one bit per candidate --
// the same set, since the range holds exactly the references with A in the
// ring's bounds.  (Marking a larger ring costs more than the distances.)
//
// One warp per query in a persistent launch (queries from an atomic counter:
// their cost varies by orders of magnitude).  Ring test for anchor a with
// d_a^2 = B = ||q - a||^2 and alpha = p/q, in integers:
//     (q - p)^2 B <= q^2 ||a - r||^2   (when p < q)   and   q^2 ||a - r||^2 <= (q + p)^2 B.
// The anchor of ring t is the candidate at position (x * |S|) >> 32, x the
// first word of Philox4x32-10 (Salmon et al., SC'11) with counter
// (query index, t, frame id, 0) and the caller's key.  The answer is the
// minimum of (||q - r||^2, r) over the final candidates, r_i and the anchors.
#include "anchor.cuh"

namespace riann {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// squared L2 of two D-byte rows read 16 bytes at a time
template <int NW>
__device__ __forceinline__ uint32_t row_sqdist(const uint4* a, const uint4* b) {
  uint32_t s = 0;
#pragma unroll
  for (int v = 0; v < NW / 4; ++v) {
    const uint4 x = a[v], y = b[v];
    uint32_t d;
    d = __vabsdiffu4(x.x, y.x); s = __dp4a(d, d, s);
    d = __vabsdiffu4(x.y, y.y); s = __dp4a(d, d, s);
    d = __vabsdiffu4(x.z, y.z); s = __dp4a(d, d, s);
    d = __vabsdiffu4(x.w, y.w); s = __dp4a(d, d, s);
  }
  return s;
}

template <int C>
__global__ void k_full_keys(const uint8_t* __restrict__ R, int n, int NP, int64_t row0,
                            unsigned long long* __restrict__ T) {
  constexpr int D = 64 * C;
  const int64_t i = row0 + blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= NP) return;
  unsigned long long key = ~0ull;
  if (j < n) {
    const uint32_t A = row_sqdist<D / 4>(reinterpret_cast<const uint4*>(R + i * D),
                                         reinterpret_cast<const uint4*>(R + (int64_t)j * D));
    key = ((unsigned long long)A << 32) | (unsigned)j;
  }
  T[i * NP + j] = key;
}

__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                              uint32_t k1, uint32_t* out0) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  *out0 = c0;
}

__device__ __forceinline__ bool in_anchor_ring(uint32_t A, uint32_t B, uint32_t p, uint32_t q) {
  const unsigned long long qq = (unsigned long long)q * q, a = qq * A;
  if (p < q && (unsigned long long)(q - p) * (q - p) * B > a) return false;
  return a <= (unsigned long long)(q + p) * (q + p) * B;
}

// First position in row[0, n) whose key is >= x (the warp searches together:
// every round splits the range in 33 parts, one probe per lane).
__device__ __forceinline__ int warp_lower_bound(const unsigned long long* __restrict__ row, int n,
                                                unsigned long long x, int lane) {
  int lo = 0, hi = n;   // answer in [lo, hi]
  while (hi - lo > 0) {
    const int len = hi - lo;
    const int step = (len + 32) / 33;
    const int pos = lo + (lane + 1) * step - 1;
    const bool below = pos < hi && __ldg(row + pos) < x;   // keys before the answer
    const unsigned b = __ballot_sync(kFull, below);
    const int c = __popc(b);                       // probes below x (a prefix of the lanes)
    const int nlo = c ? lo + c * step : lo;
    const int nhi = c < 32 ? min(hi, lo + (c + 1) * step - 1) : hi;
    lo = nlo;
    hi = nhi;
  }
  return lo;
}

template <int C>
__global__ void __launch_bounds__(kAnchorWarps * 32, kAnchorCtasPerSm) k_anchor(const __grid_constant__ AnchorArgs a) {
  constexpr int D = 64 * C, NW = D / 4;
  __shared__ __align__(16) uint32_t s_q[kAnchorWarps][NW];   // the query patch
  __shared__ __align__(16) uint32_t s_a[kAnchorWarps][NW];   // the current anchor's row
  __shared__ uint32_t s_bits[kAnchorWarps][kAnchorBitmapN / 32];   // members of an anchor's ring
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* bits = s_bits[warp];
  for (int w = lane; w < kAnchorBitmapN / 32; w += 32) bits[w] = 0u;   // kept all-zero between rings
  __syncwarp();
  const int Wq = a.W - 7;
  const int64_t Q = (int64_t)(a.H - 7) * Wq;
  const uint32_t p = (uint32_t)a.alpha_num, qa = (uint32_t)a.alpha_den;
  const unsigned below_mask = (1u << lane) - 1u;
  int32_t* buf[2];
  buf[0] = a.scratch + ((int64_t)blockIdx.x * kAnchorWarps + warp) * 2 * a.n;
  buf[1] = buf[0] + a.n;
  const uint4* q4 = reinterpret_cast<const uint4*>(s_q[warp]);
  const uint4* a4 = reinterpret_cast<const uint4*>(s_a[warp]);

  for (;;) {
    int64_t qi = 0;
    if (lane == 0) qi = atomicAdd(a.counter, 1u);
    qi = __shfl_sync(kFull, qi, 0);
    if (qi >= Q) break;
    const int y = (int)(qi / Wq), x = (int)(qi % Wq);
    for (int w = lane; w < NW; w += 32) {          // 4 bytes of (dy, dx, c) order per word
      const int dy = w / (2 * C), j = w % (2 * C);
      const uint8_t* src = a.frame + ((int64_t)(y + dy) * a.W + x) * C + 4 * j;
      s_q[warp][w] = (uint32_t)src[0] | ((uint32_t)src[1] << 8) | ((uint32_t)src[2] << 16) | ((uint32_t)src[3] << 24);
    }
    __syncwarp();
    const int ri = __ldg(a.prev + qi);
    if ((unsigned)ri >= (unsigned)a.n) {
      if (lane == 0) {
        atomicOr(a.status, RIANN_DEV_BAD_PREV);
        a.out_annf[qi] = -1;
        if (a.out_dist) a.out_dist[qi] = 0xffffffffu;
        if (a.out_count) a.out_count[qi] = 0u;
        if (a.out_rings) a.out_rings[qi] = 0u;
      }
      continue;
    }
    const uint32_t Bi = row_sqdist<NW>(q4, reinterpret_cast<const uint4*>(a.R + (int64_t)ri * D));
    unsigned long long best = ((unsigned long long)Bi << 32) | (unsigned)ri;

    // S_0: the ring of r_i = keys of row r_i with A in [ceil((q-p)^2 B / q^2), floor((q+p)^2 B / q^2)]
    const unsigned long long* row = a.T + (int64_t)ri * a.NP;
    const unsigned long long qq = (unsigned long long)qa * qa;
    const unsigned long long amin = p < qa ? ((unsigned long long)(qa - p) * (qa - p) * Bi + qq - 1) / qq : 0ull;
    const unsigned long long amax = (unsigned long long)(qa + p) * (qa + p) * Bi / qq;
    const int lo = warp_lower_bound(row, a.n, amin << 32, lane);
    const int hi = amax >= 0xffffffffull ? a.n : warp_lower_bound(row, a.n, (amax + 1) << 32, lane);
    int ns = hi > lo ? hi - lo : 0;
    const int ns0 = ns;
    unsigned long long tests = 0;
    const int32_t* src = nullptr;                   // t = 0: the range of row r_i; then a scratch list
    uint32_t t = 0;
    while (ns >= a.L && (int)t < a.max_rings) {
      uint32_t xr;
      philox4x32_10((uint32_t)qi, t, a.frame_id, 0u, a.key0, a.key1, &xr);
      const int idx = (int)(((unsigned long long)xr * (unsigned)ns) >> 32);
      int ra = src ? src[idx] : (int)(uint32_t)__ldg(row + lo + idx);
      if (!RIANN_IN_RANGE((unsigned)ra < (unsigned)a.n, a.status)) ra = ri;
      const uint4* ra4 = reinterpret_cast<const uint4*>(a.R + (int64_t)ra * D);
      for (int w = lane; w < NW / 4; w += 32) reinterpret_cast<uint4*>(s_a[warp])[w] = __ldg(ra4 + w);
      __syncwarp();
      const uint32_t Ba = row_sqdist<NW>(q4, a4);
      const unsigned long long ka = ((unsigned long long)Ba << 32) | (unsigned)ra;
      best = ka < best ? ka : best;
      int32_t* dst = buf[t & 1];
      tests += (unsigned long long)ns;
      // the anchor's ring as a range [alo, ahi) of its own row
      int alo = 0, ahi = 0;
      bool use_bits = false;
      const unsigned long long* arow = a.T + (int64_t)ra * a.NP;
      if (a.n <= kAnchorBitmapN) {
        const unsigned long long bmin = p < qa ? ((unsigned long long)(qa - p) * (qa - p) * Ba + qq - 1) / qq : 0ull;
        const unsigned long long bmax = (unsigned long long)(qa + p) * (qa + p) * Ba / qq;
        alo = warp_lower_bound(arow, a.n, bmin << 32, lane);
        ahi = bmax >= 0xffffffffull ? a.n : warp_lower_bound(arow, a.n, (bmax + 1) << 32, lane);
        use_bits = ahi - alo <= ns;
        if (use_bits) {
          for (int k = alo + lane; k < ahi; k += 32) {
            const uint32_t id = (uint32_t)__ldg(arow + k);
            if (RIANN_IN_RANGE(id < (uint32_t)a.n, a.status)) atomicOr(bits + (id >> 5), 1u << (id & 31));
          }
          __syncwarp();
        }
      }
      int m = 0;
      for (int base = 0; base < ns; base += 32) {
        const int k = base + lane;
        bool keep = false;
        int rj = 0;
        if (k < ns) {
          rj = src ? src[k] : (int)(uint32_t)__ldg(row + lo + k);
          if (!RIANN_IN_RANGE((unsigned)rj < (unsigned)a.n, a.status)) {
            rj = ri;
          } else if (use_bits) {
            keep = (bits[rj >> 5] >> (rj & 31)) & 1u;
          } else {
            const uint32_t A = row_sqdist<NW>(a4, reinterpret_cast<const uint4*>(a.R + (int64_t)rj * D));
            keep = in_anchor_ring(A, Ba, p, qa);
          }
        }
        const unsigned bal = __ballot_sync(kFull, keep);
        if (keep) dst[m + __popc(bal & below_mask)] = rj;   // order kept
        m += __popc(bal);
      }
      __syncwarp();
      if (use_bits) {   // back to all-zero
        for (int k = alo + lane; k < ahi; k += 32) {
          const uint32_t id = (uint32_t)__ldg(arow + k);
          if (id < (uint32_t)a.n) bits[id >> 5] = 0u;
        }
        __syncwarp();
      }
      src = dst;
      ns = m;
      ++t;
    }
    // the final candidates
    for (int base = 0; base < ns; base += 32) {
      const int k = base + lane;
      if (k < ns) {
        int rj = src ? src[k] : (int)(uint32_t)__ldg(row + lo + k);
        if (!RIANN_IN_RANGE((unsigned)rj < (unsigned)a.n, a.status)) rj = ri;
        const uint32_t d = row_sqdist<NW>(q4, reinterpret_cast<const uint4*>(a.R + (int64_t)rj * D));
        const unsigned long long kk = ((unsigned long long)d << 32) | (unsigned)rj;
        best = kk < best ? kk : best;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long v = __shfl_xor_sync(kFull, best, o);
      best = v < best ? v : best;
    }
    if (lane == 0) {
      a.out_annf[qi] = (int32_t)(best & 0xffffffffu);
      if (a.out_dist) a.out_dist[qi] = (uint32_t)(best >> 32);
      if (a.out_count) a.out_count[qi] = (uint32_t)ns;
      if (a.out_rings) a.out_rings[qi] = t;
      if (a.work) {
        atomicAdd(a.work, (unsigned long long)ns0);
        atomicAdd(a.work + 1, tests);
        atomicAdd(a.work + 2, (unsigned long long)ns);
      }
    }
    __syncwarp();
  }
}

// Alg. 1's random initial field: entry q = (x * n) >> 32, x from Philox4x32-10 with counter (q, 0, frame id, 1).
__global__ void k_random_field(int64_t Q, int n, uint32_t key0, uint32_t key1, uint32_t frame_id, int32_t* out) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < Q; q += (int64_t)gridDim.x * blockDim.x) {
    uint32_t x;
    philox4x32_10((uint32_t)q, 0u, frame_id, 1u, key0, key1, &x);
    out[q] = (int32_t)(((unsigned long long)x * (unsigned)n) >> 32);
  }
}

__global__ void k_fill_u32(uint32_t* p, int64_t count, uint32_t v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

}  // namespace

int full_table_stride(int n) {
  int NP = sort_chunk();
  while (NP < n) NP <<= 1;
  return NP;
}

cudaError_t build_full_table(const Index& ix, unsigned long long* T, int NP, cudaStream_t s) {
  for (int64_t r0 = 0; r0 < ix.n; r0 += 32768) {
    const int nr = (int)(ix.n - r0 < 32768 ? ix.n - r0 : 32768);
    const dim3 grid((unsigned)((NP + 255) / 256), (unsigned)nr);
    if (ix.C == 1) k_full_keys<1><<<grid, 256, 0, s>>>(ix.R, ix.n, NP, r0, T);
    else k_full_keys<3><<<grid, 256, 0, s>>>(ix.R, ix.n, NP, r0, T);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return sort_segments(T, NP, ix.n, s);
}

int anchor_resident_warps() { return kAnchorCtasPerSm * sm_count() * kAnchorWarps; }

cudaError_t launch_anchor(const AnchorArgs& a, int C, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(uint32_t), s);
  if (e == cudaSuccess && a.work) e = cudaMemsetAsync(a.work, 0, 3 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const int grid = kAnchorCtasPerSm * sm_count();
  if (C == 1) k_anchor<1><<<grid, kAnchorWarps * 32, 0, s>>>(a);
  else k_anchor<3><<<grid, kAnchorWarps * 32, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_random_field(int64_t Q, int n, uint64_t seed, uint32_t frame_id, int32_t* out, cudaStream_t s) {
  if (Q <= 0) return cudaSuccess;
  int64_t blocks = (Q + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_random_field<<<(unsigned)blocks, 256, 0, s>>>(Q, n, (uint32_t)seed, (uint32_t)(seed >> 32), frame_id, out);
  return cudaGetLastError();
}

cudaError_t launch_fill_u32(uint32_t* p, int64_t count, uint32_t value, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  int64_t blocks = (count + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_fill_u32<<<(unsigned)blocks, 256, 0, s>>>(p, count, value);
  return cudaGetLastError();
}

}  // namespace riann
