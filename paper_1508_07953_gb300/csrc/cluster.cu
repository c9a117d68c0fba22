// cluster.cu -- reference-set construction (Sec. 3.4): the collected patches
// are clustered with a high-dimensional regression tree and every cluster is
// represented by its median.  Integer reading on uint8 patches:
//   * a node with more than `leaf` patches splits on its coordinate of
//     largest variance, cnt * sum(x^2) - sum(x)^2 (lowest coordinate on ties),
//     at that coordinate's lower median m (the value of rank (cnt-1)/2):
//     {x <= m} go left, or {x < m} when that would be every patch; both sides
//     keep their order;
//   * a node is a leaf when it holds at most `leaf` patches or no coordinate
//     varies; the leaves, left to right, are the clusters;
//   * a cluster's representative is its per-coordinate lower median.
//
// The tree is built level by level over one index array: every node is a
// contiguous range of it.  k_split (one CTA per node of the level) sums x and
// x^2 per coordinate, picks the coordinate, finds m from a 256-bin histogram
// (the values are bytes: no sort), and partitions its range stably with warp
// ballots into a scratch copy; the children go to the next level's node list.
// A leaf marks its first position.  Leaves are then enumerated in position
// order (block counts, a scan, ordered writes), and k_reps takes one warp per
// leaf: lower medians by ranking each coordinate's values across the lanes
// (small leaves) or by a binary search over the 256 byte values with ballot
// counts.
#include <algorithm>

#include "common.cuh"

namespace riann {
namespace {

// threads per node: 1024 while a level has fewer nodes than two per SM (the
// top levels, where a few large nodes would leave the GPU idle), else 256
// Coordinate sums of the few large nodes of a top level, spread over many
// CTAs: CTA (node, c) sums slice c of the node into 64-bit atomics.
template <int D>
__global__ void __launch_bounds__(256) k_node_sums(const uint8_t* __restrict__ X, const int32_t* __restrict__ perm,
                                                   const int2* __restrict__ segs, int leaf,
                                                   unsigned long long* __restrict__ gsum) {
  constexpr int G = 256 / D;
  __shared__ unsigned long long s1[D], s2[D];
  const int2 sg = segs[blockIdx.x];
  const int b = sg.x, cnt = sg.y - sg.x, tid = threadIdx.x;
  if (cnt <= leaf) return;   // k_split makes it a leaf without the sums
  const int per = (cnt + gridDim.y - 1) / gridDim.y;
  const int lo = blockIdx.y * per, hi = min(cnt, lo + per);
  if (lo >= hi) return;
  for (int i = tid; i < D; i += blockDim.x) s1[i] = s2[i] = 0ull;
  __syncthreads();
  if (tid < G * D) {
    const int g = tid / D, d = tid % D;
    unsigned long long a1 = 0, a2 = 0;
    for (int i = lo + g; i < hi; i += G) {
      const unsigned x = __ldg(X + (int64_t)perm[b + i] * D + d);
      a1 += x;
      a2 += x * x;
    }
    atomicAdd(&s1[d], a1);
    atomicAdd(&s2[d], a2);
  }
  __syncthreads();
  unsigned long long* out = gsum + (size_t)blockIdx.x * 2 * D;
  for (int i = tid; i < D; i += blockDim.x) {
    atomicAdd(out + i, s1[i]);
    atomicAdd(out + D + i, s2[i]);
  }
}

// gsum (nullable): the node's coordinate sums, already computed by k_node_sums
template <int D, int T>
__global__ void __launch_bounds__(T) k_split(const uint8_t* __restrict__ X, int32_t* perm,
                                                         int32_t* tmp, uint8_t* leaf_start,
                                                         const int2* __restrict__ segs_in, int2* segs_out,
                                                         uint32_t* n_out, int leaf,
                                                         const unsigned long long* __restrict__ gsum) {
  constexpr int G = T / D;   // threads per coordinate in the sums
  __shared__ unsigned long long s1[D], s2[D];
  __shared__ uint32_t hist[256];
  __shared__ int s_dim, s_m, s_strict, s_nl;
  __shared__ uint32_t s_wl[T / 32], s_wr[T / 32];
  const int2 sg = segs_in[blockIdx.x];
  const int b = sg.x, e = sg.y, cnt = e - b;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (cnt <= leaf) {
    if (tid == 0) leaf_start[b] = 1;
    return;
  }
  for (int i = tid; i < 256; i += blockDim.x) hist[i] = 0u;
  if (gsum) {
    const unsigned long long* src = gsum + (size_t)blockIdx.x * 2 * D;
    for (int i = tid; i < D; i += blockDim.x) {
      s1[i] = src[i];
      s2[i] = src[D + i];
    }
    __syncthreads();
  } else {
    for (int i = tid; i < D; i += blockDim.x) s1[i] = s2[i] = 0ull;
    __syncthreads();
    if (tid < G * D) {
      const int g = tid / D, d = tid % D;
      unsigned long long a1 = 0, a2 = 0;
      for (int i = g; i < cnt; i += G) {
        const unsigned x = __ldg(X + (int64_t)perm[b + i] * D + d);
        a1 += x;
        a2 += x * x;
      }
      atomicAdd(&s1[d], a1);
      atomicAdd(&s2[d], a2);
    }
  }
  __syncthreads();
  if (warp == 0) {
    unsigned long long bv = 0;
    int bd = D;
    for (int d = lane; d < D; d += 32) {
      const unsigned long long v = (unsigned long long)cnt * s2[d] - s1[d] * s1[d];
      if (v > bv) {   // ascending d per lane: keeps the lowest on ties
        bv = v;
        bd = d;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int od = __shfl_xor_sync(0xffffffffu, bd, o);
      if (ov > bv || (ov == bv && od < bd)) {
        bv = ov;
        bd = od;
      }
    }
    if (lane == 0) s_dim = bv ? bd : -1;
  }
  __syncthreads();
  const int d = s_dim;
  if (d < 0) {   // no coordinate varies
    if (tid == 0) leaf_start[b] = 1;
    return;
  }
  for (int i = tid; i < cnt; i += blockDim.x) atomicAdd(&hist[__ldg(X + (int64_t)perm[b + i] * D + d)], 1u);
  __syncthreads();
  if (tid == 0) {
    const uint32_t r = (uint32_t)(cnt - 1) / 2;
    uint32_t cum = 0;
    int m = 0;
    for (; m < 256; ++m) {
      cum += hist[m];
      if (cum > r) break;
    }
    const int strict = cum == (uint32_t)cnt;   // everything <= m: the values below m split off
    const int nl = strict ? (int)(cum - hist[m]) : (int)cum;
    s_m = m;
    s_strict = strict;
    // both sides are non-empty whenever the coordinate varies; a split that
    // would leave one empty is never made
    s_nl = (nl == 0 || nl == cnt) ? -1 : nl;
  }
  __syncthreads();
  const int m = s_m, strict = s_strict, nl = s_nl;
  if (nl < 0) {
    if (tid == 0) leaf_start[b] = 1;
    return;
  }
  // stable partition into tmp[b, e), then back into perm
  int lbase = 0, rbase = 0;
  for (int c0 = 0; c0 < cnt; c0 += blockDim.x) {
    const int i = c0 + tid;
    const bool valid = i < cnt;
    const int32_t p = valid ? perm[b + i] : 0;
    const int x = valid ? (int)__ldg(X + (int64_t)p * D + d) : 0;
    const bool left = valid && (strict ? x < m : x <= m);
    const bool right = valid && !left;
    const unsigned bl = __ballot_sync(0xffffffffu, left), br = __ballot_sync(0xffffffffu, right);
    const unsigned lt = (1u << lane) - 1u;
    if (lane == 0) {
      s_wl[warp] = __popc(bl);
      s_wr[warp] = __popc(br);
    }
    __syncthreads();
    int offl = 0, offr = 0, totl = 0, totr = 0;
#pragma unroll
    for (int w = 0; w < T / 32; ++w) {
      const int a = (int)s_wl[w], c = (int)s_wr[w];
      if (w < warp) {
        offl += a;
        offr += c;
      }
      totl += a;
      totr += c;
    }
    if (left) tmp[b + lbase + offl + __popc(bl & lt)] = p;
    if (right) tmp[b + nl + rbase + offr + __popc(br & lt)] = p;
    lbase += totl;
    rbase += totr;
    __syncthreads();   // s_wl / s_wr are rewritten by the next chunk
  }
  for (int i = tid; i < cnt; i += blockDim.x) perm[b + i] = tmp[b + i];
  if (tid == 0) {
    const uint32_t k = atomicAdd(n_out, 2u);
    segs_out[k] = make_int2(b, b + nl);
    segs_out[k + 1] = make_int2(b + nl, e);
  }
}

// Leaves in position order: leaf_begin[k] = first position of leaf k, *count
// = leaves.  Three steps over blocks of 1024 positions: each block counts its
// leaf starts, one CTA scans the block counts, each block writes its starts
// at its offset (ballots and a shared scan keep them in order).
constexpr int kScanBlock = 1024;

__global__ void __launch_bounds__(kScanBlock) k_leaf_count(const uint8_t* __restrict__ leaf_start, int n,
                                                           uint32_t* __restrict__ block_count) {
  const int i = blockIdx.x * kScanBlock + threadIdx.x;
  const int c = __syncthreads_count(i < n && leaf_start[i]);
  if (threadIdx.x == 0) block_count[blockIdx.x] = (uint32_t)c;
}

__global__ void __launch_bounds__(kScanBlock) k_leaf_offsets(uint32_t* block_count, int nb, uint32_t* count) {
  __shared__ uint32_t s_w[kScanBlock / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t base = 0;
  for (int c0 = 0; c0 < nb; c0 += kScanBlock) {
    const int i = c0 + tid;
    const uint32_t v = i < nb ? block_count[i] : 0u;
    uint32_t x = v;   // inclusive warp scan
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    uint32_t off = 0, tot = 0;
    for (int w = 0; w < kScanBlock / 32; ++w) {
      if (w < warp) off += s_w[w];
      tot += s_w[w];
    }
    if (i < nb) block_count[i] = base + off + x - v;   // exclusive offset, in place
    base += tot;
    __syncthreads();
  }
  if (tid == 0) *count = base;
}

__global__ void __launch_bounds__(kScanBlock) k_leaf_write(const uint8_t* __restrict__ leaf_start, int n,
                                                           const uint32_t* __restrict__ block_off,
                                                           int32_t* __restrict__ leaf_begin) {
  __shared__ uint32_t s_w[kScanBlock / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i = blockIdx.x * kScanBlock + tid;
  const bool f = i < n && leaf_start[i];
  const unsigned bal = __ballot_sync(0xffffffffu, f);
  if (lane == 0) s_w[warp] = __popc(bal);
  __syncthreads();
  uint32_t off = block_off[blockIdx.x];
  for (int w = 0; w < warp; ++w) off += s_w[w];
  if (f) leaf_begin[off + __popc(bal & ((1u << lane) - 1u))] = i;
}

// One warp per leaf: its members' cluster id and its per-coordinate lower median.
constexpr int kSmallLeaf = 8;   // leaves up to this size rank their values per coordinate
template <int D>
__global__ void __launch_bounds__(256) k_reps(const uint8_t* __restrict__ X, const int32_t* __restrict__ perm,
                                              const int32_t* __restrict__ leaf_begin, const uint32_t* count,
                                              int n, uint8_t* reps, int32_t* assign) {
  const int lane = threadIdx.x & 31;
  const int L = (int)*count;
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (k >= L) return;
  const int start = leaf_begin[k], end = k + 1 < L ? leaf_begin[k + 1] : n, cnt = end - start;
  if (assign)
    for (int i = lane; i < cnt; i += 32) assign[perm[start + i]] = k;
  const int r = (cnt - 1) / 2;
  if (cnt <= kSmallLeaf) {
    // small leaf: lanes on coordinates; each lane ranks the leaf's values of
    // its coordinates (value, then member order) and keeps the one of rank r
    int32_t pm[kSmallLeaf];
#pragma unroll
    for (int j = 0; j < kSmallLeaf; ++j) pm[j] = j < cnt ? perm[start + j] : 0;
    for (int d = lane; d < D; d += 32) {
      int v[kSmallLeaf];
#pragma unroll
      for (int j = 0; j < kSmallLeaf; ++j) v[j] = j < cnt ? (int)__ldg(X + (int64_t)pm[j] * D + d) : 0;
      int med = 0;
#pragma unroll
      for (int j = 0; j < kSmallLeaf; ++j) {
        int rank = 0;
#pragma unroll
        for (int i = 0; i < kSmallLeaf; ++i)
          rank += (i < cnt) && (v[i] < v[j] || (v[i] == v[j] && i < j));
        if (j < cnt && rank == r) med = v[j];
      }
      reps[(int64_t)k * D + d] = (uint8_t)med;
    }
    return;
  }
  const int32_t p0 = lane < cnt ? perm[start + lane] : 0;   // the first 32 members, kept in a register
  for (int d = 0; d < D; ++d) {
    const int x0 = lane < cnt ? (int)__ldg(X + (int64_t)p0 * D + d) : 256;
    int lo = 0, hi = 255;
    while (lo < hi) {   // smallest v with #{x <= v} > r
      const int mid = (lo + hi) >> 1;
      int c = __popc(__ballot_sync(0xffffffffu, x0 <= mid));
      for (int i = 32; i < cnt; i += 32) {                      // members past the first 32
        const int j = i + lane;
        const int x = j < cnt ? (int)__ldg(X + (int64_t)perm[start + j] * D + d) : 256;
        c += __popc(__ballot_sync(0xffffffffu, x <= mid));
      }
      if (c > r) hi = mid;
      else lo = mid + 1;
    }
    if (lane == 0) reps[(int64_t)k * D + d] = (uint8_t)lo;
  }
}

__global__ void k_iota(int32_t* p, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = i;
}

template <int D>
cudaError_t run_tree(const uint8_t* X, int n, int leaf, int32_t* perm, int32_t* tmp, uint8_t* leaf_start,
                     int2* segs0, int2* segs1, uint32_t* cnts, int32_t* leaf_begin, uint8_t* reps, int32_t* assign,
                     int32_t* out_count, unsigned long long* gsum, cudaStream_t s) {
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 8);
  k_iota<<<blocks, 256, 0, s>>>(perm, n);
  cudaError_t e = cudaMemsetAsync(leaf_start, 0, (size_t)n, s);
  const int2 root = make_int2(0, n);
  if (e == cudaSuccess) e = cudaMemcpyAsync(segs0, &root, sizeof(int2), cudaMemcpyHostToDevice, s);
  int2* in = segs0;
  int2* out = segs1;
  uint32_t nseg = 1;
  while (e == cudaSuccess && nseg > 0) {
    e = cudaMemsetAsync(cnts, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) break;
    const uint32_t few = 2u * (uint32_t)sm_count();   // gsum holds this many nodes
    if (nseg < few) {
      // top levels: the sums over many CTAs, then one 1024-thread CTA per node
      e = cudaMemsetAsync(gsum, 0, sizeof(unsigned long long) * 2 * D * nseg, s);
      if (e != cudaSuccess) break;
      const unsigned slices = (4u * (uint32_t)sm_count() + nseg - 1) / nseg;
      k_node_sums<D><<<dim3(nseg, slices), 256, 0, s>>>(X, perm, in, leaf, gsum);
      k_split<D, 1024><<<nseg, 1024, 0, s>>>(X, perm, tmp, leaf_start, in, out, cnts, leaf, gsum);
    } else {
      k_split<D, 256><<<nseg, 256, 0, s>>>(X, perm, tmp, leaf_start, in, out, cnts, leaf, nullptr);
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nseg, cnts, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    std::swap(in, out);
  }
  if (e != cudaSuccess) return e;
  const int nb = (n + kScanBlock - 1) / kScanBlock;
  uint32_t* block_count = reinterpret_cast<uint32_t*>(segs0);   // the node lists are free now
  k_leaf_count<<<nb, kScanBlock, 0, s>>>(leaf_start, n, block_count);
  k_leaf_offsets<<<1, kScanBlock, 0, s>>>(block_count, nb, cnts + 1);
  k_leaf_write<<<nb, kScanBlock, 0, s>>>(leaf_start, n, block_count, leaf_begin);
  uint32_t L = 0;
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&L, cnts + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  k_reps<D><<<(L + 7) / 8, 256, 0, s>>>(X, perm, leaf_begin, cnts + 1, n, reps, assign);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  *out_count = (int32_t)L;
  return e;
}

}  // namespace

cudaError_t cluster_references(const uint8_t* X, int n, int C, int leaf, uint8_t* reps, int32_t* assign,
                               int32_t* out_count, cudaStream_t s) {
  // scratch from the stream-ordered pool: repeated calls reuse it without a
  // device-wide allocation or free
  int32_t *perm = nullptr, *tmp = nullptr, *leaf_begin = nullptr;
  uint8_t* leaf_start = nullptr;
  int2 *segs0 = nullptr, *segs1 = nullptr;
  uint32_t* cnts = nullptr;
  unsigned long long* gsum = nullptr;   // coordinate sums of a top level's nodes
  cudaError_t e = cudaMallocAsync((void**)&perm, sizeof(int32_t) * (size_t)n, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&tmp, sizeof(int32_t) * (size_t)n, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&leaf_begin, sizeof(int32_t) * (size_t)n, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&leaf_start, (size_t)n, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&segs0, sizeof(int2) * (size_t)n, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&segs1, sizeof(int2) * (size_t)n, s);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&cnts, sizeof(uint32_t) * 2, s);
  if (e == cudaSuccess)
    e = cudaMallocAsync((void**)&gsum, sizeof(unsigned long long) * 2 * 192 * 2 * (size_t)sm_count(), s);
  if (e == cudaSuccess)
    e = C == 1 ? run_tree<64>(X, n, leaf, perm, tmp, leaf_start, segs0, segs1, cnts, leaf_begin, reps, assign,
                              out_count, gsum, s)
               : run_tree<192>(X, n, leaf, perm, tmp, leaf_start, segs0, segs1, cnts, leaf_begin, reps, assign,
                               out_count, gsum, s);
  if (e != cudaSuccess) cudaGetLastError();
  for (void* p : {(void*)perm, (void*)tmp, (void*)leaf_begin, (void*)leaf_start, (void*)segs0, (void*)segs1,
                  (void*)cnts, (void*)gsum})
    if (p) cudaFreeAsync(p, s);
  const cudaError_t e2 = cudaStreamSynchronize(s);
  return e != cudaSuccess ? e : e2;
}

}  // namespace riann
