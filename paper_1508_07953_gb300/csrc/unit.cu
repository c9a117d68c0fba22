// unit.cu -- unit-normalised float variant (Sec. 3.4 / Alg. 1: unit-length
// patches): the normalised tables of an index and its brute force.  The
// arithmetic (fixed-order IEEE fp32) is in unit.cuh.
#include "unit.cuh"

namespace riann {
namespace {

// rows of X (n x D bytes) scaled to length 1: one thread per row
__global__ void k_unit_normalize(const uint8_t* __restrict__ X, int n, int D, float* __restrict__ out) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const uint8_t* x = X + (int64_t)r * D;
  uint32_t s = 0;
  for (int i = 0; i < D; ++i) s += (uint32_t)x[i] * x[i];
  const float nv = unit_scale(s);
  float* o = out + (int64_t)r * D;
  for (int i = 0; i < D; ++i) o[i] = unit_coord(x[i], s, nv);
}

// P[r][m] = bits of d(k'_m, r'), row stride Kp, pad entries 0
template <int D>
__global__ void k_unit_key_distances(const float* __restrict__ Rf, const float* __restrict__ KPf, int n, int K,
                                     int Kp, uint32_t* __restrict__ P) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * Kp) return;
  const int r = (int)(t / Kp), m = (int)(t % Kp);
  P[t] = m < K ? __float_as_uint(unit_dist<D>(KPf + (int64_t)m * D, Rf + (int64_t)r * D)) : 0u;
}

// Brute force: argmin over all references of d(q', r'), lower index on ties.
// RGB (D = 192): a CTA takes 32 queries (one per thread, q' in shared memory,
// a column per query: conflict-free) and walks the references in tiles of 16
// staged in shared memory.  A reference whose running sum already exceeds
// the best one's cannot win (the root is monotone and a tie keeps the lower
// index), so the root is taken only for the others.  Gray has its own
// packed-pair kernel below.
constexpr int kUnitRgbQB = 32, kUnitRgbRT = 16;   // 24 KB of queries + 12 KB of tile

struct UnitDenseArgs {
  FrameItem one;
  const int32_t* list;
  const uint32_t* list_count;
  int64_t Q;
  const float* Rf;
  int n;
  unsigned long long* stats;
};

__global__ void __launch_bounds__(kUnitRgbQB) k_dense_unit_rgb(const UnitDenseArgs a) {
  constexpr int C = 3, D = 64 * C, QB = kUnitRgbQB, RT = kUnitRgbRT;
  __shared__ __align__(16) float s_r[RT][D];
  __shared__ float s_q[D][QB];
  const int64_t nq = a.list ? (int64_t)*a.list_count : a.Q;
  if (!a.list && a.stats && blockIdx.x == 0 && threadIdx.x == 0) a.stats[kStatDenseQueries] = (unsigned long long)nq;
  const int64_t i = (int64_t)blockIdx.x * QB + threadIdx.x;
  if ((int64_t)blockIdx.x * QB >= nq) return;   // uniform for the CTA
  const bool live = i < nq;
  const FrameItem& it = a.one;
  int64_t qi = 0;
  if (live) {
    qi = a.list ? (int64_t)a.list[i] - it.query_begin : i;
    const int y = (int)(qi / it.Wq), x = (int)(qi % it.Wq);
    uint32_t s = 0;
    for (int dy = 0; dy < 8; ++dy)
      for (int j = 0; j < 8 * C; ++j) {
        const uint32_t v = it.frame[((int64_t)(y + dy) * it.W + x) * C + j];
        s += v * v;
      }
    const float nv = unit_scale(s);
    for (int dy = 0; dy < 8; ++dy)
      for (int j = 0; j < 8 * C; ++j)
        s_q[dy * 8 * C + j][threadIdx.x] = unit_coord(it.frame[((int64_t)(y + dy) * it.W + x) * C + j], s, nv);
  }
  float bd = __int_as_float(0x7f800000), bacc = bd;
  int bi = 0;
  for (int r0 = 0; r0 < a.n; r0 += RT) {
    const int nt = min(RT, a.n - r0);
    __syncthreads();
    {
      const float4* src = reinterpret_cast<const float4*>(a.Rf + (int64_t)r0 * D);
      float4* dst = reinterpret_cast<float4*>(&s_r[0][0]);
      for (int k = threadIdx.x; k < nt * D / 4; k += QB) dst[k] = __ldg(src + k);
    }
    __syncthreads();
    if (!live) continue;
    for (int j = 0; j < nt; ++j) {
      const float4* r4 = reinterpret_cast<const float4*>(s_r[j]);
      float acc = 0.f;
#pragma unroll
      for (int v = 0; v < D / 4; ++v) {
        const float4 rv = r4[v];
        acc = unit_step(acc, s_q[4 * v + 0][threadIdx.x], rv.x);
        acc = unit_step(acc, s_q[4 * v + 1][threadIdx.x], rv.y);
        acc = unit_step(acc, s_q[4 * v + 2][threadIdx.x], rv.z);
        acc = unit_step(acc, s_q[4 * v + 3][threadIdx.x], rv.w);
      }
      if (acc <= bacc) {
        const float d = __fsqrt_rn(acc);
        if (d < bd) {
          bd = d;
          bacc = acc;
          bi = r0 + j;
        }
      }
    }
  }
  if (live) {
    it.out_annf[qi] = bi;
    if (it.out_dist) it.out_dist[qi] = __float_as_uint(bd);
    if (it.out_count) it.out_count[qi] = (uint32_t)a.n;
  }
}

// Gray brute force on packed fp32 pairs: a thread takes two queries (one per
// half of a float2) and meets every reference value duplicated in both halves
// of a shared-memory float2, so one sub/fma pair of f32x2 instructions
// advances both queries' sums.  Each half follows the same order of
// operations as the scalar path.
constexpr int kUnitGrayThreads = 128, kUnitGrayRT = 32;

__global__ void __launch_bounds__(kUnitGrayThreads) k_dense_unit_gray(const UnitDenseArgs a) {
  constexpr int D = 64, QB = 2 * kUnitGrayThreads, RT = kUnitGrayRT;
  __shared__ __align__(16) float2 s_r[RT][D];
  const int64_t nq = a.list ? (int64_t)*a.list_count : a.Q;
  if (!a.list && a.stats && blockIdx.x == 0 && threadIdx.x == 0) a.stats[kStatDenseQueries] = (unsigned long long)nq;
  const int64_t base = (int64_t)blockIdx.x * QB;
  if (base >= nq) return;   // uniform for the CTA
  const FrameItem& it = a.one;
  int64_t qi[2] = {0, 0};
  bool live[2];
  float2 qq[D];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int64_t i = base + h * kUnitGrayThreads + threadIdx.x;
    live[h] = i < nq;
    uint32_t s = 0;
    int y = 0, x = 0;
    if (live[h]) {
      qi[h] = a.list ? (int64_t)a.list[i] - it.query_begin : i;
      y = (int)(qi[h] / it.Wq);
      x = (int)(qi[h] % it.Wq);
      for (int dy = 0; dy < 8; ++dy)
        for (int j = 0; j < 8; ++j) {
          const uint32_t v = it.frame[(int64_t)(y + dy) * it.W + x + j];
          s += v * v;
        }
    }
    const float nv = unit_scale(s);
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const float f = live[h] ? unit_coord(it.frame[(int64_t)(y + k / 8) * it.W + x + k % 8], s, nv) : 0.f;
      if (h == 0) qq[k].x = f;
      else qq[k].y = f;
    }
  }
  // best so far (distance, index) and the largest sum that can still match
  // it; a routed query starts from its previous match (usually close, so the
  // early exit below bites from the first tile), frame 0 from nothing
  float bd0 = __int_as_float(0x7f800000), bd1 = bd0;
  int bi0 = 0, bi1 = 0;
  if (it.prev) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (!live[h]) continue;
      const int rp = it.prev[qi[h]];
      if ((unsigned)rp >= (unsigned)a.n) continue;
      const float* rr = a.Rf + (int64_t)rp * D;
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) acc = unit_step(acc, h ? qq[k].y : qq[k].x, __ldg(rr + k));
      if (h) { bd1 = __fsqrt_rn(acc); bi1 = rp; }
      else { bd0 = __fsqrt_rn(acc); bi0 = rp; }
    }
  }
  float ba0 = unit_root_bound(bd0), ba1 = unit_root_bound(bd1);
  for (int r0 = 0; r0 < a.n; r0 += RT) {
    const int nt = min(RT, a.n - r0);
    __syncthreads();
    for (int k = threadIdx.x; k < nt * D; k += kUnitGrayThreads) {
      const float v = __ldg(a.Rf + (int64_t)r0 * D + k);
      s_r[k / D][k % D] = make_float2(v, v);
    }
    __syncthreads();
    // two references per pass (two independent dependency chains per thread);
    // an odd tail repeats the last reference, which cannot change the result
    for (int j = 0; j < nt; j += 2) {
      const int j2 = j + 1 < nt ? j + 1 : j;
      const float4* ra = reinterpret_cast<const float4*>(s_r[j]);
      const float4* rb = reinterpret_cast<const float4*>(s_r[j2]);
      float2 acc = make_float2(0.f, 0.f), acc2 = acc;
      bool beaten = false;
#pragma unroll
      for (int v = 0; v < D / 2; ++v) {
        const float4 x = ra[v], y = rb[v];   // values 2v and 2v + 1, each twice
        acc = unit_step2(acc, qq[2 * v], make_float2(x.x, x.y));
        acc2 = unit_step2(acc2, qq[2 * v], make_float2(y.x, y.y));
        acc = unit_step2(acc, qq[2 * v + 1], make_float2(x.z, x.w));
        acc2 = unit_step2(acc2, qq[2 * v + 1], make_float2(y.z, y.w));
        // a running sum never decreases (each step adds t^2 >= 0 and rounds
        // monotonically): once every partial sum of the warp exceeds its
        // query's bound (no larger sum has a root that beats or ties the
        // best), neither reference can win -- stop them
        if (v == 7 || v == 15 || v == 23) {
          const bool out = (!live[0] || (acc.x > ba0 && acc2.x > ba0)) && (!live[1] || (acc.y > ba1 && acc2.y > ba1));
          if (__all_sync(0xffffffffu, out)) {
            beaten = true;
            break;
          }
        }
      }
      if (beaten) continue;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const float2 s2 = u ? acc2 : acc;
        const int r = r0 + (u ? j2 : j);
        if (s2.x <= ba0) {
          const float d = __fsqrt_rn(s2.x);
          if (d < bd0 || (d == bd0 && r < bi0)) { bd0 = d; bi0 = r; ba0 = unit_root_bound(d); }
        }
        if (s2.y <= ba1) {
          const float d = __fsqrt_rn(s2.y);
          if (d < bd1 || (d == bd1 && r < bi1)) { bd1 = d; bi1 = r; ba1 = unit_root_bound(d); }
        }
      }
    }
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (!live[h]) continue;
    it.out_annf[qi[h]] = h ? bi1 : bi0;
    if (it.out_dist) it.out_dist[qi[h]] = __float_as_uint(h ? bd1 : bd0);
    if (it.out_count) it.out_count[qi[h]] = (uint32_t)a.n;
  }
}

}  // namespace

cudaError_t launch_unit_tables(Index& ix, cudaStream_t s) {
  k_unit_normalize<<<(ix.n + 127) / 128, 128, 0, s>>>(ix.R, ix.n, ix.D, ix.Rf);
  k_unit_normalize<<<(ix.K + 127) / 128, 128, 0, s>>>(ix.KP, ix.K, ix.D, ix.KPf);
  const int64_t tot = (int64_t)ix.n * ix.Kp;
  const unsigned blocks = (unsigned)((tot + 255) / 256);
  if (ix.C == 1) k_unit_key_distances<64><<<blocks, 256, 0, s>>>(ix.Rf, ix.KPf, ix.n, ix.K, ix.Kp, ix.P);
  else k_unit_key_distances<192><<<blocks, 256, 0, s>>>(ix.Rf, ix.KPf, ix.n, ix.K, ix.Kp, ix.P);
  return cudaGetLastError();
}

cudaError_t launch_dense_unit(const DenseArgs& d, Index& ix, cudaStream_t s) {
  UnitDenseArgs u;
  u.one = d.one;
  u.list = d.list;
  u.list_count = d.list_count;
  u.Q = d.Q;
  u.Rf = ix.Rf;
  u.n = ix.n;
  u.stats = d.stats;
  prof_begin(ix, kSlotDense, s);
  if (ix.C == 1) {
    const int64_t g = (d.Q + 2 * kUnitGrayThreads - 1) / (2 * kUnitGrayThreads);
    k_dense_unit_gray<<<(unsigned)(g > 0 ? g : 1), kUnitGrayThreads, 0, s>>>(u);
  } else {
    const int64_t g = (d.Q + kUnitRgbQB - 1) / kUnitRgbQB;
    k_dense_unit_rgb<<<(unsigned)(g > 0 ? g : 1), kUnitRgbQB, 0, s>>>(u);
  }
  prof_end(ix, kSlotDense, s);
  return cudaGetLastError();
}

}  // namespace riann
