// dense_tc.cu -- brute-force exact nearest neighbours on the 5th-generation
// tensor cores (tcgen05 + TMEM + TMA, sm_103a).  Used for the frame-0
// initialisation and for queries whose rings are too wide.
//
// argmin_r ||q - r||^2 = argmin_r (||r||^2 - 2 q.r), over bf16 operands that
// hold the uint8 values exactly, with exact fp32 accumulation: every product
// and every partial sum is an integer below 2^24 in magnitude.
//  * gray (D = 64): one GEMM with K = D + 16,
//      S = [q | 1 1 1 0..] . [-2r | h 2^16, m 2^8, l, 0..]   (||r||^2 = h 2^16 + m 2^8 + l),
//    every term exact in bf16 (-2r >= -510, h <= 63, m, l <= 255) and every
//    partial sum in [-2 * 64 * 255^2, 64 * 255^2], inside (-2^23, 2^23); the
//    epilogue only takes the minimum of the accumulator.
//  * RGB (D = 192): -2 q.r would reach -2.5e7 > 2^24, so the GEMM is q . r
//    (partial sums <= 192 * 255^2 < 2^24) and the epilogue forms ||r||^2 - 2 q.r.
// The argmin is bit-identical to integer arithmetic.  (INT8 MMA, tcgen05
// kind::i8, is not available on sm_103a.)
//
// Pipeline per CTA (persistent, one CTA per SM, 12 warps):
//   warp 0      TMA producer: one query tile (128 rows) per work item, then a
//               ring of reference tiles (BN rows), SWIZZLE_128B layout
//   warp 1      TMEM allocator and MMA issuer (one thread): D/16 MMAs of
//               128 x BN x 16 per reference tile (gray: + 1 for the norm
//               terms) into one of two TMEM accumulators
//   warps 4-11  epilogue: tcgen05.ld of the accumulator (2 warps per TMEM lane
//               quadrant, each half the columns), fused ||r||^2 - 2 q.r and a
//               running (value, index) minimum per query row; results merge
//               across work items with a 64-bit atomicMin on (dist << 32 | index)
//               (k-NN variant: a running best-8 list per row and half, written
//               per work item and merged by k_dense_knn_finish)
// Every wait is bounded; on timeout the CTA records RIANN_DEV_TIMEOUT, drains
// and frees its TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"

namespace riann {
namespace {

constexpr int kM = 128;
constexpr int kEpiWarps = 8;
constexpr int kThreads = (4 + kEpiWarps) * 32;
constexpr long long kSpinLimit = 2000000000LL;   // clock cycles (about 1 s): the default bound of every wait
constexpr unsigned kFull = 0xffffffffu;

template <int C>
struct Cfg;
template <>
struct Cfg<1> {
  static constexpr int D = 64, ATOMS = 1, BN = 256, STAGES = 4, TMEM_COLS = 512;
  static constexpr bool FOLD = true;    // ||r||^2 added by the tensor cores
};
template <>
struct Cfg<3> {
  static constexpr int D = 192, ATOMS = 3, BN = 128, STAGES = 3, TMEM_COLS = 256;
  static constexpr bool FOLD = false;   // ||r||^2 - 2 q.r formed in the epilogue
};

// bytes of one stage's norm-term tile (BN rows x 32 B) and of the ones tile
template <int C>
__host__ __device__ constexpr int norm_bytes() { return Cfg<C>::FOLD ? Cfg<C>::BN * 32 : 0; }
template <int C>
__host__ __device__ constexpr int ones_bytes() { return Cfg<C>::FOLD ? kM * 32 : 0; }

// k-NN: each epilogue thread stages a 32-column chunk of its row in shared
// memory (36-float stride: conflict-free 16-byte stores) when the chunk holds
// list candidates, so that a candidate's score is one load to fetch
constexpr int kKnnStageStride = 36;
template <bool KNN>
__host__ __device__ constexpr int knn_stage_bytes() { return KNN ? kEpiWarps * 32 * kKnnStageStride * 4 : 0; }

// pipeline stages: the RGB k-NN form gives one up to its staging area
template <int C, bool KNN>
__host__ __device__ constexpr int stages() { return (C == 3 && KNN) ? Cfg<C>::STAGES - 1 : Cfg<C>::STAGES; }

template <int C, bool KNN>
__host__ __device__ constexpr int smem_bytes() {
  using G = Cfg<C>;
  return 1024 /* alignment slack */ + G::ATOMS * kM * 128 + stages<C, KNN>() * G::ATOMS * G::BN * 128 +
         stages<C, KNN>() * norm_bytes<C>() + ones_bytes<C>() + 256 + knn_stage_bytes<KNN>();
}

struct TcArgs {
  CUtensorMap tmA;                // Aq  [rows][D] bf16, box 64 x 128
  CUtensorMap tmB;                // Rbf [n_pad][D] bf16, box 64 x BN
  const float* rnorm;             // [n_pad] ||r||^2 (RGB)
  const __nv_bfloat16* rn;        // [n_pad][16] norm terms in core-matrix order (gray)
  const uint32_t* qnorm;          // [rows]
  const uint32_t* count;          // device count of query rows (nullptr: Qfix)
  int64_t Qfix;
  int n_pad;
  unsigned long long* best;       // [rows] packed (dist << 32 | index), pre-set to ~0
  unsigned long long* lists;      // k-NN: [work items][kM][2 halves][kKnnMax] packed, ascending
  uint32_t* status;
  long long spin_limit;           // bound of every wait, in clock cycles
  int withhold;                   // test hook: the producer loads no reference tile, so the first
                                  // wait for one runs out after spin_limit (RIANN_DEV_TIMEOUT)
};

// k-NN: insert score s of column c into the ascending list (s < its last
// entry); an equal score already listed keeps its place, so that the lower
// column comes first (each thread visits its columns in ascending order).
template <int KM>
__device__ __forceinline__ void knn_insert(float (&ls)[KM], int (&li)[KM], float s, int c) {
#pragma unroll
  for (int p = KM - 1; p > 0; --p) {
    const bool shift = ls[p - 1] > s;
    const bool here = !shift && ls[p] > s;
    ls[p] = shift ? ls[p - 1] : (here ? s : ls[p]);
    li[p] = shift ? li[p - 1] : (here ? c : li[p]);
  }
  if (ls[0] > s) {
    ls[0] = s;
    li[0] = c;
  }
}

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity; false on timeout/abort.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          long long limit) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > limit) {
      *abort_flag = 1;
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 B, 8-row groups 1024 B apart (the layout TMA SWIZZLE_128B writes).
__device__ __forceinline__ uint64_t sw128_desc(const void* p) {
  const uint32_t addr = smem_u32(p);
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);   // start address >> 4
  d |= (uint64_t)1 << 16;                           // leading byte offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;                 // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                           // descriptor version for sm_100 family
  d |= (uint64_t)2 << 61;                           // layout: SWIZZLE_128B
  return d;
}

// Shared-memory matrix descriptor, no swizzle, K-major, K = 16: 8-row x
// 16-byte core matrices, the two along K 128 B apart (leading byte offset),
// consecutive 8-row groups 256 B apart (stride byte offset).
__device__ __forceinline__ uint64_t plain_desc(const void* p) {
  const uint32_t addr = smem_u32(p);
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)(128 >> 4) << 16;
  d |= (uint64_t)(256 >> 4) << 32;
  d |= (uint64_t)1 << 46;                           // descriptor version for sm_100 family
  return d;                                         // layout 0: no swizzle
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Instruction descriptor, kind::f16: D f32, A and B bf16, both K-major, M x N.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// tcgen05.ld of 64 consecutive accumulator columns of this warp's 32 TMEM
// lanes (one column per register), then wait for it.
template <int N>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, uint32_t (&v)[N]);

template <>
__device__ __forceinline__ void tmem_ld<64>(uint32_t taddr, uint32_t (&v)[64]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, "
      "%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, "
      "%48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%64];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31]), "=r"(v[32]), "=r"(v[33]), "=r"(v[34]), "=r"(v[35]), "=r"(v[36]), "=r"(v[37]), "=r"(v[38]), "=r"(v[39]), "=r"(v[40]), "=r"(v[41]), "=r"(v[42]), "=r"(v[43]), "=r"(v[44]), "=r"(v[45]), "=r"(v[46]), "=r"(v[47]), "=r"(v[48]), "=r"(v[49]), "=r"(v[50]), "=r"(v[51]), "=r"(v[52]), "=r"(v[53]), "=r"(v[54]), "=r"(v[55]), "=r"(v[56]), "=r"(v[57]), "=r"(v[58]), "=r"(v[59]), "=r"(v[60]), "=r"(v[61]), "=r"(v[62]), "=r"(v[63])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Two fp32 FMAs in one instruction (sm_100 family): d = a * b + c per lane.
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n .reg .b64 ra, rb, rc, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
      " mov.b64 rc, {%6, %7};\n fma.rn.f32x2 rd, ra, rb, rc;\n mov.b64 {%0, %1}, rd;\n}\n"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}

__device__ __forceinline__ float min3(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// ---------------------------------------------------------------------------
// the GEMM + argmin kernel
// ---------------------------------------------------------------------------
template <int C, bool KNN>
__global__ void __launch_bounds__(kThreads, 1) k_dense_tc(const __grid_constant__ TcArgs a) {
  using G = Cfg<C>;
  constexpr uint32_t IDESC = instr_desc(kM, G::BN);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;                                        // [ATOMS][128][128 B]
  uint8_t* sB = sA + G::ATOMS * kM * 128;                    // [STAGES][ATOMS][BN][128 B]
  constexpr int NST = stages<C, KNN>();
  uint8_t* sN = sB + NST * G::ATOMS * G::BN * 128;           // gray: [STAGES][BN x 32 B] norm terms
  uint8_t* sOnes = sN + NST * norm_bytes<C>();               // gray: [128 x 32 B] ones in columns 0..2
  uint64_t* bars = reinterpret_cast<uint64_t*>(sOnes + ones_bytes<C>());
  uint64_t* full = bars;
  uint64_t* empty = full + NST;
  uint64_t* tfull = empty + NST;
  uint64_t* tempty = tfull + 2;
  uint64_t* afull = tempty + 2;
  uint64_t* aempty = afull + 1;
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(aempty + 1);
  float* sK = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(bars) + 256);   // k-NN staging rows
  volatile int* s_abort = reinterpret_cast<volatile int*>(s_tmem + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long lim = a.spin_limit;
  const int64_t Qd = a.count ? (int64_t)*a.count : a.Qfix;
  const int64_t n_qt = (Qd + kM - 1) / kM;
  const int n_rt = a.n_pad / G::BN;
  const int nsplit = dense_nsplit(n_qt, (int)gridDim.x, n_rt, !KNN);
  const int per = (n_rt + nsplit - 1) / nsplit;
  const int64_t n_items = n_qt * nsplit;
  if ((int64_t)blockIdx.x >= n_items) return;   // uniform for the whole CTA

  if (G::FOLD) {
    // A operand of the norm MMA: every query row [1 1 1 0 .. 0] (core-matrix order)
    __nv_bfloat16* o = reinterpret_cast<__nv_bfloat16*>(sOnes);
    for (int e = threadIdx.x; e < kM * 16; e += blockDim.x) {
      const int k = ((e >> 6) & 1) * 8 + (e & 7);
      o[e] = __float2bfloat16_rn(k < 3 ? 1.f : 0.f);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the tensor cores
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&tfull[s], 1);
      mbar_init(&tempty[s], kEpiWarps);
    }
    mbar_init(afull, 1);
    mbar_init(aempty, 1);
    *s_abort = 0;
    fence_barrier_init();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                 "r"(G::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      int stage = 0;
      uint32_t phase = 0, a_phase = 0;
      bool first = true, ok = true;
      for (int64_t it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
        const int qt = (int)(it / nsplit), part = (int)(it % nsplit);
        const int rt0 = part * per, rt1 = min(n_rt, rt0 + per);
        if (!first) {
          if (!(ok = mbar_wait(aempty, a_phase, s_abort, lim))) break;
          a_phase ^= 1;
        }
        first = false;
        mbar_expect_tx(afull, G::ATOMS * kM * 128);
        for (int at = 0; at < G::ATOMS; ++at) tma_load_2d(sA + at * kM * 128, &a.tmA, afull, 64 * at, qt * kM);
        if (a.withhold) {
          // test hook: no reference tile follows; wait (bounded) for the query
          // tile to land so that no copy is in flight when the CTA leaves
          ok = mbar_wait(afull, 0, s_abort, lim);
          ok = false;
          break;
        }
        for (int rt = rt0; rt < rt1; ++rt) {
          if (!(ok = mbar_wait(&empty[stage], phase ^ 1, s_abort, lim))) break;
          mbar_expect_tx(&full[stage], G::ATOMS * G::BN * 128 + norm_bytes<C>());
          for (int at = 0; at < G::ATOMS; ++at)
            tma_load_2d(sB + (stage * G::ATOMS + at) * G::BN * 128, &a.tmB, &full[stage], 64 * at, rt * G::BN);
          if (G::FOLD)
            bulk_load(sN + stage * norm_bytes<C>(), a.rn + (int64_t)rt * G::BN * 16, norm_bytes<C>(), &full[stage]);
          if (++stage == NST) {
            stage = 0;
            phase ^= 1;
          }
        }
      }
      // tail: every stage released and the last query tile consumed before exit
      for (int s = 0; s < NST && ok; ++s) {
        ok = mbar_wait(&empty[stage], phase ^ 1, s_abort, lim);
        if (++stage == NST) {
          stage = 0;
          phase ^= 1;
        }
      }
      if (ok && !first) mbar_wait(aempty, a_phase, s_abort, lim);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      int stage = 0, acc = 0;
      uint32_t phase = 0, a_phase = 0, acc_phase = 0;
      bool ok = true;
      for (int64_t it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
        const int part = (int)(it % nsplit);
        const int rt0 = part * per, rt1 = min(n_rt, rt0 + per);
        if (!(ok = mbar_wait(afull, a_phase, s_abort, lim))) break;
        a_phase ^= 1;
        for (int rt = rt0; rt < rt1; ++rt) {
          if (!(ok = mbar_wait(&full[stage], phase, s_abort, lim))) break;
          if (!(ok = mbar_wait(&tempty[acc], acc_phase ^ 1, s_abort, lim))) break;
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(acc * G::BN);
#pragma unroll
          for (int kk = 0; kk < G::D / 16; ++kk) {
            const int at = kk >> 2, ko = (kk & 3) * 32;
            tc_mma(d, sw128_desc(sA + at * kM * 128 + ko),
                   sw128_desc(sB + (stage * G::ATOMS + at) * G::BN * 128 + ko), IDESC, kk > 0 ? 1u : 0u);
          }
          if (G::FOLD) tc_mma(d, plain_desc(sOnes), plain_desc(sN + stage * norm_bytes<C>()), IDESC, 1u);
          tc_commit(&empty[stage]);
          tc_commit(&tfull[acc]);
          if (++stage == NST) {
            stage = 0;
            phase ^= 1;
          }
          if (++acc == 2) {
            acc = 0;
            acc_phase ^= 1;
          }
        }
        if (ok) tc_commit(aempty);
      }
    }
  } else if (warp >= 4) {
    // ---------------- epilogue ----------------
    const int quad = warp & 3;                 // TMEM lanes this warp may read
    const int half = (warp - 4) >> 2;          // which half of the BN columns
    const int row = quad * 32 + lane;          // query row within the tile
    constexpr int HALF = G::BN / 2;
    int acc = 0;
    uint32_t acc_phase = 0;
    bool ok = true;
    const float2 m2 = make_float2(-2.f, -2.f);
    constexpr int CH = HALF < 64 ? HALF : 64;   // columns per TMEM load
    for (int64_t it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
      const int qt = (int)(it / nsplit), part = (int)(it % nsplit);
      const int rt0 = part * per, rt1 = min(n_rt, rt0 + per);
      float bv = __int_as_float(0x7f800000);
      int bi = 0;
      float ls[KNN ? kKnnMax : 1];
      int li[KNN ? kKnnMax : 1];
#pragma unroll
      for (int j = 0; j < (KNN ? kKnnMax : 1); ++j) {
        ls[j] = __int_as_float(0x7f800000);
        li[j] = 0;
      }
      for (int rt = rt0; rt < rt1; ++rt) {
        const int colt = rt * G::BN + half * HALF;
        // RGB: ||r||^2 of this tile's first 32 columns, fetched while the MMA runs
        float4 rn[8];
        if (!G::FOLD) {
#pragma unroll
          for (int j = 0; j < 8; ++j) rn[j] = __ldg(reinterpret_cast<const float4*>(a.rnorm + colt) + j);
        }
        ok = mbar_wait(&tfull[acc], acc_phase, s_abort, lim);
        if (!__all_sync(kFull, ok)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t tb = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * G::BN + half * HALF);
#pragma unroll 1
        for (int c = 0; c < HALF; c += CH) {
          uint32_t v[CH];
          tmem_ld<CH>(tb + (uint32_t)c, v);
#pragma unroll
          for (int h32 = 0; h32 < CH / 32; ++h32) {
            const int col0 = colt + c + 32 * h32;
            float x[32];
            if (G::FOLD) {
#pragma unroll
              for (int j = 0; j < 32; ++j) x[j] = __uint_as_float(v[32 * h32 + j]);
            } else {
              // next 32 columns' norms in flight during this chunk's arithmetic
              float4 rx[8];
              const int cn = c + 32 * h32 + 32 < HALF ? col0 + 32 : col0;
#pragma unroll
              for (int j = 0; j < 8; ++j) rx[j] = __ldg(reinterpret_cast<const float4*>(a.rnorm + cn) + j);
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const uint32_t* w = v + 32 * h32 + 4 * j;
                const float2 lo = fma2(make_float2(__uint_as_float(w[0]), __uint_as_float(w[1])), m2,
                                       make_float2(rn[j].x, rn[j].y));
                const float2 hi = fma2(make_float2(__uint_as_float(w[2]), __uint_as_float(w[3])), m2,
                                       make_float2(rn[j].z, rn[j].w));
                x[4 * j + 0] = lo.x;
                x[4 * j + 1] = lo.y;
                x[4 * j + 2] = hi.x;
                x[4 * j + 3] = hi.y;
              }
#pragma unroll
              for (int j = 0; j < 8; ++j) rn[j] = rx[j];
            }
            float m[11];
#pragma unroll
            for (int j = 0; j < 10; ++j) m[j] = min3(x[3 * j], x[3 * j + 1], x[3 * j + 2]);
            m[10] = fminf(x[30], x[31]);
            const float m0 = min3(m[0], m[1], m[2]), m1 = min3(m[3], m[4], m[5]);
            const float mm2 = min3(m[6], m[7], m[8]), m3 = fminf(m[9], m[10]);
            const float cmin = fminf(min3(m0, m1, mm2), m3);
            if (!KNN) {
              if (cmin < bv) {       // rare after the first tiles: locate the lowest column
                int jj = 31;
#pragma unroll
                for (int j = 31; j >= 0; --j)
                  if (x[j] == cmin) jj = j;
                bv = cmin;
                bi = col0 + jj;
              }
            } else if (cmin < ls[(KNN ? kKnnMax : 1) - 1]) {
              // the columns below the current k-th, in ascending order; a
              // lane's work follows its own count (the warp waits for the
              // largest), not all 32 columns
              const float thr = ls[(KNN ? kKnnMax : 1) - 1];
              float* srow = sK + ((warp - 4) * 32 + lane) * kKnnStageStride;   // this thread's own row
#pragma unroll
              for (int j = 0; j < 8; ++j)
                reinterpret_cast<float4*>(srow)[j] = make_float4(x[4 * j], x[4 * j + 1], x[4 * j + 2], x[4 * j + 3]);
              uint32_t mask = 0;
#pragma unroll
              for (int j = 0; j < 32; ++j) mask |= (x[j] < thr ? 1u : 0u) << j;
              while (mask) {
                const int jj = __ffs(mask) - 1;
                mask &= mask - 1;
                const float v = srow[jj];
                if (v < ls[(KNN ? kKnnMax : 1) - 1]) knn_insert(ls, li, v, col0 + jj);
              }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[acc]);
        if (++acc == 2) {
          acc = 0;
          acc_phase ^= 1;
        }
      }
      const int64_t i = (int64_t)qt * kM + row;
      // padding columns score +inf (RGB) or 2^24 (gray), above every real score
      if (KNN) {
        if (ok && i < Qd) {
          unsigned long long* dst = a.lists + (((size_t)it * kM + row) * 2 + half) * kKnnMax;
          const float qn = (float)a.qnorm[i];
#pragma unroll
          for (int j = 0; j < (KNN ? kKnnMax : 1); ++j)
            dst[j] = ls[j] < 16777216.f ? ((unsigned long long)(uint32_t)(qn + ls[j]) << 32) | (unsigned)li[j]
                                        : ~0ull;
        }
      } else if (ok && i < Qd && bv < 16777216.f) {
        const uint32_t dist = (uint32_t)((float)a.qnorm[i] + bv);   // exact: integer < 2^24
        atomicMin(a.best + i, ((unsigned long long)dist << 32) | (unsigned)bi);
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G::TMEM_COLS)
                 : "memory");
  }
  if (threadIdx.x == 0 && *s_abort) atomicOr(a.status, RIANN_DEV_TIMEOUT);
}

// ---------------------------------------------------------------------------
// query rows in, results out
// ---------------------------------------------------------------------------
struct PrepArgs {
  FrameItem one;                  // single frame (items == nullptr)
  const FrameItem* items;         // batched launch
  const BatchHeader* hdr;
  int64_t Q;
  const int32_t* list;
  const uint32_t* list_count;
  __nv_bfloat16* Aq;
  uint32_t* qnorm;
  unsigned long long* best;
  uint32_t* status;               // checked build: RIANN_DEV_BOUNDS for a query id outside its frame
};

// The item holding global query id gid (items sorted by query_begin).
__device__ __forceinline__ const FrameItem& item_of(const FrameItem* items, const BatchHeader* hdr, int64_t gid) {
  int lo = 0, hi = hdr->n_items - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (items[mid].query_begin <= gid) lo = mid; else hi = mid - 1;
  }
  return items[lo];
}

// Row i of Aq = bf16 bytes of the i-th query patch ((dy, dx, c) order), its
// squared norm, and a reset best slot.  One thread per query.
template <int C>
__global__ void k_dense_prep(PrepArgs a) {
  constexpr int NW = 16 * C;
  const int64_t nq = a.list ? (int64_t)*a.list_count : a.Q;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t gid = a.list ? (int64_t)a.list[i] : i;
    const FrameItem& it = a.items ? item_of(a.items, a.hdr, gid) : a.one;
    int64_t qi = gid - it.query_begin;
    if (!RIANN_IN_RANGE(qi >= 0 && qi < (int64_t)it.Hq * it.Wq, a.status)) qi = 0;
    const int y = (int)(qi / it.Wq), x = (int)(qi % it.Wq);
    uint2* dst = reinterpret_cast<uint2*>(a.Aq + i * (64 * C));
    uint32_t nrm = 0;
#pragma unroll 4
    for (int w = 0; w < NW; ++w) {
      const int dy = w / (2 * C), j = w % (2 * C);
      const uint8_t* p = it.frame + ((int64_t)(y + dy) * it.W + x) * C + 4 * j;
      const uint32_t b0 = p[0], b1 = p[1], b2 = p[2], b3 = p[3];
      nrm += b0 * b0 + b1 * b1 + b2 * b2 + b3 * b3;
      // bf16 of an integer 0..255: exact; pack two per 32-bit word
      const uint32_t h0 = __bfloat16_as_ushort(__float2bfloat16_rn((float)b0));
      const uint32_t h1 = __bfloat16_as_ushort(__float2bfloat16_rn((float)b1));
      const uint32_t h2 = __bfloat16_as_ushort(__float2bfloat16_rn((float)b2));
      const uint32_t h3 = __bfloat16_as_ushort(__float2bfloat16_rn((float)b3));
      dst[w] = make_uint2(h0 | (h1 << 16), h2 | (h3 << 16));
    }
    a.qnorm[i] = nrm;
    a.best[i] = ~0ull;
  }
}

struct FinishArgs {
  FrameItem one;
  const FrameItem* items;
  const BatchHeader* hdr;
  const int32_t* list;
  const uint32_t* list_count;
  int64_t Q;
  const unsigned long long* best;
  int n;
  unsigned long long* stats;
  uint32_t* status;               // checked build: RIANN_DEV_BOUNDS for a query id outside its frame
};

__global__ void k_dense_finish(FinishArgs a) {
  const int64_t nq = a.list ? (int64_t)*a.list_count : a.Q;
  if (!a.list && a.stats && blockIdx.x == 0 && threadIdx.x == 0) a.stats[kStatDenseQueries] = (unsigned long long)nq;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t gid = a.list ? (int64_t)a.list[i] : i;
    const FrameItem& it = a.items ? item_of(a.items, a.hdr, gid) : a.one;
    const int64_t qi = gid - it.query_begin;
    if (!RIANN_IN_RANGE(qi >= 0 && qi < (int64_t)it.Hq * it.Wq, a.status)) continue;
    const unsigned long long k = a.best[i];
    it.out_annf[qi] = (int32_t)(k & 0xffffffffu);
    if (it.out_dist) it.out_dist[qi] = (uint32_t)(k >> 32);
    if (it.out_count) it.out_count[qi] = (uint32_t)a.n;
  }
}

// k-NN: the k best of a query's per-(work item, half) lists -- every list
// ascending, ties already in index order -- and the outputs.
struct KnnFinishArgs {
  FrameItem one;
  const int32_t* list;
  const uint32_t* list_count;
  int64_t Q;
  const unsigned long long* lists;
  int grid, n_rt, n, k;
  int32_t* knn_idx;
  uint32_t* knn_dist;
  unsigned long long* stats;
};

__global__ void k_dense_knn_finish(KnnFinishArgs a) {
  const int64_t nq = a.list ? (int64_t)*a.list_count : a.Q;
  if (!a.list && a.stats && blockIdx.x == 0 && threadIdx.x == 0) a.stats[kStatDenseQueries] = (unsigned long long)nq;
  const int nsplit = dense_nsplit((nq + kM - 1) / kM, a.grid, a.n_rt);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t qt = i / kM;
    const int row = (int)(i % kM);
    unsigned long long top[kKnnMax];
#pragma unroll
    for (int j = 0; j < kKnnMax; ++j) top[j] = ~0ull;
    for (int part = 0; part < nsplit; ++part) {
      for (int half = 0; half < 2; ++half) {
        const unsigned long long* src = a.lists + (((size_t)(qt * nsplit + part) * kM + row) * 2 + half) * kKnnMax;
        for (int j = 0; j < kKnnMax; ++j) {
          const unsigned long long v = src[j];
          if (v >= top[kKnnMax - 1]) break;           // the rest of this list is larger
#pragma unroll
          for (int p = kKnnMax - 1; p > 0; --p) {      // insert (keys are distinct)
            const bool shift = top[p - 1] > v;
            top[p] = shift ? top[p - 1] : (top[p] > v ? v : top[p]);
          }
          if (top[0] > v) top[0] = v;
        }
      }
    }
    const int64_t gid = a.list ? (int64_t)a.list[i] : i;
    const int64_t qi = gid - a.one.query_begin;
#pragma unroll
    for (int j = 0; j < kKnnMax; ++j) {
      if (j < a.k) {
        a.knn_idx[qi * a.k + j] = top[j] == ~0ull ? -1 : (int32_t)(top[j] & 0xffffffffu);
        if (a.knn_dist) a.knn_dist[qi * a.k + j] = (uint32_t)(top[j] >> 32);
      }
    }
    a.one.out_annf[qi] = (int32_t)(top[0] & 0xffffffffu);
    if (a.one.out_dist) a.one.out_dist[qi] = (uint32_t)(top[0] >> 32);
    if (a.one.out_count) a.one.out_count[qi] = (uint32_t)a.n;
  }
}

// The dynamic shared-memory limit is an attribute of the kernel on each
// device: set once per (device, instantiation), under a lock.
constexpr int kAttrDevices = 64;

template <int C, bool KNN>
cudaError_t launch_tc(const TcArgs& t, cudaStream_t s) {
  static std::mutex mu;
  static bool attr[kAttrDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kAttrDevices) return cudaErrorInvalidDevice;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!attr[dev]) {
      e = cudaFuncSetAttribute(k_dense_tc<C, KNN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<C, KNN>());
      if (e != cudaSuccess) return e;
      attr[dev] = true;
    }
  }
  k_dense_tc<C, KNN><<<sm_count(), kThreads, smem_bytes<C, KNN>(), s>>>(t);
  return cudaGetLastError();
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

}  // namespace

// 2-D tensor map over bf16 rows of D elements: boxes of 64 elements x box_rows
// rows with the 128-byte swizzle (the operand layout the MMA descriptors use).
bool make_row_map(CUtensorMap* m, const void* base, uint64_t rows, int D, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)D, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)D * 2};
  cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1u, 1u};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int dense_ref_rows_per_tile(int C) { return C == 1 ? Cfg<1>::BN : Cfg<3>::BN; }

// Work items of a launch: n_qt * nsplit, at most n_qt (nsplit = 1) or below
// 4 * grid (nsplit = ceil(2 grid / n_qt) with n_qt < 2 grid); each item holds
// kM rows x 2 halves x kKnnMax entries.
int64_t dense_knn_list_entries(int64_t Q) {
  const int64_t n_qt = (Q + kM - 1) / kM;
  const int64_t g4 = 4 * (int64_t)sm_count();
  return (n_qt > g4 ? n_qt : g4) * kM * 2 * kKnnMax;
}

cudaError_t launch_dense_tc(const DenseArgs& d, Index& ix, Workspace& ws, cudaStream_t s) {
  if (!ix.tm_ready) return cudaErrorNotSupported;
  const int C = ix.C;
  PrepArgs p;
  p.one = d.one;
  p.items = d.items;
  p.hdr = d.hdr;
  p.Q = d.Q;
  p.list = d.list;
  p.list_count = d.list_count;
  p.Aq = ws.Aq;
  p.qnorm = ws.qnorm;
  p.best = ws.best;
  p.status = ix.status;
  int64_t blocks = (d.Q + 255) / 256;
  const int64_t cap = (int64_t)sm_count() * 16;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  prof_begin(ix, kSlotPrep, s);
  if (C == 1) k_dense_prep<1><<<(unsigned)blocks, 256, 0, s>>>(p);
  else k_dense_prep<3><<<(unsigned)blocks, 256, 0, s>>>(p);
  prof_end(ix, kSlotPrep, s);

  TcArgs t;
  t.tmA = ws.tmAq;
  t.tmB = ix.tmRbf;
  t.rnorm = ix.rnorm;
  t.rn = ix.RN;
  t.qnorm = ws.qnorm;
  t.count = d.list ? d.list_count : nullptr;
  t.Qfix = d.Q;
  t.n_pad = ix.n_pad;
  t.best = ws.best;
  t.lists = ws.knn_lists;
  t.status = ix.status;
  t.spin_limit = d.spin_limit > 0 ? d.spin_limit : kSpinLimit;
  t.withhold = d.withhold;
  const bool knn = d.knn > 0;
  if (knn && (!ws.knn_lists || dense_knn_list_entries(d.Q) > ws.knn_cap)) return cudaErrorInvalidValue;
  prof_begin(ix, kSlotDense, s);
  cudaError_t e = C == 1 ? (knn ? launch_tc<1, true>(t, s) : launch_tc<1, false>(t, s))
                         : (knn ? launch_tc<3, true>(t, s) : launch_tc<3, false>(t, s));
  prof_end(ix, kSlotDense, s);
  if (e != cudaSuccess) return e;
  if (knn) {
    KnnFinishArgs f;
    f.one = d.one;
    f.list = d.list;
    f.list_count = d.list_count;
    f.Q = d.Q;
    f.lists = ws.knn_lists;
    f.grid = sm_count();
    f.n_rt = ix.n_pad / dense_ref_rows_per_tile(C);
    f.n = ix.n;
    f.k = d.knn;
    f.knn_idx = d.knn_idx;
    f.knn_dist = d.knn_dist;
    f.stats = d.stats;
    k_dense_knn_finish<<<(unsigned)blocks, 256, 0, s>>>(f);
    return cudaGetLastError();
  }

  FinishArgs f;
  f.one = d.one;
  f.items = d.items;
  f.hdr = d.hdr;
  f.list = d.list;
  f.list_count = d.list_count;
  f.Q = d.Q;
  f.best = ws.best;
  f.n = ix.n;
  f.stats = d.stats;
  f.status = ix.status;
  k_dense_finish<<<(unsigned)blocks, 256, 0, s>>>(f);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Allocation-free brute force.
//
// Some callers may not allocate device memory once they are running: a
// real-time video pipeline that fixes its memory budget at start-up, or a
// plug-in whose host application owns every allocation.  For them the
// brute-force path can run with its scratch (bf16 query rows, query norms and
// the packed per-query best slots) in the fixed device array below instead of
// the index's growable scratch.  Every GPU that loads this library holds the
// array until the process exits.
//
// Host code must not pass `g_noalloc_scratch` itself to a kernel: on the host
// that name is only a stand-in for the device symbol.  The device address is
// looked up once per device (cudaGetSymbolAddress, with that device current)
// on the first call made on that device, together with the TMA descriptors
// over it.  That first call must therefore come before any stream capture: a
// call made while `s` is capturing, before the set-up has succeeded on its
// device, is refused (and a failed set-up is retried by the next call).
// All calls share the array and it keeps the last call's contents; the
// per-query best slots are reset by every call before use.  Calls that overlap
// on the GPU (e.g. issued on two streams) race on the array.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoallocBytes = size_t(16) << 20;   // 16 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

struct NoallocLayout {
  int64_t rows;        // query rows that fit (multiple of 128)
  size_t qnorm_off;    // byte offset of the uint32 norms
  size_t best_off;     // byte offset of the uint64 best slots
};

NoallocLayout noalloc_layout(int C) {
  const size_t per = (size_t)128 * C + 4 + 8;            // bf16 row + norm + best slot
  int64_t rows = (int64_t)((kNoallocBytes - 1024) / per) / kM * kM;
  NoallocLayout L;
  L.rows = rows;
  L.qnorm_off = align256((size_t)rows * 128 * C);
  L.best_off = align256(L.qnorm_off + (size_t)rows * 4);
  return L;
}

struct NoallocDevice {
  std::mutex mu;
  bool ready = false;              // set-up succeeded on this device
  unsigned char* base = nullptr;   // device address of g_noalloc_scratch
  CUtensorMap map[2];              // [0] gray rows (D = 64), [1] RGB rows (D = 192)
  bool map_ok[2] = {false, false};
};

constexpr int kMaxDevices = 64;
NoallocDevice g_noalloc_dev[kMaxDevices];

}  // namespace

int64_t noalloc_max_queries(int C) { return noalloc_layout(C).rows; }

// Returns cudaErrorInvalidValue when the frame has more queries than fit.
cudaError_t launch_exact_nn_noalloc(const DenseArgs& d, Index& ix, cudaStream_t s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  NoallocDevice& nd = g_noalloc_dev[dev];
  {
    std::lock_guard<std::mutex> lock(nd.mu);
    if (!nd.ready) {
      // the set-up's runtime calls must not run inside a stream capture
      cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
      e = cudaStreamIsCapturing(s, &cap);
      if (e != cudaSuccess) return e;
      if (cap != cudaStreamCaptureStatusNone) return cudaErrorStreamCaptureUnsupported;
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return e;
      nd.base = static_cast<unsigned char*>(p);
      for (int k = 0; k < 2; ++k) {
        const int C = k ? 3 : 1;
        nd.map_ok[k] = make_row_map(&nd.map[k], nd.base, (uint64_t)noalloc_layout(C).rows, 64 * C, kM);
      }
      nd.ready = true;
    }
  }
  const int C = ix.C;
  const int k = C == 1 ? 0 : 1;
  if (!nd.map_ok[k] || !ix.tm_ready) return cudaErrorNotSupported;
  const NoallocLayout L = noalloc_layout(C);
  if (d.Q > L.rows) return cudaErrorInvalidValue;
  __nv_bfloat16* Aq = reinterpret_cast<__nv_bfloat16*>(nd.base);
  uint32_t* qnorm = reinterpret_cast<uint32_t*>(nd.base + L.qnorm_off);
  unsigned long long* best = reinterpret_cast<unsigned long long*>(nd.base + L.best_off);

  PrepArgs p;
  p.one = d.one;
  p.items = nullptr;
  p.hdr = nullptr;
  p.Q = d.Q;
  p.list = nullptr;
  p.list_count = nullptr;
  p.Aq = Aq;
  p.qnorm = qnorm;
  p.best = best;
  p.status = ix.status;
  int64_t blocks = (d.Q + 255) / 256;
  const int64_t cap = (int64_t)sm_count() * 16;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  if (C == 1) k_dense_prep<1><<<(unsigned)blocks, 256, 0, s>>>(p);
  else k_dense_prep<3><<<(unsigned)blocks, 256, 0, s>>>(p);

  TcArgs t;
  t.tmA = nd.map[k];
  t.tmB = ix.tmRbf;
  t.rnorm = ix.rnorm;
  t.rn = ix.RN;
  t.qnorm = qnorm;
  t.count = nullptr;
  t.Qfix = d.Q;
  t.n_pad = ix.n_pad;
  t.best = best;
  t.lists = nullptr;
  t.status = ix.status;
  t.spin_limit = kSpinLimit;
  t.withhold = 0;
  e = C == 1 ? launch_tc<1, false>(t, s) : launch_tc<3, false>(t, s);
  if (e != cudaSuccess) return e;

  FinishArgs f;
  f.one = d.one;
  f.items = nullptr;
  f.hdr = nullptr;
  f.list = nullptr;
  f.list_count = nullptr;
  f.Q = d.Q;
  f.best = best;
  f.n = ix.n;
  f.stats = nullptr;
  f.status = ix.status;
  k_dense_finish<<<(unsigned)blocks, 256, 0, s>>>(f);
  return cudaGetLastError();
}

}  // namespace riann
