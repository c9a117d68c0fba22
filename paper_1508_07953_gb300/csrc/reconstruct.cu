// reconstruct.cu -- rebuild a frame from its ANN field (Sec. 4): every patch
// is replaced by its matched reference patch and overlapping patches are
// averaged; the reconstruction error E = ||f_GT - f_R||_2 / ||f_GT||_2 comes
// from two exact integer sums.
//
// One thread per output pixel (all channels); a CTA owns an 8 x 32 tile and
// stages the field entries of the (8 + 7) x (32 + 7) query patches that cover
// it.  Pixel (y, x) is covered by the patches with top-left corner
// (y - dy, x - dx), 0 <= dy, dx < 8, inside the valid query grid; it receives
// byte (dy, dx, c) of each such patch's match.  The average is rounded half
// up to 8 bits in integers: (2 sum + count) / (2 count).  Gray: the CTA also
// stages the 585 matched rows (64 B each, padded to 68 B so that the 32
// patches a warp reads at one (dy, dx) fall in distinct banks) with 16-byte
// loads and gathers bytes from shared memory.  RGB (192-byte rows): the
// gathers go to global memory, where each row is reused from L1.
#include "reconstruct.cuh"

namespace riann {
namespace {

constexpr int kTY = 8, kTX = 32;
constexpr int kPY = kTY + kPatch - 1, kPX = kTX + kPatch - 1;

template <int C>
__global__ void __launch_bounds__(kTY * kTX) k_reconstruct(const ReconArgs a) {
  constexpr int D = 64 * C;
  constexpr int RW = C == 1 ? 17 : 1;            // staged row stride in words (gray)
  __shared__ int32_t s_f[kPY][kPX];               // field entries of the covering patches
  __shared__ uint32_t s_rows[C == 1 ? kPY * kPX : 1][RW];
  __shared__ unsigned long long s_red[2][kTY * kTX / 32];
  const int H = a.H, W = a.W, Hq = H - 7, Wq = W - 7;
  const int ty0 = blockIdx.y * kTY, tx0 = blockIdx.x * kTX;
  for (int i = threadIdx.x; i < kPY * kPX; i += blockDim.x) {
    const int py = ty0 - 7 + i / kPX, px = tx0 - 7 + i % kPX;
    int32_t r = -1;
    if (py >= 0 && py < Hq && px >= 0 && px < Wq) {
      r = a.annf[(int64_t)py * Wq + px];
      if ((unsigned)r >= (unsigned)a.n) {
        atomicOr(a.status, RIANN_DEV_BAD_PREV);
        r = -1;
      }
    }
    s_f[i / kPX][i % kPX] = r;
  }
  __syncthreads();
  if (C == 1) {
    // one 16-byte load per quarter row (rows are 64-byte aligned); the
    // shared rows keep their 68-byte stride, so the words are stored singly
    const uint4* R4 = reinterpret_cast<const uint4*>(a.R);
    for (int i = threadIdx.x; i < kPY * kPX * 4; i += blockDim.x) {
      const int p = i >> 2, c = i & 3;
      const int32_t r = s_f[p / kPX][p % kPX];
      const uint4 v = r >= 0 ? __ldg(R4 + (int64_t)r * 4 + c) : make_uint4(0u, 0u, 0u, 0u);
      uint32_t* d = &s_rows[p][4 * c];
      d[0] = v.x;
      d[1] = v.y;
      d[2] = v.z;
      d[3] = v.w;
    }
    __syncthreads();
  }

  const int ly = threadIdx.x / kTX, lx = threadIdx.x % kTX;
  const int y = ty0 + ly, x = tx0 + lx;
  unsigned long long e2 = 0, g2 = 0;
  if (y < H && x < W) {
    uint32_t sum[C] = {};
    uint32_t cnt = 0;
#pragma unroll 2
    for (int dy = 0; dy < kPatch; ++dy) {
#pragma unroll
      for (int dx = 0; dx < kPatch; ++dx) {
        const int pr = ly + 7 - dy, pc = lx + 7 - dx;       // patch (y - dy, x - dx)
        const int32_t r = s_f[pr][pc];
        if (r >= 0) {
          if (C == 1) {
            sum[0] += (s_rows[pr * kPX + pc][dy * 2 + (dx >> 2)] >> (8 * (dx & 3))) & 0xffu;
          } else {
            const uint8_t* p = a.R + (int64_t)r * D + (dy * kPatch + dx) * C;
#pragma unroll
            for (int c = 0; c < C; ++c) sum[c] += __ldg(p + c);
          }
          ++cnt;
        }
      }
    }
    const int64_t o = ((int64_t)y * W + x) * C;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const uint32_t v = cnt ? (2u * sum[c] + cnt) / (2u * cnt) : 0u;
      if (a.out) a.out[o + c] = (uint8_t)v;
      if (a.frame) {
        const int f = a.frame[o + c];
        const int d = f - (int)v;
        e2 += (unsigned long long)(d * d);
        g2 += (unsigned long long)(f * f);
      }
    }
  }
  if (a.err2) {
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
      e2 += __shfl_xor_sync(0xffffffffu, e2, s);
      g2 += __shfl_xor_sync(0xffffffffu, g2, s);
    }
    if ((threadIdx.x & 31) == 0) {
      s_red[0][threadIdx.x >> 5] = e2;
      s_red[1][threadIdx.x >> 5] = g2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long te = 0, tg = 0;
      for (int w = 0; w < kTY * kTX / 32; ++w) {
        te += s_red[0][w];
        tg += s_red[1][w];
      }
      atomicAdd(a.err2, te);
      atomicAdd(a.err2 + 1, tg);
    }
  }
}

}  // namespace

cudaError_t launch_reconstruct(const ReconArgs& a, int C, cudaStream_t s) {
  if (a.err2) {
    const cudaError_t e = cudaMemsetAsync(a.err2, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
  }
  const dim3 grid((unsigned)((a.W + kTX - 1) / kTX), (unsigned)((a.H + kTY - 1) / kTY));
  if (C == 1) k_reconstruct<1><<<grid, kTY * kTX, 0, s>>>(a);
  else k_reconstruct<3><<<grid, kTY * kTX, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace riann
