// stack.cu -- 3-D spatio-temporal patches (Sec. 1: the method extends from 2-D
// patches to 8 x 8 x T volumes).  Three consecutive gray frames are
// interleaved into one 3-channel frame, out[y][x][tau] = f_tau[y][x] (tau = 0
// the oldest), so that the query patch at (y, x) in (dy, dx, c) order is the
// volume in (dy, dx, tau) order and every later step runs unchanged on a
// 3-channel index of reference volumes.
//
// HBM-bound: 3 H W bytes in, 3 H W bytes out.  A thread takes 4 pixels: one
// 32-bit load per frame, three 32-bit stores; the ragged tail (H W not a
// multiple of 4, or unaligned pointers) goes byte by byte.
#include "common.cuh"

namespace riann {
namespace {

__global__ void k_stack3(const uint8_t* __restrict__ f0, const uint8_t* __restrict__ f1,
                         const uint8_t* __restrict__ f2, int64_t npix, bool vec, uint8_t* __restrict__ out) {
  const int64_t nv = vec ? npix / 4 : 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) {
    const uint32_t a = __ldg(reinterpret_cast<const uint32_t*>(f0) + i);
    const uint32_t b = __ldg(reinterpret_cast<const uint32_t*>(f1) + i);
    const uint32_t c = __ldg(reinterpret_cast<const uint32_t*>(f2) + i);
    // bytes out: a0 b0 c0 a1 | b1 c1 a2 b2 | c2 a3 b3 c3
    const uint32_t w0 = __byte_perm(__byte_perm(a, b, 0x0140), c, 0x2410);   // a0 b0 a1 . -> a0 b0 c0 a1
    const uint32_t w1 = __byte_perm(__byte_perm(b, c, 0x0251), a, 0x2610);   // b1 c1 b2 . -> b1 c1 a2 b2
    const uint32_t w2 = __byte_perm(__byte_perm(c, a, 0x0372), b, 0x2710);   // c2 a3 c3 . -> c2 a3 b3 c3
    uint32_t* o = reinterpret_cast<uint32_t*>(out) + 3 * i;
    o[0] = w0;
    o[1] = w1;
    o[2] = w2;
  }
  for (int64_t p = 4 * nv + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += stride) {
    out[3 * p + 0] = f0[p];
    out[3 * p + 1] = f1[p];
    out[3 * p + 2] = f2[p];
  }
}

}  // namespace

cudaError_t launch_stack3(const uint8_t* f0, const uint8_t* f1, const uint8_t* f2, int64_t npix, uint8_t* out,
                          cudaStream_t s) {
  const bool vec = ((reinterpret_cast<uintptr_t>(f0) | reinterpret_cast<uintptr_t>(f1) |
                     reinterpret_cast<uintptr_t>(f2) | reinterpret_cast<uintptr_t>(out)) & 3) == 0;
  int64_t blocks = (npix / 4 + 255) / 256;
  const int64_t cap = (int64_t)sm_count() * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  k_stack3<<<(unsigned)blocks, 256, 0, s>>>(f0, f1, f2, npix, vec, out);
  return cudaGetLastError();
}

}  // namespace riann
