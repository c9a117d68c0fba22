// reconstruct.cuh -- declarations of the Sec. 4 reconstruction kernel.
#pragma once

#include "common.cuh"

namespace riann {

// Arguments of the reconstruction kernel (Sec. 4 patch replacement).
struct ReconArgs {
  const int32_t* annf;            // [H-7][W-7]
  const uint8_t* R;
  int n;
  int32_t H, W;
  const uint8_t* frame;           // nullable: f_GT
  uint8_t* out;                   // nullable: f_R
  unsigned long long* err2;       // nullable: [2] sum (f_GT - f_R)^2, sum f_GT^2
  uint32_t* status;
};

cudaError_t launch_reconstruct(const ReconArgs& a, int C, cudaStream_t s);

}  // namespace riann
