// api.cu -- the C ABI of include/riann.h: argument checks, device memory of
// the index and its scratch, and the launch sequence of one frame.
#include <cstdio>
#include <cstring>
#include <new>

#include "common.cuh"

namespace riann {


int sm_count() {
  static int cached = 0;
  if (!cached) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached = v > 0 ? v : 1;
  }
  return cached;
}

cudaError_t launch_dense(const DenseArgs& a, Index& ix, cudaStream_t s) {
  return launch_dense_tc(a, ix, s);
}

void prof_begin(Index& ix, int slot, cudaStream_t s) {
  if (!ix.profile) return;
  cudaEventRecord(ix.prof_ev[slot][0], s);
}

void prof_end(Index& ix, int slot, cudaStream_t s) {
  if (!ix.profile) return;
  cudaEventRecord(ix.prof_ev[slot][1], s);
  ix.prof_recorded[slot] = true;
}

namespace {

int from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return RIANN_OK;
  if (e == cudaErrorMemoryAllocation) return RIANN_ERR_OOM;
  return RIANN_ERR_CUDA;
}

template <class T>
cudaError_t dalloc(T** p, size_t count, size_t& total) {
  const size_t bytes = sizeof(T) * (count ? count : 1);
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e == cudaSuccess) total += bytes;
  return e;
}

void free_scratch(Index& ix) {
  cudaFree(ix.dense_list);
  cudaFree(ix.dense_count);
  cudaFree(ix.best);
  cudaFree(ix.Aq);
  cudaFree(ix.qnorm);
  ix.qnorm = nullptr;
  ix.dense_list = nullptr;
  ix.dense_count = nullptr;
  ix.best = nullptr;
  ix.Aq = nullptr;
  ix.scratch_q = 0;
}

void free_index(Index* ix) {
  if (!ix) return;
  cudaFree(ix->R);
  cudaFree(ix->KP);
  cudaFree(ix->Rbf);
  cudaFree(ix->rnorm);
  cudaFree(ix->P);
  cudaFree(ix->TA);
  cudaFree(ix->Tid);
  cudaFree(ix->E);
  cudaFree(ix->RB);
  cudaFree(ix->CW);
  cudaFree(ix->CWE);
  cudaFree(ix->status);
  cudaFree(ix->stats);
  for (int k = 0; k < kSlots; ++k)
    for (int j = 0; j < 2; ++j)
      if (ix->prof_ev[k][j]) cudaEventDestroy(ix->prof_ev[k][j]);
  free_scratch(*ix);
  delete ix;
}

// Grow the index scratch to hold Q queries.  Allocation synchronises the device.
int ensure_scratch(Index& ix, int64_t Q) {
  if (ix.scratch_q >= Q) return RIANN_OK;
  free_scratch(ix);
  size_t dummy = 0;
  const int64_t Qpad = (Q + kDenseTileM - 1) / kDenseTileM * kDenseTileM;
  cudaError_t e = dalloc(&ix.dense_list, (size_t)Q, dummy);
  if (e == cudaSuccess) e = dalloc(&ix.dense_count, 1, dummy);
  if (e == cudaSuccess) e = dalloc(&ix.best, (size_t)Q, dummy);
  if (e == cudaSuccess) e = dalloc(&ix.Aq, (size_t)Qpad * ix.D, dummy);
  if (e == cudaSuccess) e = dalloc(&ix.qnorm, (size_t)Qpad, dummy);
  if (e != cudaSuccess) {
    free_scratch(ix);
    cudaGetLastError();
    return from_cuda(e);
  }
  if (!make_row_map(&ix.tmAq, ix.Aq, (uint64_t)Qpad, ix.D, kDenseTileM)) {
    free_scratch(ix);
    return RIANN_ERR_UNSUPPORTED;
  }
  ix.scratch_q = Q;
  return RIANN_OK;
}

bool params_ok(const riann_params* p) {
  return p && p->alpha_den >= 1 && p->alpha_den <= 8 && p->alpha_num >= 0 &&
         p->alpha_num <= 8 * p->alpha_den && p->ring_limit >= -1 && p->cap >= 0;
}

bool frame_ok(int32_t H, int32_t W) {
  return H >= kPatch && W >= kPatch && (int64_t)(H - 7) * (int64_t)(W - 7) < (int64_t)INT32_MAX &&
         (int64_t)H * W * 3 < ((int64_t)1 << 40);
}

}  // namespace
}  // namespace riann

using namespace riann;

struct riann_index_s : public Index {};

extern "C" {

riann_params riann_default_params(int32_t n) {
  riann_params p;
  p.alpha_num = 1;
  p.alpha_den = 4;
  p.ring_limit = n / 8;
  p.cap = 0;
  return p;
}

const char* riann_strerror(int code) {
  switch (code) {
    case RIANN_OK: return "ok";
    case RIANN_ERR_INVALID_ARG: return "invalid argument";
    case RIANN_ERR_OOM: return "out of memory";
    case RIANN_ERR_UNSUPPORTED: return "unsupported device or feature";
    case RIANN_ERR_CUDA: return "CUDA runtime error";
    case RIANN_ERR_TIMEOUT: return "bounded device wait timed out";
    case RIANN_ERR_ADMISSION: return "admission rejected: budget exceeded";
    case RIANN_ERR_DEVICE: return "kernel reported invalid input (see status bits)";
    case RIANN_ERR_TOO_LARGE: return "frame has more queries than the fixed scratch of riann_exact_nn_noalloc holds";
    default: return "unknown error";
  }
}

int riann_build_reference_index(const uint8_t* d_patches, int32_t n, int32_t channels,
                                const uint8_t* d_keypoints, int32_t K, riann_stream_t stream,
                                riann_index_t* out) {
  if (!out) return RIANN_ERR_INVALID_ARG;
  *out = nullptr;
  if (!d_patches || !d_keypoints || n < 1 || n > (1 << 24) || K < 1 || K > kMaxK ||
      (channels != 1 && channels != 3))
    return RIANN_ERR_INVALID_ARG;
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RIANN_ERR_CUDA;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10 || minor != 3) return RIANN_ERR_UNSUPPORTED;

  riann_index_s* ix = new (std::nothrow) riann_index_s();
  if (!ix) return RIANN_ERR_OOM;
  ix->device = dev;
  ix->n = n;
  ix->K = K;
  ix->C = channels;
  ix->D = 64 * channels;
  ix->n_pad = (n + kDenseTileN - 1) / kDenseTileN * kDenseTileN;
  ix->Kp = (K + 3) / 4 * 4;
  ix->G = (K + 3) / 4;
  ix->GP = (ix->G + 3) / 4 * 4;
  ix->nw = (n + 3) / 4 * 4;
  const int D = ix->D;
  size_t& tot = ix->device_bytes;
  cudaError_t e = dalloc(&ix->R, (size_t)n * D, tot);
  if (e == cudaSuccess) e = dalloc(&ix->KP, (size_t)K * D, tot);
  if (e == cudaSuccess) e = dalloc(&ix->Rbf, (size_t)ix->n_pad * D, tot);
  if (e == cudaSuccess) e = dalloc(&ix->rnorm, (size_t)ix->n_pad, tot);
  if (e == cudaSuccess) e = dalloc(&ix->P, (size_t)n * ix->Kp, tot);
  if (e == cudaSuccess) e = dalloc(&ix->TA, (size_t)n * K, tot);
  if (e == cudaSuccess) e = dalloc(&ix->Tid, (size_t)n * K, tot);
  if (e == cudaSuccess) e = dalloc(&ix->E, (size_t)K * kBuckets, tot);
  if (e == cudaSuccess) e = dalloc(&ix->RB, (size_t)K * (kBuckets + 1), tot);
  if (e == cudaSuccess) e = dalloc(&ix->CW, (size_t)K * ix->G * ix->nw, tot);
  if (e == cudaSuccess) e = dalloc(&ix->CWE, (size_t)K * ix->GP * n, tot);
  if (e == cudaSuccess) e = dalloc(&ix->status, 1, tot);
  if (e == cudaSuccess) e = dalloc(&ix->stats, kStats, tot);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(ix->status, 0, sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ix->stats, 0, sizeof(unsigned long long) * kStats, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ix->R, d_patches, (size_t)n * D, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ix->KP, d_keypoints, (size_t)K * D, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = launch_index_build(*ix, s);
  if (e == cudaSuccess &&
      !make_row_map(&ix->tmRbf, ix->Rbf, (uint64_t)ix->n_pad, D, dense_ref_rows_per_tile(channels))) {
    cudaStreamSynchronize(s);
    free_index(ix);
    return RIANN_ERR_UNSUPPORTED;
  }
  ix->tm_ready = true;
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaStreamSynchronize(s);
    free_index(ix);
    return from_cuda(e);
  }
  *out = ix;
  return RIANN_OK;
}

void riann_index_destroy(riann_index_t idx) {
  if (!idx) return;
  cudaDeviceSynchronize();
  free_index(idx);
}

int riann_index_info(riann_index_t idx, riann_index_info_t* out) {
  if (!idx || !out) return RIANN_ERR_INVALID_ARG;
  out->n = idx->n;
  out->K = idx->K;
  out->channels = idx->C;
  out->dim = idx->D;
  out->device_bytes = idx->device_bytes;
  return RIANN_OK;
}

int riann_index_tables(riann_index_t idx, riann_stream_t stream, uint32_t* P, uint32_t* TA,
                       int32_t* Tid) {
  if (!idx) return RIANN_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t cnt = (size_t)idx->n * idx->K;
  cudaError_t e = cudaSuccess;
  if (P)
    e = cudaMemcpy2DAsync(P, sizeof(uint32_t) * idx->K, idx->P, sizeof(uint32_t) * idx->Kp,
                          sizeof(uint32_t) * idx->K, (size_t)idx->n, cudaMemcpyDefault, s);
  if (e == cudaSuccess && TA) e = cudaMemcpyAsync(TA, idx->TA, cnt * sizeof(uint32_t), cudaMemcpyDefault, s);
  if (e == cudaSuccess && Tid) e = cudaMemcpyAsync(Tid, idx->Tid, cnt * sizeof(int32_t), cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return from_cuda(e);
}

int riann_annf_frame(riann_index_t idx, const riann_params* p, riann_stream_t stream,
                     const uint8_t* d_frame, int32_t H, int32_t W, const int32_t* d_prev_annf,
                     int32_t* d_out_annf, uint32_t* d_out_dist, uint32_t* d_out_count) {
  if (!idx || !params_ok(p) || !d_frame || !d_out_annf || !frame_ok(H, W) ||
      (const void*)d_prev_annf == (const void*)d_out_annf)
    return RIANN_ERR_INVALID_ARG;
  Index& ix = *idx;
  std::lock_guard<std::mutex> lock(ix.mu);
  const int Hq = H - 7, Wq = W - 7;
  const int64_t Q = (int64_t)Hq * Wq;
  int rc = ensure_scratch(ix, Q);
  if (rc) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e0 = cudaMemsetAsync(ix.stats, 0, sizeof(unsigned long long) * kStats, s);
  if (e0 != cudaSuccess) return from_cuda(e0);

  DenseArgs da;
  da.frame = d_frame;
  da.H = H;
  da.W = W;
  da.Hq = Hq;
  da.Wq = Wq;
  da.Q = Q;
  da.out_annf = d_out_annf;
  da.out_dist = d_out_dist;
  da.out_count = d_out_count;
  da.R = ix.R;
  da.n = ix.n;
  da.stats = ix.stats;
  if (!d_prev_annf) {
    da.list = nullptr;
    da.list_count = nullptr;
    return from_cuda(launch_dense(da, ix, s));
  }
  cudaError_t e = cudaMemsetAsync(ix.dense_count, 0, sizeof(uint32_t), s);
  if (e != cudaSuccess) return from_cuda(e);
  SparseArgs sa;
  sa.frame = d_frame;
  sa.H = H;
  sa.W = W;
  sa.Hq = Hq;
  sa.Wq = Wq;
  sa.prev = d_prev_annf;
  sa.out_annf = d_out_annf;
  sa.out_dist = d_out_dist;
  sa.out_count = d_out_count;
  sa.R = ix.R;
  sa.KP = ix.KP;
  sa.P = ix.P;
  sa.TA = ix.TA;
  sa.Tid = ix.Tid;
  sa.E = ix.E;
  sa.RB = ix.RB;
  sa.CW = ix.CW;
  sa.CWE = ix.CWE;
  sa.GP = ix.GP;
  sa.nw = ix.nw;
  sa.n = ix.n;
  sa.K = ix.K;
  sa.Kp = ix.Kp;
  sa.G = ix.G;
  sa.alpha_num = p->alpha_num;
  sa.alpha_den = p->alpha_den;
  sa.ring_limit = p->ring_limit;
  sa.dense_list = ix.dense_list;
  sa.dense_count = ix.dense_count;
  sa.status = ix.status;
  sa.stats = ix.stats;
  prof_begin(ix, kSlotSparse, s);
  e = launch_sparse(sa, ix.C, s);
  prof_end(ix, kSlotSparse, s);
  if (e != cudaSuccess) return from_cuda(e);
  if (p->ring_limit >= 0) {
    da.list = ix.dense_list;
    da.list_count = ix.dense_count;
    e = launch_dense(da, ix, s);
  }
  return from_cuda(e);
}

int riann_exact_nn(riann_index_t idx, riann_stream_t stream, const uint8_t* d_frame, int32_t H,
                   int32_t W, int32_t* d_out_annf, uint32_t* d_out_dist) {
  if (!idx || !d_frame || !d_out_annf || !frame_ok(H, W)) return RIANN_ERR_INVALID_ARG;
  Index& ix = *idx;
  std::lock_guard<std::mutex> lock(ix.mu);
  const int64_t Q = (int64_t)(H - 7) * (W - 7);
  int rc = ensure_scratch(ix, Q);
  if (rc) return rc;
  DenseArgs da;
  da.frame = d_frame;
  da.H = H;
  da.W = W;
  da.Hq = H - 7;
  da.Wq = W - 7;
  da.Q = Q;
  da.list = nullptr;
  da.list_count = nullptr;
  da.out_annf = d_out_annf;
  da.out_dist = d_out_dist;
  da.out_count = nullptr;
  da.R = ix.R;
  da.n = ix.n;
  da.stats = nullptr;
  return from_cuda(launch_dense(da, ix, reinterpret_cast<cudaStream_t>(stream)));
}

int riann_frame_stats(riann_index_t idx, riann_stream_t stream, riann_frame_stats_t* out) {
  if (!idx || !out) return RIANN_ERR_INVALID_ARG;
  unsigned long long v[kStats];
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(v, idx->stats, sizeof(v), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return from_cuda(e);
  out->ring_queries = v[kStatRingQueries];
  out->dense_queries = v[kStatDenseQueries];
  out->sum_seed = v[kStatSumSeed];
  out->sum_candidates = v[kStatSumS];
  return RIANN_OK;
}

int riann_profile_enable(riann_index_t idx, int on) {
  if (!idx) return RIANN_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(idx->mu);
  if (on) {
    for (int k = 0; k < kSlots; ++k)
      for (int j = 0; j < 2; ++j)
        if (!idx->prof_ev[k][j]) {
          cudaError_t e = cudaEventCreate(&idx->prof_ev[k][j]);
          if (e != cudaSuccess) return from_cuda(e);
        }
  }
  idx->profile = on != 0;
  for (int k = 0; k < kSlots; ++k) idx->prof_recorded[k] = false;
  return RIANN_OK;
}

int riann_profile_read(riann_index_t idx, riann_stream_t stream, float* ms, int32_t nslots) {
  if (!idx || !ms || nslots < 1) return RIANN_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(idx->mu);
  cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return from_cuda(e);
  for (int k = 0; k < nslots; ++k) {
    ms[k] = -1.f;
    if (k < kSlots && idx->profile && idx->prof_recorded[k]) {
      e = cudaEventElapsedTime(&ms[k], idx->prof_ev[k][0], idx->prof_ev[k][1]);
      if (e != cudaSuccess) return from_cuda(e);
      idx->prof_recorded[k] = false;
    }
  }
  return RIANN_OK;
}

int64_t riann_exact_nn_noalloc_max_queries(int32_t channels) {
  if (channels != 1 && channels != 3) return 0;
  return noalloc_max_queries(channels);
}

int riann_exact_nn_noalloc(riann_index_t idx, riann_stream_t stream, const uint8_t* d_frame, int32_t H,
                           int32_t W, int32_t* d_out_annf, uint32_t* d_out_dist) {
  if (!idx || !d_frame || !d_out_annf || !frame_ok(H, W)) return RIANN_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return RIANN_ERR_CUDA;
  if (dev != idx->device) return RIANN_ERR_INVALID_ARG;
  const int64_t Q = (int64_t)(H - 7) * (W - 7);
  if (Q > noalloc_max_queries(idx->C)) return RIANN_ERR_TOO_LARGE;
  DenseArgs da;
  da.frame = d_frame;
  da.H = H;
  da.W = W;
  da.Hq = H - 7;
  da.Wq = W - 7;
  da.Q = Q;
  da.list = nullptr;
  da.list_count = nullptr;
  da.out_annf = d_out_annf;
  da.out_dist = d_out_dist;
  da.out_count = nullptr;
  da.R = idx->R;
  da.n = idx->n;
  da.stats = nullptr;
  cudaError_t e = launch_exact_nn_noalloc(da, *idx, reinterpret_cast<cudaStream_t>(stream));
  if (e == cudaErrorInvalidValue) return RIANN_ERR_TOO_LARGE;
  if (e == cudaErrorNotSupported) return RIANN_ERR_UNSUPPORTED;
  return from_cuda(e);
}

int riann_status(riann_index_t idx, riann_stream_t stream, uint32_t* bits) {
  if (!idx) return RIANN_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  uint32_t v = 0;
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemcpy(&v, idx->status, sizeof(v), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && v) e = cudaMemset(idx->status, 0, sizeof(uint32_t));
  if (bits) *bits = v;
  if (e != cudaSuccess) return from_cuda(e);
  return v ? RIANN_ERR_DEVICE : RIANN_OK;
}

}  // extern "C"
