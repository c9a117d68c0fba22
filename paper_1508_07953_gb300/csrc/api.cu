// api.cu -- the C ABI of include/riann.h: argument checks, device memory of
// the index, per-call workspaces, the launch sequence of a frame or a batch of
// frames, per-stream sessions (the previous field kept on the device, Alg. 1
// line "r_i = ANNF^(t-1)(x, y)"), batch contexts replayed as CUDA graphs, and
// the ring-kernel autotuner.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "reconstruct.cuh"
#include "anchor.cuh"
#include "trace.h"

namespace riann {

// SM count of the current device (cached per device).
int sm_count() {
  constexpr int kDevices = 64;
  static std::atomic<int> cached[kDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevices) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
  }
  int c = cached[dev].load(std::memory_order_relaxed);
  if (!c) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    c = v > 0 ? v : 1;
    cached[dev].store(c, std::memory_order_relaxed);
  }
  return c;
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

bool params_ok(const riann_params* p) {
  return p && p->alpha_den >= 1 && p->alpha_den <= 8 && p->alpha_num >= 0 &&
         p->alpha_num <= 8 * p->alpha_den && p->ring_limit >= -1 && p->cap >= 0 && p->cap <= kMaxScanDepth;
}

bool frame_ok(int32_t H, int32_t W) {
  return H >= kPatch && W >= kPatch && (int64_t)(H - 7) * (int64_t)(W - 7) < (int64_t)INT32_MAX &&
         (int64_t)H * W * 3 < ((int64_t)1 << 40);
}

FrameItem make_item(const uint8_t* frame, const int32_t* prev, int32_t* out, uint32_t* dist, uint32_t* count,
                    int H, int W, int shape) {
  FrameItem it;
  it.frame = frame;
  it.prev = prev;
  it.out_annf = out;
  it.out_dist = dist;
  it.out_count = count;
  it.H = H;
  it.W = W;
  it.Hq = H - 7;
  it.Wq = W - 7;
  it.tiles_x = (it.Wq + ring_tile_cols(shape) - 1) / ring_tile_cols(shape);
  it.query_begin = 0;
  return it;
}

int item_tiles(const FrameItem& it, int shape) {
  return it.tiles_x * ((it.Hq + ring_tile_rows(shape) - 1) / ring_tile_rows(shape));
}

SparseArgs sparse_args(const Index& ix, const riann_params* p, Workspace& ws, unsigned long long* stats) {
  SparseArgs sa;
  std::memset(&sa, 0, sizeof(sa));
  sa.R = ix.R;
  sa.KP = ix.KP;
  sa.P = ix.P;
  sa.TA = ix.TA;
  sa.Tid = ix.Tid;
  sa.E = ix.E;
  sa.RB = ix.RB;
  sa.partner = ix.partner;
  sa.Tid2 = ix.Tid2;
  sa.OFF = ix.OFF;
  sa.CW = ix.CW;
  sa.CE = ix.CE;
  sa.Ke = ix.Ke;
  sa.n = ix.n;
  sa.K = ix.K;
  sa.Kp = ix.Kp;
  sa.G = ix.G;
  sa.nw = ix.nw;
  sa.alpha_num = p->alpha_num;
  sa.alpha_den = p->alpha_den;
  sa.ring_limit = p->ring_limit;
  sa.depth = p->cap ? p->cap : ix.depth;
  sa.unit = ix.unit ? 1 : 0;
  sa.Rf = ix.Rf;
  sa.KPf = ix.KPf;
  sa.dense_list = ws.dense_list;
  sa.counters = ws.counters;
  sa.status = ix.status;
  sa.stats = stats;
  return sa;
}

DenseArgs dense_args(const Index& ix, unsigned long long* stats) {
  DenseArgs da;
  std::memset(&da, 0, sizeof(da));
  da.R = ix.R;
  da.n = ix.n;
  da.stats = stats;
  return da;
}

// One frame on a workspace: brute force when there is no previous field,
// else the ring kernel followed by brute force for the queries it routed.
// k > 0: also the k-NN output (knn_idx, knn_dist [Q][k]).
cudaError_t run_frame(Index& ix, Workspace& ws, const riann_params* p, cudaStream_t s, const FrameItem& it,
                      unsigned long long* stats, int k = 0, int32_t* knn_idx = nullptr,
                      uint32_t* knn_dist = nullptr) {
  NvtxRange range(k ? "riann k-NN frame" : "riann frame");
  cudaError_t e = cudaSuccess;
  if (stats) e = cudaMemsetAsync(stats, 0, sizeof(unsigned long long) * kStats, s);
  if (e != cudaSuccess) return e;
  const int64_t Q = (int64_t)it.Hq * it.Wq;
  DenseArgs da = dense_args(ix, stats);
  da.one = it;
  da.Q = Q;
  da.knn = k;
  da.knn_idx = knn_idx;
  da.knn_dist = knn_dist;
  if (!it.prev) {
    da.list = nullptr;
    da.list_count = nullptr;
    return ix.unit ? launch_dense_unit(da, ix, s) : launch_dense_tc(da, ix, ws, s);
  }
  e = cudaMemsetAsync(ws.counters, 0, sizeof(uint32_t) * 4, s);
  if (e != cudaSuccess) return e;
  SparseArgs sa = sparse_args(ix, p, ws, stats);
  sa.one = it;
  sa.knn = k;
  sa.knn_idx = knn_idx;
  sa.knn_dist = knn_dist;
  prof_begin(ix, kSlotSparse, s);
  e = launch_sparse(sa, ix.C, ix.tile_shape, s);
  prof_end(ix, kSlotSparse, s);
  if (e != cudaSuccess || p->ring_limit < 0) return e;
  da.list = ws.dense_list;
  da.list_count = ws.counters;
  return ix.unit ? launch_dense_unit(da, ix, s) : launch_dense_tc(da, ix, ws, s);
}

void free_index(Index* ix) {
  if (!ix) return;
  cudaFree(ix->R);
  cudaFree(ix->KP);
  cudaFree(ix->Rbf);
  cudaFree(ix->RN);
  cudaFree(ix->rnorm);
  cudaFree(ix->P);
  cudaFree(ix->TA);
  cudaFree(ix->Tid);
  cudaFree(ix->E);
  cudaFree(ix->RB);
  cudaFree(ix->partner);
  cudaFree(ix->Tid2);
  cudaFree(ix->OFF);
  cudaFree(ix->CW);
  cudaFree(ix->CE);
  cudaFree(ix->Rf);
  cudaFree(ix->KPf);
  cudaFree(ix->status);
  cudaFree(ix->stats);
  for (int k = 0; k < kSlots; ++k)
    for (int j = 0; j < 2; ++j)
      if (ix->prof_ev[k][j]) cudaEventDestroy(ix->prof_ev[k][j]);
  free_workspace(ix->ws);
  delete ix;
}

}  // namespace

void free_workspace(Workspace& ws) {
  cudaFree(ws.dense_list);
  cudaFree(ws.counters);
  cudaFree(ws.best);
  cudaFree(ws.Aq);
  cudaFree(ws.qnorm);
  cudaFree(ws.knn_lists);
  ws.knn_lists = nullptr;
  ws.knn_cap = 0;
  ws.dense_list = nullptr;
  ws.counters = nullptr;
  ws.best = nullptr;
  ws.Aq = nullptr;
  ws.qnorm = nullptr;
  ws.cap_q = 0;
  ws.bytes = 0;
}

int ensure_workspace(Workspace& ws, const Index& ix, int64_t Q) {
  if (ws.cap_q >= Q) return RIANN_OK;
  free_workspace(ws);
  const int64_t Qpad = (Q + kDenseTileM - 1) / kDenseTileM * kDenseTileM;
  size_t& b = ws.bytes;
  cudaError_t e = dalloc(&ws.dense_list, (size_t)Q, b);
  if (e == cudaSuccess) e = dalloc(&ws.counters, 4, b);
  if (e == cudaSuccess) e = dalloc(&ws.best, (size_t)Q, b);
  if (e == cudaSuccess) e = dalloc(&ws.Aq, (size_t)Qpad * ix.D, b);
  if (e == cudaSuccess) e = dalloc(&ws.qnorm, (size_t)Qpad, b);
  if (e != cudaSuccess) {
    free_workspace(ws);
    cudaGetLastError();
    return from_cuda(e);
  }
  if (!make_row_map(&ws.tmAq, ws.Aq, (uint64_t)Qpad, ix.D, kDenseTileM)) {
    free_workspace(ws);
    return RIANN_ERR_UNSUPPORTED;
  }
  ws.cap_q = Q;
  return RIANN_OK;
}

int ensure_knn_lists(Workspace& ws, int64_t Q) {
  const int64_t need = dense_knn_list_entries(Q);
  if (ws.knn_cap >= need) return RIANN_OK;
  if (ws.knn_lists) {
    cudaFree(ws.knn_lists);
    ws.bytes -= (size_t)ws.knn_cap * sizeof(unsigned long long);
    ws.knn_lists = nullptr;
    ws.knn_cap = 0;
  }
  const cudaError_t e = dalloc(&ws.knn_lists, (size_t)need, ws.bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return from_cuda(e);
  }
  ws.knn_cap = need;
  return RIANN_OK;
}

}  // namespace riann

using namespace riann;

struct riann_index_s : public Index {};

// Per-stream state (a video stream's previous field, kept on the device).
struct riann_session_s {
  Index* ix = nullptr;
  int H = 0, W = 0;
  int64_t Q = 0;
  Workspace ws;                  // scratch of riann_session_frame
  int32_t* field[2] = {nullptr, nullptr};
  uint32_t* dist = nullptr;
  uint32_t* count = nullptr;
  uint8_t* dframe = nullptr;     // device copy of a frame given in host memory
  int cur = 0;                   // field[cur] holds the latest field
  bool have_prev = false;
  int64_t frames = 0;
  size_t bytes = 0;
  std::mutex mu;
};

constexpr int kBranches = 4;   // streams the ring launches of a batched step are spread over

// A batch context: scratch for the union of its frames, pinned descriptor
// staging, and the captured graph of one batched step.
struct riann_batch_s {
  Index* ix = nullptr;
  int max_items = 0;
  int64_t cap_q = 0;
  bool use_graph = true;
  Workspace ws;
  FrameItem* h_items = nullptr;  // pinned [max_items]
  BatchHeader* h_hdr = nullptr;  // pinned
  FrameItem* d_items = nullptr;
  BatchHeader* d_hdr = nullptr;
  unsigned long long* stats = nullptr;   // [kStats] counters of the last run
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  riann_params gp{};             // parameters baked into the graph
  int g_shape = -1, g_depth = -1;
  int g_items = 0;                     // ring launches of a step ...
  std::vector<int> g_tiles;            // ... and the grid of each (slot i: its largest frame so far)
  int tiles_shape = -1;                // tile shape g_tiles counts in
  cudaStream_t cap_stream = nullptr;   // private stream the graph is captured on
  cudaStream_t branch[kBranches] = {};
  cudaEvent_t fork = nullptr, join[kBranches] = {};
  cudaEvent_t done = nullptr;
  bool pending = false;
  int64_t runs = 0, graph_builds = 0;
  size_t bytes = 0;
  std::mutex mu;
};

namespace {

void free_session(riann_session_s* s) {
  if (!s) return;
  cudaFree(s->field[0]);
  cudaFree(s->field[1]);
  cudaFree(s->dist);
  cudaFree(s->count);
  cudaFree(s->dframe);
  free_workspace(s->ws);
  delete s;
}

void free_batch(riann_batch_s* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->done) cudaEventDestroy(b->done);
  if (b->fork) cudaEventDestroy(b->fork);
  for (int k = 0; k < kBranches; ++k) {
    if (b->join[k]) cudaEventDestroy(b->join[k]);
    if (b->branch[k]) cudaStreamDestroy(b->branch[k]);
  }
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  cudaFreeHost(b->h_items);
  cudaFreeHost(b->h_hdr);
  cudaFree(b->d_items);
  cudaFree(b->d_hdr);
  cudaFree(b->stats);
  free_workspace(b->ws);
  delete b;
}

// The launch sequence of one batched step (captured into the graph): the
// descriptor upload, one ring launch per slot (grid b->g_tiles[i]) spread
// over the branch streams so that the frames' tails overlap, then one
// brute-force launch over the queries of all frames.
cudaError_t enqueue_batch(riann_batch_s* b, const riann_params* p, cudaStream_t s) {
  Index& ix = *b->ix;
  cudaError_t e = cudaMemcpyAsync(b->d_items, b->h_items, sizeof(FrameItem) * b->max_items,
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_hdr, b->h_hdr, sizeof(BatchHeader), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->ws.counters, 0, sizeof(uint32_t) * 4, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->stats, 0, sizeof(unsigned long long) * kStats, s);
  if (e != cudaSuccess) return e;
  SparseArgs sa = sparse_args(ix, p, b->ws, b->stats);
  sa.items = b->d_items;
  sa.hdr = b->d_hdr;
  const int nb = b->g_items < kBranches ? b->g_items : kBranches;
  e = cudaEventRecord(b->fork, s);
  for (int k = 0; k < nb && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->branch[k], b->fork, 0);
  for (int i = 0; i < b->g_items && e == cudaSuccess; ++i) {
    sa.item = i;
    e = launch_sparse_item(sa, ix.C, ix.tile_shape, b->g_tiles[i], b->branch[i % nb]);
  }
  for (int k = 0; k < nb && e == cudaSuccess; ++k) {
    e = cudaEventRecord(b->join[k], b->branch[k]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->join[k], 0);
  }
  if (e != cudaSuccess) return e;
  DenseArgs da = dense_args(ix, b->stats);
  da.items = b->d_items;
  da.hdr = b->d_hdr;
  da.Q = b->cap_q;
  da.list = b->ws.dense_list;
  da.list_count = b->ws.counters;
  return launch_dense_tc(da, ix, b->ws, s);
}

}  // namespace

namespace {

int build_index(const uint8_t* d_patches, int32_t n, int32_t channels, const uint8_t* d_keypoints, int32_t K,
                riann_stream_t stream, bool unit, int scan_order, riann_index_t* out) {
  if (!out) return RIANN_ERR_INVALID_ARG;
  *out = nullptr;
  if (scan_order != RIANN_SCAN_AUTO && scan_order != RIANN_SCAN_PAIRS && scan_order != RIANN_SCAN_SINGLE)
    return RIANN_ERR_INVALID_ARG;
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
  ix->unit = unit;
  ix->pair_scan = scan_order == RIANN_SCAN_PAIRS || (scan_order == RIANN_SCAN_AUTO && n >= kPairMinN);
  ix->n = n;
  ix->K = K;
  ix->C = channels;
  ix->D = 64 * channels;
  ix->n_pad = (n + kDenseTileN - 1) / kDenseTileN * kDenseTileN;
  ix->Kp = (K + 3) / 4 * 4;
  ix->G = (K + 3) / 4;
  // a fourth group in the scan pays once there are 16 or more (measured)
  ix->depth = ix->G >= 16 ? 4 : 3;
  ix->nw = (n + 3) / 4 * 4;
  ix->Ke = (K + 15) / 16 * 16;
  const int D = ix->D;
  size_t& tot = ix->device_bytes;
  cudaError_t e = dalloc(&ix->R, (size_t)n * D, tot);
  if (e == cudaSuccess) e = dalloc(&ix->KP, (size_t)K * D, tot);
  if (e == cudaSuccess) e = dalloc(&ix->Rbf, (size_t)ix->n_pad * D, tot);
  if (e == cudaSuccess) e = dalloc(&ix->RN, (size_t)ix->n_pad * 16, tot);
  if (e == cudaSuccess) e = dalloc(&ix->rnorm, (size_t)ix->n_pad, tot);
  if (e == cudaSuccess) e = dalloc(&ix->P, (size_t)n * ix->Kp, tot);
  if (e == cudaSuccess) e = dalloc(&ix->TA, (size_t)n * K, tot);
  if (e == cudaSuccess) e = dalloc(&ix->Tid, (size_t)n * K, tot);
  if (e == cudaSuccess) e = dalloc(&ix->E, (size_t)K * kBuckets, tot);
  if (e == cudaSuccess) e = dalloc(&ix->RB, (size_t)K * (kBuckets + 1), tot);
  if (e == cudaSuccess) e = dalloc(&ix->partner, (size_t)K, tot);
  if (e == cudaSuccess) e = dalloc(&ix->Tid2, (size_t)n * K, tot);
  if (e == cudaSuccess) e = dalloc(&ix->OFF, (size_t)K * (kPairCodes * kPairCodes + 1), tot);
  if (e == cudaSuccess) e = dalloc(&ix->CW, (size_t)K * ix->G * ix->nw, tot);
  if (e == cudaSuccess) e = dalloc(&ix->CE, (size_t)K * n * ix->Ke, tot);
  if (e == cudaSuccess) e = dalloc(&ix->status, 1, tot);
  if (e == cudaSuccess) e = dalloc(&ix->stats, kStats, tot);
  if (e == cudaSuccess && unit) e = dalloc(&ix->Rf, (size_t)n * D, tot);
  if (e == cudaSuccess && unit) e = dalloc(&ix->KPf, (size_t)K * D, tot);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(ix->status, 0, sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ix->stats, 0, sizeof(unsigned long long) * kStats, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ix->R, d_patches, (size_t)n * D, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ix->KP, d_keypoints, (size_t)K * D, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = launch_index_build(*ix, s);
  if (e == cudaSuccess) e = ring_prepare(channels);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaStreamSynchronize(s);
    free_index(ix);
    return from_cuda(e);
  }
  if (!make_row_map(&ix->tmRbf, ix->Rbf, (uint64_t)ix->n_pad, D, dense_ref_rows_per_tile(channels))) {
    cudaStreamSynchronize(s);
    free_index(ix);
    return RIANN_ERR_UNSUPPORTED;
  }
  ix->tm_ready = true;
  *out = ix;
  return RIANN_OK;
}

}  // namespace

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
    case RIANN_ERR_TOO_LARGE: return "more queries than the fixed scratch or the batch context holds";
    default: return "unknown error";
  }
}


int riann_build_reference_index(const uint8_t* d_patches, int32_t n, int32_t channels,
                                const uint8_t* d_keypoints, int32_t K, riann_stream_t stream,
                                riann_index_t* out) {
  return build_index(d_patches, n, channels, d_keypoints, K, stream, false, RIANN_SCAN_AUTO, out);
}

int riann_build_reference_index_ex(const uint8_t* d_patches, int32_t n, int32_t channels,
                                   const uint8_t* d_keypoints, int32_t K, int32_t scan_order,
                                   riann_stream_t stream, riann_index_t* out) {
  return build_index(d_patches, n, channels, d_keypoints, K, stream, false, scan_order, out);
}

int riann_build_unit_index(const uint8_t* d_patches, int32_t n, int32_t channels, const uint8_t* d_keypoints,
                           int32_t K, riann_stream_t stream, riann_index_t* out) {
  return build_index(d_patches, n, channels, d_keypoints, K, stream, true, RIANN_SCAN_AUTO, out);
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
  out->unit = idx->unit ? 1 : 0;
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

riann_anchor_params riann_default_anchor_params(void) {
  riann_anchor_params p;
  p.alpha_num = 1;
  p.alpha_den = 4;
  p.L = 20;
  p.max_rings = 64;
  p.seed = 0;
  p.frame_id = 0;
  return p;
}

}  // extern "C"

struct riann_full_s {
  riann_index_t idx = nullptr;
  unsigned long long* T = nullptr;   // [n][NP]
  int NP = 0;
  int32_t* scratch = nullptr;        // [resident warps][2][n]
  uint32_t* counter = nullptr;
  unsigned long long* work = nullptr;   // [3] counters of the last frame
  size_t bytes = 0;
};

extern "C" {

int riann_full_create(riann_index_t idx, riann_stream_t stream, riann_full_t* out) {
  if (!idx || !out) return RIANN_ERR_INVALID_ARG;
  *out = nullptr;
  if (idx->unit) return RIANN_ERR_UNSUPPORTED;
  riann_full_s* f = new (std::nothrow) riann_full_s();
  if (!f) return RIANN_ERR_OOM;
  f->idx = idx;
  f->NP = full_table_stride(idx->n);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = dalloc(&f->T, (size_t)idx->n * f->NP, f->bytes);
  if (e == cudaSuccess) e = dalloc(&f->scratch, (size_t)anchor_resident_warps() * 2 * idx->n, f->bytes);
  if (e == cudaSuccess) e = dalloc(&f->counter, 1, f->bytes);
  if (e == cudaSuccess) e = dalloc(&f->work, 3, f->bytes);
  if (e == cudaSuccess) e = build_full_table(*idx, f->T, f->NP, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaStreamSynchronize(s);
    cudaFree(f->T);
    cudaFree(f->scratch);
    cudaFree(f->counter);
    cudaFree(f->work);
    delete f;
    return from_cuda(e);
  }
  *out = f;
  return RIANN_OK;
}

void riann_full_destroy(riann_full_t f) {
  if (!f) return;
  cudaDeviceSynchronize();
  cudaFree(f->T);
  cudaFree(f->scratch);
  cudaFree(f->counter);
  cudaFree(f->work);
  delete f;
}

int riann_random_field(riann_stream_t stream, int32_t H, int32_t W, int32_t n, uint64_t seed, uint32_t frame_id,
                       int32_t* d_out_annf) {
  if (!d_out_annf || !frame_ok(H, W) || n < 1) return RIANN_ERR_INVALID_ARG;
  return from_cuda(launch_random_field((int64_t)(H - 7) * (W - 7), n, seed, frame_id, d_out_annf,
                                       reinterpret_cast<cudaStream_t>(stream)));
}

int riann_anchor_work(riann_full_t f, riann_stream_t stream, uint64_t* out3) {
  if (!f || !out3) return RIANN_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(out3, f->work, 3 * sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return from_cuda(e);
}

int riann_full_table(riann_full_t f, riann_stream_t stream, uint64_t* host_T) {
  if (!f || !host_T) return RIANN_ERR_INVALID_ARG;
  const int n = f->idx->n;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpy2DAsync(host_T, sizeof(uint64_t) * n, f->T, sizeof(uint64_t) * f->NP,
                                    sizeof(uint64_t) * n, (size_t)n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return from_cuda(e);
}

int riann_anchor_frame(riann_full_t f, const riann_anchor_params* p, riann_stream_t stream,
                       const uint8_t* d_frame, int32_t H, int32_t W, const int32_t* d_prev,
                       int32_t* d_out_annf, uint32_t* d_out_dist, uint32_t* d_out_count,
                       uint32_t* d_out_rings) {
  NvtxRange range("riann anchor-loop frame");
  if (!f || !p || !d_frame || !d_out_annf || !frame_ok(H, W) || p->alpha_den < 1 || p->alpha_den > 8 ||
      p->alpha_num < 0 || p->alpha_num > 8 * p->alpha_den || p->L < 1 || p->max_rings < 0 || p->max_rings > 4096 ||
      (const void*)d_prev == (const void*)d_out_annf)
    return RIANN_ERR_INVALID_ARG;
  Index& ix = *f->idx;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int64_t Q = (int64_t)(H - 7) * (W - 7);
  if (!d_prev) {   // no previous field: brute force (Alg. 1's initialisation read as exact NN)
    int rc = riann_exact_nn(f->idx, stream, d_frame, H, W, d_out_annf, d_out_dist);
    if (rc) return rc;
    cudaError_t e = d_out_count ? launch_fill_u32(d_out_count, Q, (uint32_t)ix.n, s) : cudaSuccess;
    if (e == cudaSuccess && d_out_rings) e = launch_fill_u32(d_out_rings, Q, 0u, s);
    return from_cuda(e);
  }
  AnchorArgs a;
  a.frame = d_frame;
  a.H = H;
  a.W = W;
  a.prev = d_prev;
  a.out_annf = d_out_annf;
  a.out_dist = d_out_dist;
  a.out_count = d_out_count;
  a.out_rings = d_out_rings;
  a.R = ix.R;
  a.n = ix.n;
  a.NP = f->NP;
  a.T = f->T;
  a.alpha_num = p->alpha_num;
  a.alpha_den = p->alpha_den;
  a.L = p->L;
  a.max_rings = p->max_rings;
  a.key0 = (uint32_t)p->seed;
  a.key1 = (uint32_t)(p->seed >> 32);
  a.frame_id = p->frame_id;
  a.scratch = f->scratch;
  a.counter = f->counter;
  a.work = f->work;
  a.status = ix.status;
  return from_cuda(launch_anchor(a, ix.C, s));
}

int riann_reconstruct(riann_index_t idx, riann_stream_t stream, const int32_t* d_annf, int32_t H, int32_t W,
                      const uint8_t* d_frame, uint8_t* d_out, unsigned long long* d_err2) {
  if (!idx || !d_annf || !frame_ok(H, W) || (d_err2 && !d_frame)) return RIANN_ERR_INVALID_ARG;
  ReconArgs a;
  a.annf = d_annf;
  a.R = idx->R;
  a.n = idx->n;
  a.H = H;
  a.W = W;
  a.frame = d_frame;
  a.out = d_out;
  a.err2 = d_err2;
  a.status = idx->status;
  return from_cuda(launch_reconstruct(a, idx->C, reinterpret_cast<cudaStream_t>(stream)));
}

int riann_reconstruct_payload(riann_index_t idx, riann_stream_t stream, const uint8_t* d_payload, int32_t channels,
                              const int32_t* d_annf, int32_t H, int32_t W, const uint8_t* d_frame, uint8_t* d_out,
                              unsigned long long* d_err2) {
  if (!idx || !d_payload || (channels != 1 && channels != 3) || !d_annf || !frame_ok(H, W) ||
      (d_err2 && !d_frame))
    return RIANN_ERR_INVALID_ARG;
  // gray rows are read 16 bytes at a time
  if (reinterpret_cast<uintptr_t>(d_payload) % 16 != 0) return RIANN_ERR_INVALID_ARG;
  ReconArgs a;
  a.annf = d_annf;
  a.R = d_payload;
  a.n = idx->n;
  a.H = H;
  a.W = W;
  a.frame = d_frame;
  a.out = d_out;
  a.err2 = d_err2;
  a.status = idx->status;
  return from_cuda(launch_reconstruct(a, channels, reinterpret_cast<cudaStream_t>(stream)));
}

int riann_annf_frame(riann_index_t idx, const riann_params* p, riann_stream_t stream,
                     const uint8_t* d_frame, int32_t H, int32_t W, const int32_t* d_prev_annf,
                     int32_t* d_out_annf, uint32_t* d_out_dist, uint32_t* d_out_count) {
  if (!idx || !params_ok(p) || !d_frame || !d_out_annf || !frame_ok(H, W) ||
      (const void*)d_prev_annf == (const void*)d_out_annf)
    return RIANN_ERR_INVALID_ARG;
  Index& ix = *idx;
  std::lock_guard<std::mutex> lock(ix.mu);
  const int64_t Q = (int64_t)(H - 7) * (W - 7);
  int rc = ensure_workspace(ix.ws, ix, Q);
  if (rc) return rc;
  const FrameItem it = make_item(d_frame, d_prev_annf, d_out_annf, d_out_dist, d_out_count, H, W, ix.tile_shape);
  return from_cuda(run_frame(ix, ix.ws, p, reinterpret_cast<cudaStream_t>(stream), it, ix.stats));
}

int riann_knn_frame(riann_index_t idx, const riann_params* p, riann_stream_t stream, const uint8_t* d_frame,
                    int32_t H, int32_t W, const int32_t* d_prev_annf, int32_t k, int32_t* d_out_annf,
                    int32_t* d_out_knn, uint32_t* d_out_knn_dist, uint32_t* d_out_count) {
  if (!idx || !params_ok(p) || !d_frame || !d_out_annf || !d_out_knn || !frame_ok(H, W) || k < 1 ||
      k > RIANN_KNN_MAX || (const void*)d_prev_annf == (const void*)d_out_annf ||
      (const void*)d_prev_annf == (const void*)d_out_knn)
    return RIANN_ERR_INVALID_ARG;
  if (idx->unit) return RIANN_ERR_UNSUPPORTED;
  Index& ix = *idx;
  std::lock_guard<std::mutex> lock(ix.mu);
  const int64_t Q = (int64_t)(H - 7) * (W - 7);
  int rc = ensure_workspace(ix.ws, ix, Q);
  if (rc == RIANN_OK) rc = ensure_knn_lists(ix.ws, Q);
  if (rc) return rc;
  const FrameItem it = make_item(d_frame, d_prev_annf, d_out_annf, nullptr, d_out_count, H, W, ix.tile_shape);
  return from_cuda(run_frame(ix, ix.ws, p, reinterpret_cast<cudaStream_t>(stream), it, ix.stats, k, d_out_knn,
                             d_out_knn_dist));
}

int riann_cluster_references(riann_stream_t stream, const uint8_t* d_patches, int32_t n, int32_t channels,
                             int32_t leaf, uint8_t* d_out_reps, int32_t* d_out_assign, int32_t* out_count) {
  if (out_count) *out_count = 0;
  if (!d_patches || !d_out_reps || !out_count || n < 1 || (channels != 1 && channels != 3) || leaf < 1 ||
      (const void*)d_out_reps == (const void*)d_patches)
    return RIANN_ERR_INVALID_ARG;
  return from_cuda(cluster_references(d_patches, n, channels, leaf, d_out_reps, d_out_assign, out_count,
                                      reinterpret_cast<cudaStream_t>(stream)));
}

int riann_stack_frames(riann_stream_t stream, const uint8_t* d_f0, const uint8_t* d_f1, const uint8_t* d_f2,
                       int32_t H, int32_t W, uint8_t* d_out) {
  if (!d_f0 || !d_f1 || !d_f2 || !d_out || H < 1 || W < 1 || (int64_t)H * W >= ((int64_t)1 << 40) ||
      d_out == d_f0 || d_out == d_f1 || d_out == d_f2)
    return RIANN_ERR_INVALID_ARG;
  return from_cuda(launch_stack3(d_f0, d_f1, d_f2, (int64_t)H * W, d_out, reinterpret_cast<cudaStream_t>(stream)));
}

int riann_exact_nn(riann_index_t idx, riann_stream_t stream, const uint8_t* d_frame, int32_t H, int32_t W,
                   int32_t* d_out_annf, uint32_t* d_out_dist) {
  if (!idx || !d_frame || !d_out_annf || !frame_ok(H, W)) return RIANN_ERR_INVALID_ARG;
  Index& ix = *idx;
  std::lock_guard<std::mutex> lock(ix.mu);
  const int64_t Q = (int64_t)(H - 7) * (W - 7);
  int rc = ensure_workspace(ix.ws, ix, Q);
  if (rc) return rc;
  DenseArgs da = dense_args(ix, nullptr);
  da.one = make_item(d_frame, nullptr, d_out_annf, d_out_dist, nullptr, H, W, ix.tile_shape);
  da.Q = Q;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  return from_cuda(ix.unit ? launch_dense_unit(da, ix, cs) : launch_dense_tc(da, ix, ix.ws, cs));
}

int riann_test_wait_expiry(riann_index_t idx, riann_stream_t stream, const uint8_t* d_frame, int32_t H, int32_t W,
                           int32_t* d_out_annf, int64_t spin_cycles) {
  if (!idx || !d_frame || !d_out_annf || !frame_ok(H, W) || spin_cycles < 1000 || spin_cycles > 2000000000LL)
    return RIANN_ERR_INVALID_ARG;
  if (idx->unit) return RIANN_ERR_UNSUPPORTED;
  Index& ix = *idx;
  std::lock_guard<std::mutex> lock(ix.mu);
  const int64_t Q = (int64_t)(H - 7) * (W - 7);
  int rc = ensure_workspace(ix.ws, ix, Q);
  if (rc) return rc;
  DenseArgs da = dense_args(ix, nullptr);
  da.one = make_item(d_frame, nullptr, d_out_annf, nullptr, nullptr, H, W, ix.tile_shape);
  da.Q = Q;
  da.spin_limit = spin_cycles;
  da.withhold = 1;
  return from_cuda(launch_dense_tc(da, ix, ix.ws, reinterpret_cast<cudaStream_t>(stream)));
}

int riann_test_corrupt_offsets(riann_index_t idx, int32_t key, int32_t extra) {
  if (!idx || key < 0 || key >= idx->K - 1 || extra < 1 || extra > 64) return RIANN_ERR_INVALID_ARG;
  if (!idx->pair_scan) return RIANN_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(idx->mu);
  constexpr int kCells = kPairCodes * kPairCodes;
  std::vector<uint32_t> v((size_t)kCells, (uint32_t)(idx->n + extra));
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess)
    e = cudaMemcpy(idx->OFF + (size_t)key * (kCells + 1) + 1, v.data(), sizeof(uint32_t) * kCells,
                   cudaMemcpyHostToDevice);
  return from_cuda(e);
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
  out->sum_filtered = v[kStatSumFiltered];
  out->sum_exact = v[kStatSumExact];
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
  if (idx->unit) return RIANN_ERR_UNSUPPORTED;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return RIANN_ERR_CUDA;
  if (dev != idx->device) return RIANN_ERR_INVALID_ARG;
  const int64_t Q = (int64_t)(H - 7) * (W - 7);
  if (Q > noalloc_max_queries(idx->C)) return RIANN_ERR_TOO_LARGE;
  DenseArgs da = dense_args(*idx, nullptr);
  da.one = make_item(d_frame, nullptr, d_out_annf, d_out_dist, nullptr, H, W, idx->tile_shape);
  da.Q = Q;
  cudaError_t e = launch_exact_nn_noalloc(da, *idx, reinterpret_cast<cudaStream_t>(stream));
  if (e == cudaErrorInvalidValue) return RIANN_ERR_TOO_LARGE;
  if (e == cudaErrorNotSupported) return RIANN_ERR_UNSUPPORTED;
  if (e == cudaErrorStreamCaptureUnsupported) return RIANN_ERR_INVALID_ARG;
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

// ---------------------------------------------------------------------------
// sessions
// ---------------------------------------------------------------------------
int riann_session_create(riann_index_t idx, int32_t H, int32_t W, riann_session_t* out) {
  if (!out) return RIANN_ERR_INVALID_ARG;
  *out = nullptr;
  if (!idx || !frame_ok(H, W)) return RIANN_ERR_INVALID_ARG;
  riann_session_s* s = new (std::nothrow) riann_session_s();
  if (!s) return RIANN_ERR_OOM;
  s->ix = idx;
  s->H = H;
  s->W = W;
  s->Q = (int64_t)(H - 7) * (W - 7);
  cudaError_t e = dalloc(&s->field[0], (size_t)s->Q, s->bytes);
  if (e == cudaSuccess) e = dalloc(&s->field[1], (size_t)s->Q, s->bytes);
  if (e == cudaSuccess) e = dalloc(&s->dist, (size_t)s->Q, s->bytes);
  if (e == cudaSuccess) e = dalloc(&s->count, (size_t)s->Q, s->bytes);
  if (e == cudaSuccess) e = dalloc(&s->dframe, (size_t)H * W * idx->C, s->bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_session(s);
    return from_cuda(e);
  }
  *out = s;
  return RIANN_OK;
}

void riann_session_destroy(riann_session_t s) {
  if (!s) return;
  cudaDeviceSynchronize();
  free_session(s);
}

int riann_session_reset(riann_session_t s) {
  if (!s) return RIANN_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  s->have_prev = false;
  return RIANN_OK;
}

int riann_session_info(riann_session_t s, riann_session_info_t* out) {
  if (!s || !out) return RIANN_ERR_INVALID_ARG;
  out->H = s->H;
  out->W = s->W;
  out->frames = s->frames;
  out->has_field = s->have_prev ? 1 : 0;
  out->device_bytes = s->bytes + s->ws.bytes;
  return RIANN_OK;
}

int64_t riann_session_state_bytes(riann_index_t idx, int32_t H, int32_t W) {
  if (!idx || !frame_ok(H, W)) return 0;
  const int64_t Q = (int64_t)(H - 7) * (W - 7);
  return Q * 16 + (int64_t)H * W * idx->C;
}

int riann_session_frame(riann_session_t s, const riann_params* p, riann_stream_t stream, const uint8_t* d_frame,
                        int32_t* d_out_annf, uint32_t* d_out_dist, uint32_t* d_out_count) {
  if (!s || !params_ok(p) || !d_frame) return RIANN_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  Index& ix = *s->ix;
  int rc = ensure_workspace(s->ws, ix, s->Q);
  if (rc) return rc;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  const int nxt = s->cur ^ 1;
  const FrameItem it = make_item(d_frame, s->have_prev ? s->field[s->cur] : nullptr, s->field[nxt], s->dist,
                                 s->count, s->H, s->W, ix.tile_shape);
  cudaError_t e = run_frame(ix, s->ws, p, cs, it, nullptr);
  const size_t fb = sizeof(int32_t) * (size_t)s->Q;
  if (e == cudaSuccess && d_out_annf) e = cudaMemcpyAsync(d_out_annf, s->field[nxt], fb, cudaMemcpyDeviceToDevice, cs);
  if (e == cudaSuccess && d_out_dist) e = cudaMemcpyAsync(d_out_dist, s->dist, fb, cudaMemcpyDeviceToDevice, cs);
  if (e == cudaSuccess && d_out_count) e = cudaMemcpyAsync(d_out_count, s->count, fb, cudaMemcpyDeviceToDevice, cs);
  if (e != cudaSuccess) return from_cuda(e);
  s->cur = nxt;
  s->have_prev = true;
  ++s->frames;
  return RIANN_OK;
}

int riann_session_frame_host(riann_session_t s, const riann_params* p, riann_stream_t stream, const uint8_t* h_frame,
                             int32_t* h_out_annf, uint32_t* h_out_dist, uint32_t* h_out_count) {
  if (!s || !params_ok(p) || !h_frame || !h_out_annf) return RIANN_ERR_INVALID_ARG;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(s->dframe, h_frame, (size_t)s->H * s->W * s->ix->C, cudaMemcpyHostToDevice, cs);
  if (e != cudaSuccess) return from_cuda(e);
  int rc = riann_session_frame(s, p, stream, s->dframe, nullptr, nullptr, nullptr);
  if (rc) return rc;
  const size_t fb = sizeof(int32_t) * (size_t)s->Q;
  e = cudaMemcpyAsync(h_out_annf, s->field[s->cur], fb, cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess && h_out_dist) e = cudaMemcpyAsync(h_out_dist, s->dist, fb, cudaMemcpyDeviceToHost, cs);
  if (e == cudaSuccess && h_out_count) e = cudaMemcpyAsync(h_out_count, s->count, fb, cudaMemcpyDeviceToHost, cs);
  return from_cuda(e);
}

int riann_session_field(riann_session_t s, riann_stream_t stream, int32_t* out) {
  if (!s || !out) return RIANN_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  if (!s->have_prev) return RIANN_ERR_INVALID_ARG;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(out, s->field[s->cur], sizeof(int32_t) * (size_t)s->Q, cudaMemcpyDefault, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  return from_cuda(e);
}

int riann_session_restore(riann_session_t s, riann_stream_t stream, const int32_t* field) {
  if (!s || !field) return RIANN_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(s->field[s->cur], field, sizeof(int32_t) * (size_t)s->Q, cudaMemcpyDefault, cs);
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e != cudaSuccess) return from_cuda(e);
  s->have_prev = true;
  return RIANN_OK;
}

int riann_session_outputs(riann_session_t s, int32_t** d_annf, uint32_t** d_dist, uint32_t** d_count) {
  if (!s) return RIANN_ERR_INVALID_ARG;
  if (d_annf) *d_annf = s->field[s->cur];
  if (d_dist) *d_dist = s->dist;
  if (d_count) *d_count = s->count;
  return RIANN_OK;
}

uint8_t* riann_session_frame_buffer(riann_session_t s) { return s ? s->dframe : nullptr; }

int riann_session_copy_outputs(riann_session_t s, riann_stream_t stream, int32_t* annf, uint32_t* dist,
                               uint32_t* count) {
  if (!s) return RIANN_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  if (!s->have_prev) return RIANN_ERR_INVALID_ARG;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  const size_t fb = sizeof(int32_t) * (size_t)s->Q;
  cudaError_t e = cudaSuccess;
  if (annf) e = cudaMemcpyAsync(annf, s->field[s->cur], fb, cudaMemcpyDefault, cs);
  if (e == cudaSuccess && dist) e = cudaMemcpyAsync(dist, s->dist, fb, cudaMemcpyDefault, cs);
  if (e == cudaSuccess && count) e = cudaMemcpyAsync(count, s->count, fb, cudaMemcpyDefault, cs);
  return from_cuda(e);
}

// ---------------------------------------------------------------------------
// batch contexts
// ---------------------------------------------------------------------------
int riann_batch_create(riann_index_t idx, int32_t max_items, int64_t max_queries, int32_t flags,
                       riann_batch_t* out) {
  if (!out) return RIANN_ERR_INVALID_ARG;
  *out = nullptr;
  if (!idx || max_items < 1 || max_items > 4096 || max_queries < 1 || max_queries >= INT32_MAX)
    return RIANN_ERR_INVALID_ARG;
  if (idx->unit) return RIANN_ERR_UNSUPPORTED;
  riann_batch_s* b = new (std::nothrow) riann_batch_s();
  if (!b) return RIANN_ERR_OOM;
  b->ix = idx;
  b->max_items = max_items;
  b->cap_q = max_queries;
  b->use_graph = (flags & RIANN_BATCH_NO_GRAPH) == 0;
  int rc = ensure_workspace(b->ws, *idx, max_queries);
  cudaError_t e = rc ? cudaErrorMemoryAllocation : cudaSuccess;
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_items, sizeof(FrameItem) * max_items);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_hdr, sizeof(BatchHeader));
  if (e == cudaSuccess) e = dalloc(&b->d_items, (size_t)max_items, b->bytes);
  if (e == cudaSuccess) e = dalloc(&b->d_hdr, 1, b->bytes);
  if (e == cudaSuccess) e = dalloc(&b->stats, kStats, b->bytes);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int k = 0; k < kBranches && e == cudaSuccess; ++k) {
    e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->branch[k], cudaStreamNonBlocking);
  }
  if (e == cudaSuccess) b->g_tiles.assign((size_t)max_items, 0);
  if (e == cudaSuccess && b->use_graph) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_batch(b);
    return rc ? rc : from_cuda(e);
  }
  std::memset(b->h_items, 0, sizeof(FrameItem) * max_items);
  *out = b;
  return RIANN_OK;
}

void riann_batch_destroy(riann_batch_t b) {
  if (!b) return;
  cudaDeviceSynchronize();
  free_batch(b);
}

int riann_batch_run(riann_batch_t b, const riann_params* p, riann_stream_t stream, riann_session_t* sessions,
                    const uint8_t* const* d_frames, int32_t n) {
  if (!b || !params_ok(p) || !sessions || !d_frames || n < 1 || n > b->max_items) return RIANN_ERR_INVALID_ARG;
  NvtxRange range("riann batched step");
  std::lock_guard<std::mutex> lock(b->mu);
  Index& ix = *b->ix;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  for (int i = 0; i < n; ++i) {
    if (!sessions[i] || sessions[i]->ix != b->ix || !d_frames[i]) return RIANN_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (sessions[j] == sessions[i]) return RIANN_ERR_INVALID_ARG;
  }
  // the previous step's graph has read the staging buffer once its event passed
  if (b->pending) {
    cudaError_t e = cudaEventSynchronize(b->done);
    if (e != cudaSuccess) return from_cuda(e);
    b->pending = false;
  }
  int64_t queries = 0;
  for (int i = 0; i < n; ++i) queries += sessions[i]->Q;
  if (queries > b->cap_q) return RIANN_ERR_TOO_LARGE;
  queries = 0;
  for (int i = 0; i < n; ++i) {
    riann_session_s* s = sessions[i];
    FrameItem it = make_item(d_frames[i], s->have_prev ? s->field[s->cur] : nullptr, s->field[s->cur ^ 1], s->dist,
                             s->count, s->H, s->W, ix.tile_shape);
    it.query_begin = queries;
    queries += s->Q;
    b->h_items[i] = it;
  }
  b->h_hdr->n_items = n;
  b->h_hdr->total_queries = queries;
  // ring launch grids: a slot keeps the grid of its largest frame so far (a
  // smaller frame's extra CTAs leave at once); slots past n stay empty
  if (b->tiles_shape != ix.tile_shape) {
    std::fill(b->g_tiles.begin(), b->g_tiles.end(), 0);
    b->g_items = 0;
    b->tiles_shape = ix.tile_shape;
  }
  bool grown = n > b->g_items;
  for (int i = 0; i < n; ++i) {
    const int t = item_tiles(b->h_items[i], ix.tile_shape);
    if (t > b->g_tiles[i]) {
      b->g_tiles[i] = t;
      grown = true;
    }
  }
  if (n > b->g_items) b->g_items = n;
  for (int i = n; i < b->g_items; ++i) b->h_items[i] = FrameItem{};
  cudaError_t e = cudaSuccess;
  if (b->use_graph) {
    const bool stale = !b->exec || grown || b->gp.alpha_num != p->alpha_num || b->gp.alpha_den != p->alpha_den ||
                       b->gp.ring_limit != p->ring_limit || b->gp.cap != p->cap || b->g_shape != ix.tile_shape ||
                       b->g_depth != ix.depth;
    if (stale) {
      if (b->exec) cudaGraphExecDestroy(b->exec);
      if (b->graph) cudaGraphDestroy(b->graph);
      b->exec = nullptr;
      b->graph = nullptr;
      const bool saved_prof = ix.profile;
      ix.profile = false;   // no profiler events inside the graph
      // capture on the context's own stream (the caller's may be the legacy
      // default stream, which cannot be captured); the graph runs on `cs`
      e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        const cudaError_t e2 = enqueue_batch(b, p, b->cap_stream);
        e = cudaStreamEndCapture(b->cap_stream, &b->graph);
        if (e == cudaSuccess) e = e2;
      }
      ix.profile = saved_prof;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return from_cuda(e);
      }
      b->gp = *p;
      b->g_shape = ix.tile_shape;
      b->g_depth = ix.depth;
      ++b->graph_builds;
    }
    e = cudaGraphLaunch(b->exec, cs);
  } else {
    const bool saved_prof = ix.profile;
    ix.profile = false;
    e = enqueue_batch(b, p, cs);
    ix.profile = saved_prof;
  }
  if (e == cudaSuccess) e = cudaEventRecord(b->done, cs);
  if (e != cudaSuccess) return from_cuda(e);
  b->pending = true;
  ++b->runs;
  for (int i = 0; i < n; ++i) {
    riann_session_s* s = sessions[i];
    s->cur ^= 1;
    s->have_prev = true;
    ++s->frames;
  }
  return RIANN_OK;
}

int riann_batch_stats(riann_batch_t b, riann_stream_t stream, riann_frame_stats_t* out) {
  if (!b || !out) return RIANN_ERR_INVALID_ARG;
  unsigned long long v[kStats];
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(v, b->stats, sizeof(v), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return from_cuda(e);
  out->ring_queries = v[kStatRingQueries];
  out->dense_queries = v[kStatDenseQueries];
  out->sum_seed = v[kStatSumSeed];
  out->sum_candidates = v[kStatSumS];
  out->sum_filtered = v[kStatSumFiltered];
  out->sum_exact = v[kStatSumExact];
  return RIANN_OK;
}

int riann_batch_info(riann_batch_t b, riann_batch_info_t* out) {
  if (!b || !out) return RIANN_ERR_INVALID_ARG;
  out->max_items = b->max_items;
  out->max_queries = b->cap_q;
  out->uses_graph = b->use_graph ? 1 : 0;
  out->runs = b->runs;
  out->graph_builds = b->graph_builds;
  out->device_bytes = b->bytes + b->ws.bytes;
  return RIANN_OK;
}

// ---------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------
int riann_set_tuning(riann_index_t idx, const riann_tuning_t* t) {
  if (!idx || !t || t->tile_shape < 0 || t->tile_shape >= kTileShapes || t->depth < 1 || t->depth > kMaxScanDepth)
    return RIANN_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(idx->mu);
  idx->tile_shape = t->tile_shape;
  idx->depth = t->depth;
  return RIANN_OK;
}

int riann_get_tuning(riann_index_t idx, riann_tuning_t* out) {
  if (!idx || !out) return RIANN_ERR_INVALID_ARG;
  out->tile_shape = idx->tile_shape;
  out->depth = idx->depth;
  out->ms = -1.f;
  return RIANN_OK;
}

int riann_autotune(riann_index_t idx, const riann_params* p, riann_stream_t stream, const uint8_t* d_frame,
                   int32_t H, int32_t W, const int32_t* d_prev_annf, int32_t iters, riann_tuning_t* results,
                   int32_t max_results, int32_t* n_results) {
  if (!idx || !params_ok(p) || !d_frame || !d_prev_annf || !frame_ok(H, W) || iters < 1) return RIANN_ERR_INVALID_ARG;
  Index& ix = *idx;
  std::lock_guard<std::mutex> lock(ix.mu);
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  const int64_t Q = (int64_t)(H - 7) * (W - 7);
  int rc = ensure_workspace(ix.ws, ix, Q);
  if (rc) return rc;
  int32_t* out = nullptr;
  size_t dummy = 0;
  cudaError_t e = dalloc(&out, (size_t)Q, dummy);
  if (e != cudaSuccess) return from_cuda(e);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  riann_params q = *p;
  q.cap = 0;
  std::vector<riann_tuning_t> all;
  const bool saved_prof = ix.profile;
  ix.profile = false;
  const int saved_shape = ix.tile_shape, saved_depth = ix.depth;
  for (int shape = 0; shape < kTileShapes && e == cudaSuccess; ++shape) {
    for (int depth = 1; depth <= kMaxScanDepth && e == cudaSuccess; ++depth) {
      ix.tile_shape = shape;
      ix.depth = depth;
      const FrameItem it = make_item(d_frame, d_prev_annf, out, nullptr, nullptr, H, W, shape);
      e = run_frame(ix, ix.ws, &q, cs, it, nullptr);   // warm-up
      if (e == cudaSuccess) e = cudaEventRecord(e0, cs);
      for (int k = 0; k < iters && e == cudaSuccess; ++k) e = run_frame(ix, ix.ws, &q, cs, it, nullptr);
      if (e == cudaSuccess) e = cudaEventRecord(e1, cs);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      riann_tuning_t t;
      t.tile_shape = shape;
      t.depth = depth;
      t.ms = ms / (float)iters;
      all.push_back(t);
    }
  }
  ix.profile = saved_prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess || all.empty()) {
    ix.tile_shape = saved_shape;
    ix.depth = saved_depth;
    return from_cuda(e);
  }
  const riann_tuning_t best = *std::min_element(all.begin(), all.end(), [](const riann_tuning_t& a,
                                                                             const riann_tuning_t& b) {
    return a.ms < b.ms;
  });
  ix.tile_shape = best.tile_shape;
  ix.depth = best.depth;
  if (results)
    for (int i = 0; i < (int)all.size() && i < max_results; ++i) results[i] = all[i];
  if (n_results) *n_results = (int32_t)all.size();
  return RIANN_OK;
}

}  // extern "C"
