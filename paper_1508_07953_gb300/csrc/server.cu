// server.cu -- the served form: continuous batching of many video streams.
//
// Host-side scheduler around the batched step.  Streams are admitted while
// their resident state (two ANN fields, distances, counts and a frame buffer,
// riann_session_state_bytes) fits a device-memory budget, their queries fit
// the per-tick capacity of the batch contexts and (rate admission) the GPU
// time they claim at their declared frame rate, priced at the measured GPU
// time per query of their index, fits a load limit.  Frames are submitted into a
// stream's pinned input slots (two per stream, so a frame can arrive while the
// previous one is being copied); a newer frame replaces an undispatched older
// one (counted as dropped).  riann_server_step completes the tick in flight
// and launches the next one over every stream with a pending frame: frames
// that arrived while the GPU was busy join the next tick, streams join and
// leave between ticks.  Latency of a frame = completion of its tick (seen by
// the host) - its arrival time, both on riann_server_clock().
#include <chrono>
#include <cstring>
#include <deque>
#include <new>
#include <vector>

#include "common.cuh"
#include "trace.h"

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct ServerStream {
  bool open = false;
  int32_t H = 0, W = 0, C = 0;
  int64_t Q = 0;
  riann_session_t sess = nullptr;
  uint8_t* h_in[2] = {nullptr, nullptr};   // pinned input slots
  int32_t* h_out = nullptr;                // pinned: latest completed field
  int pending_slot = -1;                   // slot holding an undispatched frame
  double pending_t = 0;
  int64_t pending_id = -1;
  int busy_slot = -1;                      // slot read by the tick in flight
  double busy_t = 0;
  int64_t busy_id = -1;
  int64_t submitted = 0, dropped = 0, completed = 0;
  size_t state_bytes = 0;
  double fps = 0;                          // declared frame rate (rate admission)
};

}  // namespace

struct riann_server_s {
  riann_index_t idx[2] = {nullptr, nullptr};     // [0] gray, [1] RGB
  riann_batch_t batch[2] = {nullptr, nullptr};
  size_t budget = 0, used = 0;
  int64_t cap_q[2] = {0, 0};                     // per-tick query capacity per index
  int64_t open_q[2] = {0, 0};
  riann_params params{};
  std::vector<ServerStream> streams;
  cudaEvent_t done = nullptr;
  bool inflight = false;
  std::vector<int> members;                      // streams of the tick in flight
  std::deque<riann_server_result_t> results;
  int64_t ticks = 0, frames_done = 0, queries_done = 0, rejected = 0;
  int64_t submitted = 0, dropped = 0;            // over all streams, open or closed
  bool plain = false;                            // per-frame path instead of the batched step
  // rate admission: GPU time per query per index, measured with events
  // around each index's part of a tick and averaged (weight 0.2 per tick)
  double load_limit = 0;
  double ns_q[2] = {0, 0};
  cudaEvent_t ev[2][2] = {};
  int64_t tick_q[2] = {0, 0};                    // queries per index in the tick in flight
  std::mutex mu;
};

namespace {

int chan_slot(int C) { return C == 3 ? 1 : 0; }

void close_stream(riann_server_s* s, ServerStream& st) {
  if (!st.open) return;
  riann_session_destroy(st.sess);
  cudaFreeHost(st.h_in[0]);
  cudaFreeHost(st.h_in[1]);
  cudaFreeHost(st.h_out);
  s->used -= st.state_bytes;
  s->open_q[chan_slot(st.C)] -= st.Q;
  st = ServerStream();
}

// Complete the tick in flight (blocking when `wait`); false if still running.
bool finish_tick(riann_server_s* s, bool wait) {
  if (!s->inflight) return true;
  if (wait) {
    if (cudaEventSynchronize(s->done) != cudaSuccess) return false;
  } else if (cudaEventQuery(s->done) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const double t = now_s();
  for (int id : s->members) {
    ServerStream& st = s->streams[id];
    if (!st.open || st.busy_slot < 0) continue;
    riann_server_result_t r;
    r.stream_id = id;
    r.frame_id = st.busy_id;
    r.t_arrival = st.busy_t;
    r.t_done = t;
    s->results.push_back(r);
    st.busy_slot = -1;
    ++st.completed;
    ++s->frames_done;
    s->queries_done += st.Q;
  }
  for (int k = 0; k < 2; ++k) {
    if (s->tick_q[k] <= 0) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, s->ev[k][0], s->ev[k][1]) == cudaSuccess && ms > 0.f) {
      const double ns = 1e6 * (double)ms / (double)s->tick_q[k];
      s->ns_q[k] = s->ns_q[k] > 0 ? 0.8 * s->ns_q[k] + 0.2 * ns : ns;
    }
    cudaGetLastError();
    s->tick_q[k] = 0;
  }
  s->members.clear();
  s->inflight = false;
  return true;
}

// GPU seconds per second claimed by the open streams at the current estimates.
double claimed_load(const riann_server_s* s) {
  double l = 0;
  for (const auto& st : s->streams)
    if (st.open && st.fps > 0) l += st.fps * (double)st.Q * s->ns_q[chan_slot(st.C)] * 1e-9;
  return l;
}

}  // namespace

extern "C" {

double riann_server_clock(void) { return now_s(); }

int riann_server_create(riann_index_t gray, riann_index_t rgb, size_t budget_bytes, int64_t max_tick_queries,
                        int32_t max_streams, const riann_params* p, int32_t flags, double load_limit,
                        riann_server_t* out) {
  if (!out) return RIANN_ERR_INVALID_ARG;
  *out = nullptr;
  if ((!gray && !rgb) || !p || max_streams < 1 || max_streams > 4096 || max_tick_queries < 1)
    return RIANN_ERR_INVALID_ARG;
  riann_index_info_t gi, ci;
  if (gray && (riann_index_info(gray, &gi) || gi.channels != 1)) return RIANN_ERR_INVALID_ARG;
  if (rgb && (riann_index_info(rgb, &ci) || ci.channels != 3)) return RIANN_ERR_INVALID_ARG;
  if ((gray && gi.unit) || (rgb && ci.unit)) return RIANN_ERR_UNSUPPORTED;
  riann_server_s* s = new (std::nothrow) riann_server_s();
  if (!s) return RIANN_ERR_OOM;
  s->idx[0] = gray;
  s->idx[1] = rgb;
  s->budget = budget_bytes;
  s->params = *p;
  s->plain = (flags & RIANN_SERVER_PLAIN) != 0;
  s->load_limit = load_limit;
  s->streams.resize((size_t)max_streams);
  int rc = RIANN_OK;
  for (int k = 0; k < 2 && rc == RIANN_OK; ++k) {
    if (!s->idx[k]) continue;
    s->cap_q[k] = max_tick_queries;
    rc = riann_batch_create(s->idx[k], max_streams, max_tick_queries, 0, &s->batch[k]);
  }
  if (rc == RIANN_OK && cudaEventCreateWithFlags(&s->done, cudaEventDisableTiming) != cudaSuccess)
    rc = RIANN_ERR_CUDA;
  for (int k = 0; k < 2 && rc == RIANN_OK; ++k)
    for (int j = 0; j < 2 && rc == RIANN_OK; ++j)
      if (cudaEventCreate(&s->ev[k][j]) != cudaSuccess) rc = RIANN_ERR_CUDA;
  if (rc != RIANN_OK) {
    for (int k = 0; k < 2; ++k) riann_batch_destroy(s->batch[k]);
    if (s->done) cudaEventDestroy(s->done);
    for (int k = 0; k < 2; ++k)
      for (int j = 0; j < 2; ++j)
        if (s->ev[k][j]) cudaEventDestroy(s->ev[k][j]);
    delete s;
    return rc;
  }
  *out = s;
  return RIANN_OK;
}

void riann_server_destroy(riann_server_t s) {
  if (!s) return;
  cudaDeviceSynchronize();
  for (auto& st : s->streams) close_stream(s, st);
  for (int k = 0; k < 2; ++k) riann_batch_destroy(s->batch[k]);
  if (s->done) cudaEventDestroy(s->done);
  for (int k = 0; k < 2; ++k)
    for (int j = 0; j < 2; ++j)
      if (s->ev[k][j]) cudaEventDestroy(s->ev[k][j]);
  delete s;
}

int riann_server_open(riann_server_t s, int32_t H, int32_t W, int32_t C, double fps, int32_t* stream_id) {
  if (!s || !stream_id || (C != 1 && C != 3)) return RIANN_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  *stream_id = -1;
  const int k = chan_slot(C);
  if (!s->idx[k] || H < 8 || W < 8) return RIANN_ERR_INVALID_ARG;
  const int64_t Q = (int64_t)(H - 7) * (W - 7);
  const int64_t bytes = riann_session_state_bytes(s->idx[k], H, W);
  int slot = -1;
  for (size_t i = 0; i < s->streams.size(); ++i)
    if (!s->streams[i].open) {
      slot = (int)i;
      break;
    }
  bool fits = slot >= 0 && s->used + (size_t)bytes <= s->budget && s->open_q[k] + Q <= s->cap_q[k];
  if (fits && s->load_limit > 0 && fps > 0) {
    if (s->ns_q[k] > 0) {
      fits = claimed_load(s) + fps * (double)Q * s->ns_q[k] * 1e-9 <= s->load_limit;
    } else {   // no measurement yet: one rate-declaring stream per index until there is
      for (const auto& o : s->streams)
        if (o.open && o.fps > 0 && chan_slot(o.C) == k) fits = false;
    }
  }
  if (!fits) {
    ++s->rejected;
    return RIANN_ERR_ADMISSION;
  }
  ServerStream st;
  st.H = H;
  st.W = W;
  st.C = C;
  st.Q = Q;
  int rc = riann_session_create(s->idx[k], H, W, &st.sess);
  const size_t fb = (size_t)H * W * C;
  if (rc == RIANN_OK && (cudaMallocHost((void**)&st.h_in[0], fb) != cudaSuccess ||
                         cudaMallocHost((void**)&st.h_in[1], fb) != cudaSuccess ||
                         cudaMallocHost((void**)&st.h_out, sizeof(int32_t) * (size_t)Q) != cudaSuccess))
    rc = RIANN_ERR_OOM;
  if (rc != RIANN_OK) {
    cudaGetLastError();
    riann_session_destroy(st.sess);
    cudaFreeHost(st.h_in[0]);
    cudaFreeHost(st.h_in[1]);
    cudaFreeHost(st.h_out);
    return rc;
  }
  st.open = true;
  st.fps = fps;
  st.state_bytes = (size_t)bytes;
  s->used += st.state_bytes;
  s->open_q[k] += Q;
  s->streams[slot] = st;
  *stream_id = slot;
  return RIANN_OK;
}

int riann_server_close(riann_server_t s, int32_t id) {
  if (!s || id < 0 || id >= (int)s->streams.size()) return RIANN_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  ServerStream& st = s->streams[id];
  if (!st.open) return RIANN_ERR_INVALID_ARG;
  if (st.busy_slot >= 0 && !finish_tick(s, true)) return RIANN_ERR_CUDA;
  close_stream(s, st);
  return RIANN_OK;
}

int riann_server_submit(riann_server_t s, int32_t id, const uint8_t* h_frame, int64_t frame_id, double t_arrival) {
  if (!s || !h_frame || id < 0 || id >= (int)s->streams.size()) return RIANN_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  ServerStream& st = s->streams[id];
  if (!st.open) return RIANN_ERR_INVALID_ARG;
  // write into the slot the tick in flight does not read
  const int slot = st.busy_slot == 0 ? 1 : 0;
  if (st.pending_slot >= 0) {   // an undispatched older frame is replaced
    ++st.dropped;
    ++s->dropped;
  }
  std::memcpy(st.h_in[slot], h_frame, (size_t)st.H * st.W * st.C);
  st.pending_slot = slot;
  st.pending_t = t_arrival;
  st.pending_id = frame_id;
  ++st.submitted;
  ++s->submitted;
  return RIANN_OK;
}

int riann_server_step(riann_server_t s, riann_stream_t stream, int32_t wait, int32_t* launched) {
  if (!s) return RIANN_ERR_INVALID_ARG;
  riann::NvtxRange range("riann served tick");
  std::lock_guard<std::mutex> lock(s->mu);
  if (launched) *launched = 0;
  if (!finish_tick(s, wait != 0)) return RIANN_OK;   // still running: nothing started
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  std::vector<riann_session_t> sess[2];
  std::vector<const uint8_t*> frames[2];
  for (size_t i = 0; i < s->streams.size(); ++i) {
    ServerStream& st = s->streams[i];
    if (!st.open || st.pending_slot < 0) continue;
    uint8_t* dframe = riann_session_frame_buffer(st.sess);
    cudaError_t e = cudaMemcpyAsync(dframe, st.h_in[st.pending_slot], (size_t)st.H * st.W * st.C,
                                    cudaMemcpyHostToDevice, cs);
    if (e != cudaSuccess) return RIANN_ERR_CUDA;
    st.busy_slot = st.pending_slot;
    st.busy_t = st.pending_t;
    st.busy_id = st.pending_id;
    st.pending_slot = -1;
    const int k = chan_slot(st.C);
    sess[k].push_back(st.sess);
    frames[k].push_back(dframe);
    s->members.push_back((int)i);
  }
  if (s->members.empty()) return RIANN_OK;
  for (int k = 0; k < 2; ++k) {
    if (sess[k].empty()) continue;
    int64_t q = 0;
    for (int id : s->members)
      if (chan_slot(s->streams[id].C) == k) q += s->streams[id].Q;
    s->tick_q[k] = q;
    if (cudaEventRecord(s->ev[k][0], cs) != cudaSuccess) return RIANN_ERR_CUDA;
    if (s->plain) {
      for (size_t i = 0; i < sess[k].size(); ++i) {
        const int rc = riann_session_frame(sess[k][i], &s->params, stream, frames[k][i], nullptr, nullptr, nullptr);
        if (rc) return rc;
      }
    } else {
      const int rc = riann_batch_run(s->batch[k], &s->params, stream, sess[k].data(), frames[k].data(),
                                     (int32_t)sess[k].size());
      if (rc) return rc;
    }
    if (cudaEventRecord(s->ev[k][1], cs) != cudaSuccess) return RIANN_ERR_CUDA;
  }
  for (int id : s->members) {
    ServerStream& st = s->streams[id];
    int32_t* d_annf = nullptr;
    riann_session_outputs(st.sess, &d_annf, nullptr, nullptr);
    if (cudaMemcpyAsync(st.h_out, d_annf, sizeof(int32_t) * (size_t)st.Q, cudaMemcpyDeviceToHost, cs) != cudaSuccess)
      return RIANN_ERR_CUDA;
  }
  if (cudaEventRecord(s->done, cs) != cudaSuccess) return RIANN_ERR_CUDA;
  s->inflight = true;
  ++s->ticks;
  if (launched) *launched = (int32_t)s->members.size();
  return RIANN_OK;
}

int riann_server_poll(riann_server_t s, riann_server_result_t* out, int32_t max, int32_t* n) {
  if (!s || !n || (max > 0 && !out)) return RIANN_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  int k = 0;
  while (k < max && !s->results.empty()) {
    out[k++] = s->results.front();
    s->results.pop_front();
  }
  *n = k;
  return RIANN_OK;
}

int riann_server_field(riann_server_t s, int32_t id, int32_t* out) {
  if (!s || !out || id < 0 || id >= (int)s->streams.size()) return RIANN_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  ServerStream& st = s->streams[id];
  if (!st.open || st.completed == 0 || st.busy_slot >= 0) return RIANN_ERR_INVALID_ARG;
  std::memcpy(out, st.h_out, sizeof(int32_t) * (size_t)st.Q);
  return RIANN_OK;
}

int riann_server_info(riann_server_t s, riann_server_info_t* out) {
  if (!s || !out) return RIANN_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  std::memset(out, 0, sizeof(*out));
  for (const auto& st : s->streams)
    if (st.open) ++out->open_streams;
  out->submitted = s->submitted;
  out->dropped = s->dropped;
  out->budget_bytes = s->budget;
  out->used_bytes = s->used;
  out->ticks = s->ticks;
  out->frames_done = s->frames_done;
  out->queries_done = s->queries_done;
  out->rejected = s->rejected;
  out->load = claimed_load(s);
  out->ns_per_query[0] = s->ns_q[0];
  out->ns_per_query[1] = s->ns_q[1];
  return RIANN_OK;
}

int riann_server_stream_counts(riann_server_t s, int32_t id, int64_t* submitted, int64_t* dropped,
                               int64_t* completed) {
  if (!s || id < 0 || id >= (int)s->streams.size()) return RIANN_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(s->mu);
  const ServerStream& st = s->streams[id];
  if (submitted) *submitted = st.submitted;
  if (dropped) *dropped = st.dropped;
  if (completed) *completed = st.completed;
  return RIANN_OK;
}

}  // extern "C"
