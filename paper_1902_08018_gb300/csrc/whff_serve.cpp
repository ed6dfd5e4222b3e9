// whff_serve.cpp -- control-loop request server: resident models, admission by
// device-memory footprint, continuous batching and CUDA-graph replay.
//
// The paper's controller runs one deformation GEMV per light millisecond and
// tolerates a missed deadline at a cost in yield (Sec. 1: corrections are due
// within 50 ms; a firm real-time system).  Here several resident models
// receive step requests; requests that arrive while a model's previous pass
// is on the GPU wait in its queue and are folded into the next pass as extra
// right-hand sides (continuous batching).  Columns are applied in arrival
// order, so the carried state s <- decay*s + y evolves exactly as if every
// request had been served alone, and each column's y is computed by the same
// kernel arithmetic whatever the batch as long as the pass stays on the CUDA
// cores (the kernels treat right-hand sides independently; a pass wide enough
// for the tensor cores rounds differently, within the same bar).  Different
// models' passes run concurrently on a pool of streams; passes longer than
// kSliceBytes of stream are captured as row slits, so that the persistent
// grid of a big model releases the SMs between slits to the kernels of
// smaller, higher-priority models.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <string>
#include <vector>

#include "whff.h"
#include "whff_blob.h"

namespace whff {
void set_error(const std::string& msg);
}
using whff::set_error;

namespace {

enum ModelState { kRemoved = 0, kAdmitted = 1, kWaiting = 2 };

struct Model {
  int state = kRemoved;
  whff_handle* h = nullptr;
  int64_t M = 0, N = 0;
  double decay = 0.0;
  double* d_state = nullptr;
  float* x_pin = nullptr;    // max_batch x N, pinned
  double* y_pin = nullptr;   // max_batch x M, pinned
  std::vector<whff_graph*> graphs;  // bucket b -> graph for R = 1 << b
  size_t footprint = 0;
  int64_t slice_rows = 0;  // rows per slit of a captured pass (0: whole matrix)
};

constexpr size_t kSliceBytes = size_t(512) << 20;  // about 80 us of HBM streaming per slit

int bucket_of(int n) {  // largest b with 2^b <= n
  int b = 0;
  while ((2 << b) <= n) ++b;
  return b;
}

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct whff_server {
  size_t budget = 0, used = 0;
  int max_batch = 8;
  int nbuckets = 4;
  std::vector<cudaStream_t> streams;        // capture pool
  std::vector<cudaStream_t> model_streams;  // one per model, priority by footprint
  std::vector<Model> models;
};

namespace {

// One stream per model; smaller footprints (shorter passes) get higher priority,
// so that a cheap model's pass is not stuck behind a long one.
int make_model_streams(whff_server* s) {
  for (auto st : s->model_streams) cudaStreamDestroy(st);
  s->model_streams.clear();
  int lo = 0, hi = 0;  // CUDA: numerically lower = higher priority
  if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess) return WHFF_ECUDA;
  const int nm = (int)s->models.size();
  std::vector<int> order(nm);
  for (int i = 0; i < nm; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return s->models[a].footprint < s->models[b].footprint; });
  std::vector<int> prio(nm, lo);
  const int levels = lo - hi + 1;
  for (int rank = 0; rank < nm; ++rank)
    prio[order[rank]] = hi + (nm > 1 ? (rank * (levels - 1)) / (nm - 1) : 0);
  for (int i = 0; i < nm; ++i) {
    cudaStream_t st;
    if (cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, prio[i]) != cudaSuccess) return WHFF_ECUDA;
    s->model_streams.push_back(st);
  }
  return WHFF_OK;
}

}  // namespace

namespace {
void release_model(Model& m) {
  for (auto* g : m.graphs) whff_graph_destroy(g);
  m.graphs.clear();
  cudaFree(m.d_state);
  cudaFreeHost(m.x_pin);
  cudaFreeHost(m.y_pin);
  m.d_state = nullptr;
  m.x_pin = nullptr;
  m.y_pin = nullptr;
  cudaGetLastError();
}

// Footprint of a model on the device: resident matrix and workspaces, state,
// one staging pair per batch bucket.
int model_footprint(const whff_server* s, whff_handle* h, Model& m) {
  int fmt, rate;
  size_t dev_bytes = 0;
  if (whff_info(h, &fmt, &rate, &m.M, &m.N, &dev_bytes)) return WHFF_EINVAL;
  size_t staging = 0;
  for (int b = 0; b < s->nbuckets; ++b) staging += (size_t)(1 << b) * (size_t)(m.N * 4 + m.M * 8);
  m.footprint = dev_bytes + (size_t)m.M * 8 + staging;
  return WHFF_OK;
}

int admit(whff_server* s, Model& m);

// Admit waiting models in registration order while the oldest one fits the
// budget (first come, first served: a small model does not overtake a big one).
int admit_waiting(whff_server* s) {
  for (auto& m : s->models) {
    if (m.state != kWaiting) continue;
    if (s->used + m.footprint > s->budget) break;
    const int e = admit(s, m);
    if (e) return e;
  }
  return WHFF_OK;
}
}  // namespace

extern "C" void whff_server_destroy(whff_server* s) {
  if (!s) return;
  for (auto& st : s->streams) cudaStreamSynchronize(st);
  for (auto& st : s->model_streams) cudaStreamSynchronize(st);
  for (auto& m : s->models) release_model(m);
  for (auto& st : s->streams) cudaStreamDestroy(st);
  for (auto& st : s->model_streams) cudaStreamDestroy(st);
  cudaGetLastError();
  delete s;
}

extern "C" int whff_server_create(size_t hbm_budget, int max_batch, int nstreams, whff_server** out) {
  if (!out || max_batch < 1 || max_batch > 8 || (max_batch & (max_batch - 1)) || nstreams < 1 || nstreams > 64) {
    set_error("whff_server_create: max_batch must be 1, 2, 4 or 8 and nstreams in 1..64");
    return WHFF_EINVAL;
  }
  *out = nullptr;
  auto* s = new whff_server;
  s->budget = hbm_budget;
  s->max_batch = max_batch;
  s->nbuckets = bucket_of(max_batch) + 1;
  for (int i = 0; i < nstreams; ++i) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      whff_server_destroy(s);
      set_error("whff_server_create: cudaStreamCreate failed");
      return WHFF_ECUDA;
    }
    s->streams.push_back(st);
  }
  *out = s;
  return WHFF_OK;
}

extern "C" int whff_server_add_model_ex(whff_server* s, whff_handle* h, double decay, unsigned flags,
                                        int* model_id) {
  if (!s || !h || !model_id || (flags & ~(unsigned)WHFF_SERVER_WAIT)) {
    set_error("whff_server_add_model: null argument or unknown flag");
    return WHFF_EINVAL;
  }
  Model m;
  if (model_footprint(s, h, m)) {
    set_error("whff_server_add_model: bad handle");
    return WHFF_EINVAL;
  }
  m.h = h;
  m.decay = decay;
  bool waiting_ahead = false;  // registrations are admitted in order
  for (const auto& o : s->models) waiting_ahead |= o.state == kWaiting;
  if (s->used + m.footprint > s->budget || waiting_ahead) {
    if (!(flags & WHFF_SERVER_WAIT)) {
      set_error("whff_server_add_model: device-memory budget exceeded (" + std::to_string(s->used + m.footprint) +
                " > " + std::to_string(s->budget) + " bytes)");
      return WHFF_EBUSY;
    }
    m.state = kWaiting;  // admitted by whff_server_remove_model once memory frees up
    *model_id = (int)s->models.size();
    s->models.push_back(m);
    return WHFF_OK;
  }
  const int e = admit(s, m);
  if (e) return e;
  *model_id = (int)s->models.size();
  s->models.push_back(m);
  return WHFF_OK;
}

extern "C" int whff_server_add_model(whff_server* s, whff_handle* h, double decay, int* model_id) {
  return whff_server_add_model_ex(s, h, decay, 0u, model_id);
}

extern "C" int whff_server_model_state(const whff_server* s, int model_id, int* state) {
  if (!s || !state || model_id < 0 || model_id >= (int)s->models.size()) {
    set_error("whff_server_model_state: bad argument");
    return WHFF_EINVAL;
  }
  *state = s->models[model_id].state;
  return WHFF_OK;
}

extern "C" int whff_server_remove_model(whff_server* s, int model_id) {
  if (!s || model_id < 0 || model_id >= (int)s->models.size() || s->models[model_id].state == kRemoved) {
    set_error("whff_server_remove_model: bad or removed model");
    return WHFF_EINVAL;
  }
  Model& m = s->models[model_id];
  if (m.state == kAdmitted) {
    if (model_id < (int)s->model_streams.size()) cudaStreamSynchronize(s->model_streams[model_id]);
    release_model(m);
    s->used -= m.footprint;
  }
  m.state = kRemoved;
  m.h = nullptr;
  return admit_waiting(s);
}

namespace {
// Allocate a model's state and staging and capture its graphs; on success it
// counts against the budget.
int admit(whff_server* s, Model& m) {
  whff_handle* h = m.h;
  const double decay = m.decay;
  int fmt, rate;
  if (whff_info(h, &fmt, &rate, nullptr, nullptr, nullptr)) return WHFF_EINVAL;
  auto fail = [&](int code, const char* what) {
    release_model(m);
    set_error(std::string("whff_server_add_model: ") + what);
    return code;
  };
  if (cudaMalloc(&m.d_state, (size_t)m.M * 8) != cudaSuccess || cudaMemset(m.d_state, 0, (size_t)m.M * 8) != cudaSuccess)
    return fail(WHFF_ENOMEM, "state allocation failed");
  if (cudaMallocHost(&m.x_pin, (size_t)s->max_batch * m.N * 4) != cudaSuccess ||
      cudaMallocHost(&m.y_pin, (size_t)s->max_batch * m.M * 8) != cudaSuccess)
    return fail(WHFF_ENOMEM, "pinned staging allocation failed");
  // long passes are captured as row slits of at most kSliceBytes each (time
  // slicing); the handle's own setting is restored afterwards
  int64_t own_slice = 0;
  whff_get_slice_rows(h, &own_slice);
  const int64_t align = whff::row_align(fmt);
  size_t fixed = whff_compressed_size(fmt, rate, m.M, m.N), held = 0;
  if (!fixed) whff_info(h, nullptr, nullptr, nullptr, nullptr, &held);  // fixed accuracy: bounded by all it holds
  const double row_bytes = (double)(fixed ? fixed : held) / (double)m.M;
  int64_t slice = 0;
  if (row_bytes * (double)m.M > (double)kSliceBytes)
    slice = std::max<int64_t>(align, (int64_t)((double)kSliceBytes / row_bytes) / align * align);
  if (whff_set_slice_rows(h, slice)) return fail(WHFF_EINVAL, "slice setting failed");
  for (int b = 0; b < s->nbuckets; ++b) {
    whff_graph* g = nullptr;
    int e = whff_graph_create_host(h, m.x_pin, 1 << b, m.N, m.y_pin, m.M, m.d_state, decay, s->streams[0], &g);
    if (e) {
      whff_set_slice_rows(h, own_slice);
      return fail(e, "graph capture failed");
    }
    m.graphs.push_back(g);
  }
  whff_set_slice_rows(h, own_slice);
  m.slice_rows = slice;
  s->used += m.footprint;
  m.state = kAdmitted;
  return WHFF_OK;
}
}  // namespace

extern "C" int whff_server_reset_state(whff_server* s, int model_id) {
  if (!s || model_id < 0 || model_id >= (int)s->models.size() || s->models[model_id].state != kAdmitted) {
    set_error("whff_server_reset_state: bad model");
    return WHFF_EINVAL;
  }
  Model& m = s->models[model_id];
  if (cudaMemset(m.d_state, 0, (size_t)m.M * 8) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
    set_error("whff_server_reset_state: CUDA error");
    return WHFF_ECUDA;
  }
  return WHFF_OK;
}

extern "C" int whff_server_read_state(whff_server* s, int model_id, double* host_out) {
  if (!s || !host_out || model_id < 0 || model_id >= (int)s->models.size() ||
      s->models[model_id].state != kAdmitted) {
    set_error("whff_server_read_state: bad argument or model not admitted");
    return WHFF_EINVAL;
  }
  Model& m = s->models[model_id];
  if (cudaMemcpy(host_out, m.d_state, (size_t)m.M * 8, cudaMemcpyDeviceToHost) != cudaSuccess) {
    set_error("whff_server_read_state: CUDA error");
    return WHFF_ECUDA;
  }
  return WHFF_OK;
}

// Replay a request trace in real time.  Request i is for model[i], arrives at
// arrival_s[i] seconds after the start (non-decreasing) and carries the N
// floats at x[i].  Dispatch is earliest-deadline-first over the idle models
// with queued requests; each model's pass runs on its own stream.  With
// drop_after_s > 0 the server is firm real-time: a request still queued
// drop_after_s after its arrival is discarded (status 2) instead of served
// late.  On return latency_s[i] = completion - arrival as seen by the host
// (for a dropped request: the age at which it was discarded), batch[i] =
// requests in its pass (0 if dropped), status[i] (if not NULL) = 0 served in
// time, 1 served late, 2 dropped, and y[i] (if y and y[i] are not NULL) its M
// doubles.  max_wait_s bounds the whole run (WHFF_ETIMEOUT if it expires).
extern "C" int whff_server_run(whff_server* s, int n, const int* model, const double* arrival_s,
                               const float* const* x, double* const* y, double* latency_s, int* batch,
                               int* status, double drop_after_s, double max_wait_s) {
  if (!s || n < 0 || (n && (!model || !arrival_s || !x || !latency_s || !batch))) {
    set_error("whff_server_run: bad argument");
    return WHFF_EINVAL;
  }
  const int nm = (int)s->models.size();
  for (int i = 0; i < n; ++i)
    if (model[i] < 0 || model[i] >= nm || !x[i] || (i && arrival_s[i] < arrival_s[i - 1])) {
      set_error("whff_server_run: bad request " + std::to_string(i));
      return WHFF_EINVAL;
    }
  std::vector<char> live(nm);
  for (int m = 0; m < nm; ++m) live[m] = s->models[m].state == kAdmitted;
  if ((int)s->model_streams.size() != nm && make_model_streams(s) != WHFF_OK) {
    set_error("whff_server_run: cannot create model streams");
    return WHFF_ECUDA;
  }
  struct Pass {
    std::vector<int> reqs;
    cudaEvent_t ev = nullptr;
    bool busy = false;
  };
  std::vector<std::deque<int>> queue(nm);
  std::vector<Pass> inflight(nm);
  for (auto& p : inflight)
    if (cudaEventCreateWithFlags(&p.ev, cudaEventDisableTiming) != cudaSuccess) {
      set_error("whff_server_run: cudaEventCreate failed");
      return WHFF_ECUDA;
    }
  const bool firm = drop_after_s > 0.0;
  int next_arrival = 0, done = 0;
  int err = WHFF_OK;
  const double t0 = now_s();
  while (done < n) {
    const double t = now_s() - t0;
    if (t > max_wait_s) {
      err = WHFF_ETIMEOUT;
      set_error("whff_server_run: watchdog expired with requests open");
      break;
    }
    while (next_arrival < n && arrival_s[next_arrival] <= t) {
      const int r = next_arrival++;
      if (live[model[r]]) {
        queue[model[r]].push_back(r);
      } else {  // the model is waiting for memory or was removed: refused
        latency_s[r] = 0.0;
        batch[r] = 0;
        if (status) status[r] = 3;
        ++done;
      }
    }
    for (int m = 0; m < nm; ++m) {  // completions
      Pass& p = inflight[m];
      if (!p.busy) continue;
      cudaError_t q = cudaEventQuery(p.ev);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) {
        err = WHFF_ECUDA;
        set_error(std::string("whff_server_run: pass failed: ") + cudaGetErrorString(q));
        break;
      }
      const double tc = now_s() - t0;
      const Model& md = s->models[m];
      for (size_t k = 0; k < p.reqs.size(); ++k) {
        const int r = p.reqs[k];
        latency_s[r] = tc - arrival_s[r];
        batch[r] = (int)p.reqs.size();
        if (status) status[r] = (firm && latency_s[r] > drop_after_s) ? 1 : 0;
        if (y && y[r]) std::memcpy(y[r], md.y_pin + k * md.M, (size_t)md.M * 8);
      }
      done += (int)p.reqs.size();
      p.reqs.clear();
      p.busy = false;
    }
    if (err) break;
    if (firm) {  // discard requests whose deadline has already passed
      const double tn = now_s() - t0;
      for (int m = 0; m < nm; ++m)
        while (!queue[m].empty() && tn - arrival_s[queue[m].front()] > drop_after_s) {
          const int r = queue[m].front();
          queue[m].pop_front();
          latency_s[r] = tn - arrival_s[r];
          batch[r] = 0;
          if (status) status[r] = 2;
          ++done;
        }
    }
    for (;;) {  // dispatch: earliest deadline (oldest queued request) first
      int best = -1;
      for (int m = 0; m < nm; ++m)
        if (!inflight[m].busy && !queue[m].empty() &&
            (best < 0 || arrival_s[queue[m].front()] < arrival_s[queue[best].front()]))
          best = m;
      if (best < 0) break;
      const int m = best;
      Pass& p = inflight[m];
      const int take = 1 << bucket_of(std::min<int>((int)queue[m].size(), s->max_batch));
      Model& md = s->models[m];
      for (int c = 0; c < take; ++c) {
        const int r = queue[m].front();
        queue[m].pop_front();
        std::memcpy(md.x_pin + (size_t)c * md.N, x[r], (size_t)md.N * 4);
        p.reqs.push_back(r);
      }
      cudaStream_t st = s->model_streams[m];
      int e = whff_graph_launch(md.graphs[bucket_of(take)], st);
      if (e == WHFF_OK && cudaEventRecord(p.ev, st) != cudaSuccess) e = WHFF_ECUDA;
      if (e) {
        err = e;
        break;
      }
      p.busy = true;
    }
    if (err) break;
  }
  if (err) cudaDeviceSynchronize();
  for (auto& p : inflight) cudaEventDestroy(p.ev);
  cudaGetLastError();
  return err;
}
