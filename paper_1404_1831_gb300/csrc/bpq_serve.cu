// Continuous batching of a query stream over one resident index (the request
// loop of a search service; the paper describes the per-query path of §2.3.3,
// §3.1 and §3.2, which every batch runs unchanged).
//
// A server owns a fixed pool of slots.  A slot is one batch in flight: its own
// non-blocking CUDA stream, a device workspace (query tables, visited cells, HBPQ
// tables), device and page-locked host buffers for the queries and results, and a
// completion event.  The host loop
//   1. retires every slot whose event has completed (results are in host memory),
//   2. fills every free slot with a batch of waiting requests and enqueues it:
//      H2D copy of the queries, the search pipeline, D2H copy of the results,
//      event record -- all asynchronous on the slot's stream,
// so a batch is launched while earlier batches are still running and their
// kernels overlap on the GPU.  Admission is by device memory: a batch takes
// waiting requests (oldest first) only while the workspace that bpq_search needs
// for them at their largest budget L fits the slot's share of the device budget.
// With grouping on, a batch takes requests of one budget class (L within a
// factor of two), so short queries are not held back by the long queries of the
// same batch.  Each query is searched exactly as bpq_search searches it alone.
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <memory>
#include <thread>
#include <vector>

#include "bpq_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  int64_t id;         // request number (submission order)
  int32_t L;
  double arrival;     // seconds on the server's clock
  const float* q;     // D floats (the caller's array, or `own`)
  std::vector<float> own;
};

struct Slot {
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
  bpq::DevBuf ws, q, ids, dists;
  size_t ws_bytes = 0;
  float* q_pin = nullptr;
  int32_t* L_pin = nullptr;
  int32_t* ids_pin = nullptr;
  float* dists_pin = nullptr;
  std::vector<int64_t> L64;
  std::vector<Req> reqs;
  bool busy = false;
};

struct Done {
  int64_t id;
  double arrival, finish;
  std::vector<int32_t> ids;
  std::vector<float> dists;
};

int budget_class(int64_t L) {
  int c = 0;
  while ((int64_t(2) << c) <= L && c < 40) ++c;
  return c;  // floor(log2(L))
}

}  // namespace

struct bpq_server {
  const bpq_index* ix = nullptr;
  bpq_server_config cfg{};
  int D = 0;
  std::vector<std::unique_ptr<Slot>> slots;
  std::deque<Req> pending[41];  // by budget class (one queue when grouping is off)
  int64_t next_id = 0;
  Clock::time_point t0;
  // completed requests not yet taken (incremental interface)
  std::deque<Done> done;
  // trace mode: results go straight to the caller's arrays
  int32_t* trace_ids = nullptr;
  float* trace_dists = nullptr;
  double* trace_latency = nullptr;
  // statistics
  int64_t batches = 0, queries = 0, max_in_flight = 0;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

void release(bpq_server* s) {
  for (auto& p : s->slots) {
    Slot& sl = *p;
    if (sl.st) cudaStreamSynchronize(sl.st);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.st) cudaStreamDestroy(sl.st);
    if (sl.q_pin) cudaFreeHost(sl.q_pin);
    if (sl.L_pin) cudaFreeHost(sl.L_pin);
    if (sl.ids_pin) cudaFreeHost(sl.ids_pin);
    if (sl.dists_pin) cudaFreeHost(sl.dists_pin);
  }
  s->slots.clear();  // the device buffers are released by their destructors
}

bool any_pending(const bpq_server* s) {
  for (const auto& q : s->pending)
    if (!q.empty()) return true;
  return false;
}

// Retires the finished slots; returns the number retired.
int retire(bpq_server* s, bool block_one) {
  int n = 0;
  for (auto& p : s->slots) {
    Slot& sl = *p;
    if (!sl.busy) continue;
    cudaError_t e = cudaEventQuery(sl.done);
    if (e == cudaErrorNotReady && block_one && n == 0) e = cudaEventSynchronize(sl.done);
    if (e == cudaErrorNotReady) continue;
    BPQ_CUDA(e);
    const double t = s->now();
    const int k = s->cfg.k;
    for (size_t j = 0; j < sl.reqs.size(); ++j) {
      const Req& r = sl.reqs[j];
      if (s->trace_ids) {
        memcpy(s->trace_ids + r.id * k, sl.ids_pin + j * k, (size_t)k * 4);
        memcpy(s->trace_dists + r.id * k, sl.dists_pin + j * k, (size_t)k * 4);
        s->trace_latency[r.id] = t - r.arrival;
      } else {
        Done d{r.id, r.arrival, t, std::vector<int32_t>(sl.ids_pin + j * k, sl.ids_pin + (j + 1) * k),
               std::vector<float>(sl.dists_pin + j * k, sl.dists_pin + (j + 1) * k)};
        s->done.push_back(std::move(d));
      }
    }
    sl.reqs.clear();
    sl.busy = false;
    ++n;
    block_one = false;
  }
  return n;
}

// Fills one free slot with a batch; returns false when nothing was launched.
bool launch_one(bpq_server* s) {
  Slot* sl = nullptr;
  for (auto& c : s->slots)
    if (!c->busy) {
      sl = c.get();
      break;
    }
  if (!sl) return false;
  // the class whose oldest request is the oldest overall
  int cls = -1;
  for (int c = 0; c <= 40; ++c)
    if (!s->pending[c].empty() && (cls < 0 || s->pending[c].front().id < s->pending[cls].front().id)) cls = c;
  if (cls < 0) return false;
  std::deque<Req>& pq = s->pending[cls];
  const int k = s->cfg.k, D = s->D;
  int64_t n = 0, Lmax = 0;
  sl->reqs.clear();
  while (!pq.empty() && n < s->cfg.max_batch) {
    const int64_t Lb = std::max<int64_t>(Lmax, pq.front().L);
    // admission by device memory: the batch must fit the slot's workspace whole
    if (n > 0 && bpq_search_workspace_size(s->ix, n + 1, Lb, k, s->cfg.scorer) > sl->ws_bytes) break;
    Lmax = Lb;
    Req r = std::move(pq.front());
    pq.pop_front();
    memcpy(sl->q_pin + n * D, r.q, (size_t)D * 4);
    sl->L_pin[n] = r.L;
    sl->L64[n] = r.L;
    sl->reqs.push_back(std::move(r));
    ++n;
  }
  cudaStream_t st = sl->st;
  BPQ_CUDA(cudaMemcpyAsync(sl->q.p, sl->q_pin, (size_t)n * D * 4, cudaMemcpyHostToDevice, st));
  bpq::run_queries(*s->ix, sl->q.as<float>(), n, sl->L64.data(), 1, k, s->cfg.scorer, sl->ids.as<int32_t>(),
                   sl->dists.as<float>(), nullptr, 0, nullptr, nullptr, sl->ws.p, sl->ws_bytes, st, sl->L_pin);
  BPQ_CUDA(cudaMemcpyAsync(sl->ids_pin, sl->ids.p, (size_t)n * k * 4, cudaMemcpyDeviceToHost, st));
  BPQ_CUDA(cudaMemcpyAsync(sl->dists_pin, sl->dists.p, (size_t)n * k * 4, cudaMemcpyDeviceToHost, st));
  BPQ_CUDA(cudaEventRecord(sl->done, st));
  sl->busy = true;
  ++s->batches;
  s->queries += n;
  int64_t inflight = 0;
  for (const auto& c : s->slots) inflight += c->busy;
  s->max_in_flight = std::max(s->max_in_flight, inflight);
  return true;
}

void enqueue(bpq_server* s, Req&& r) {
  const int c = s->cfg.group_by_budget ? budget_class(r.L) : 0;
  s->pending[c].push_back(std::move(r));
}

struct Guard {
  int prev = -1;
  explicit Guard(int dev) {
    BPQ_CUDA(cudaGetDevice(&prev));
    if (prev != dev) BPQ_CUDA(cudaSetDevice(dev));
  }
  ~Guard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

template <typename F>
int guarded(F&& f) {
  try {
    bpq::set_last_error("");
    f();
    return BPQ_OK;
  } catch (const bpq::Error& e) {
    bpq::set_last_error(e.what());
    return e.code;
  } catch (const std::bad_alloc&) {
    bpq::set_last_error("host allocation failed");
    return BPQ_ENOMEM;
  } catch (const std::exception& e) {
    bpq::set_last_error(e.what());
    return BPQ_EINVAL;
  } catch (...) {
    bpq::set_last_error("unknown failure");
    return BPQ_ECUDA;
  }
}

}  // namespace

extern "C" {

int bpq_server_create(bpq_server** out, const bpq_index* ix, const bpq_server_config* cfg) {
  return guarded([&] {
    BPQ_CHECK(out && ix && cfg, BPQ_EINVAL, "NULL pointer");
    *out = nullptr;
    BPQ_CHECK(ix->n_pending == 0, BPQ_ESTATE, "points were added since the last bpq_finalize");
    BPQ_CHECK(cfg->slots >= 1 && cfg->slots <= 64, BPQ_EINVAL, "slots must be in [1, 64]");
    BPQ_CHECK(cfg->k >= 1 && cfg->k <= bpq::MAX_K, BPQ_EINVAL, "k must be in [1, 1024]");
    BPQ_CHECK(cfg->max_batch >= 1 && cfg->max_batch <= (1 << 20), BPQ_EINVAL, "max_batch must be in [1, 2^20]");
    BPQ_CHECK(cfg->L_max >= 1 && cfg->L_max < ((int64_t)1 << 31), BPQ_EINVAL, "L_max must be in [1, 2^31)");
    BPQ_CHECK(cfg->scorer >= BPQ_SCORER_FBPQ && cfg->scorer <= BPQ_SCORER_HBPQ_RECON, BPQ_EINVAL, "bad scorer");
    const bool local = cfg->scorer == BPQ_SCORER_HBPQ || cfg->scorer == BPQ_SCORER_HBPQ_RECON;
    BPQ_CHECK(local == (ix->p.variant == BPQ_VARIANT_LOCAL), BPQ_EINVAL, "scorer does not match the codebook variant");
    const size_t one = bpq_search_workspace_size(ix, 1, cfg->L_max, cfg->k, cfg->scorer);
    const size_t share = cfg->device_bytes / (size_t)cfg->slots;
    BPQ_CHECK(share >= one, BPQ_ECAPACITY, "device_bytes / slots does not hold one query at L_max");
    Guard g(ix->device);
    auto* s = new bpq_server();
    try {
      s->ix = ix;
      s->cfg = *cfg;
      s->D = ix->p.D;
      const size_t full = bpq_search_workspace_size(ix, cfg->max_batch, cfg->L_max, cfg->k, cfg->scorer);
      for (int i = 0; i < cfg->slots; ++i) {
        s->slots.push_back(std::make_unique<Slot>());
        Slot& sl = *s->slots.back();
        BPQ_CUDA(cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking));
        BPQ_CUDA(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
        sl.ws_bytes = std::min(share, full);
        sl.ws.alloc(sl.ws_bytes);
        sl.q.alloc((size_t)cfg->max_batch * s->D * 4);
        sl.ids.alloc((size_t)cfg->max_batch * cfg->k * 4);
        sl.dists.alloc((size_t)cfg->max_batch * cfg->k * 4);
        BPQ_CUDA(cudaMallocHost(&sl.q_pin, (size_t)cfg->max_batch * s->D * 4));
        BPQ_CUDA(cudaMallocHost(&sl.L_pin, (size_t)cfg->max_batch * 4));
        BPQ_CUDA(cudaMallocHost(&sl.ids_pin, (size_t)cfg->max_batch * cfg->k * 4));
        BPQ_CUDA(cudaMallocHost(&sl.dists_pin, (size_t)cfg->max_batch * cfg->k * 4));
        sl.L64.resize(cfg->max_batch);
      }
      s->t0 = Clock::now();
    } catch (...) {
      release(s);
      delete s;
      throw;
    }
    *out = s;
  });
}

int bpq_server_submit(bpq_server* s, const float* queries_host, const int64_t* L_host, int64_t n,
                      int64_t* first_request_out) {
  return guarded([&] {
    BPQ_CHECK(s && (n == 0 || (queries_host && L_host)), BPQ_EINVAL, "NULL pointer");
    BPQ_CHECK(n >= 0, BPQ_EINVAL, "n < 0");
    for (int64_t i = 0; i < n; ++i)
      BPQ_CHECK(L_host[i] >= 1 && L_host[i] <= s->cfg.L_max, BPQ_EINVAL, "every L must be in [1, L_max]");
    if (first_request_out) *first_request_out = s->next_id;
    const double t = s->now();
    for (int64_t i = 0; i < n; ++i) {
      Req r;
      r.id = s->next_id++;
      r.L = (int32_t)L_host[i];
      r.arrival = t;
      r.own.assign(queries_host + i * s->D, queries_host + (i + 1) * s->D);
      r.q = r.own.data();
      enqueue(s, std::move(r));
    }
  });
}

int bpq_server_progress(bpq_server* s, int32_t wait) {
  return guarded([&] {
    BPQ_CHECK(s, BPQ_EINVAL, "NULL pointer");
    Guard g(s->ix->device);
    int retired = retire(s, false);
    bool launched = false;
    while (any_pending(s) && launch_one(s)) launched = true;
    if (wait && !retired && !launched) {
      bool busy = false;
      for (const auto& sl : s->slots) busy |= sl->busy;
      if (busy) retire(s, true);
      while (any_pending(s) && launch_one(s)) {
      }
    }
  });
}

int bpq_server_take(bpq_server* s, int64_t max_n, int64_t* request_out, int32_t* ids_out, float* dists_out,
                    double* latency_s_out, int64_t* n_out) {
  return guarded([&] {
    BPQ_CHECK(s && n_out && max_n >= 0, BPQ_EINVAL, "bad argument");
    BPQ_CHECK(max_n == 0 || (request_out && ids_out && dists_out), BPQ_EINVAL, "NULL output");
    const int k = s->cfg.k;
    int64_t n = 0;
    while (n < max_n && !s->done.empty()) {
      const Done& d = s->done.front();
      request_out[n] = d.id;
      memcpy(ids_out + n * k, d.ids.data(), (size_t)k * 4);
      memcpy(dists_out + n * k, d.dists.data(), (size_t)k * 4);
      if (latency_s_out) latency_s_out[n] = d.finish - d.arrival;
      s->done.pop_front();
      ++n;
    }
    *n_out = n;
  });
}

int bpq_server_run_trace(bpq_server* s, const float* queries_host, const int64_t* L_host, const double* arrival_s,
                         int64_t n, int32_t* ids_out, float* dists_out, double* latency_s_out) {
  return guarded([&] {
    BPQ_CHECK(s && n >= 0, BPQ_EINVAL, "bad argument");
    if (n == 0) return;
    BPQ_CHECK(queries_host && L_host && arrival_s && ids_out && dists_out && latency_s_out, BPQ_EINVAL,
              "NULL pointer");
    for (int64_t i = 0; i < n; ++i) {
      BPQ_CHECK(L_host[i] >= 1 && L_host[i] <= s->cfg.L_max, BPQ_EINVAL, "every L must be in [1, L_max]");
      BPQ_CHECK(std::isfinite(arrival_s[i]) && (i == 0 || arrival_s[i] >= arrival_s[i - 1]), BPQ_EINVAL,
                "arrival times must be finite and non-decreasing");
    }
    bool busy0 = any_pending(s);
    for (const auto& sl : s->slots) busy0 |= sl->busy;
    BPQ_CHECK(!busy0, BPQ_ESTATE, "the server has requests in progress");
    Guard g(s->ix->device);
    s->trace_ids = ids_out;
    s->trace_dists = dists_out;
    s->trace_latency = latency_s_out;
    const int64_t id0 = s->next_id;
    try {
      s->t0 = Clock::now();
      int64_t next = 0, finished = 0;
      const int64_t q0 = s->queries;
      while (finished < n) {
        const double t = s->now();
        while (next < n && arrival_s[next] <= t) {
          Req r;
          r.id = next;  // trace requests index the caller's arrays
          r.L = (int32_t)L_host[next];
          r.arrival = arrival_s[next];
          r.q = queries_host + next * s->D;
          enqueue(s, std::move(r));
          ++next;
        }
        const int64_t before = s->queries;
        retire(s, false);
        while (any_pending(s) && launch_one(s)) {
        }
        int64_t inflight = 0;
        for (const auto& sl : s->slots) inflight += sl->busy;
        // every launched query whose slot is free again has been delivered
        finished = (s->queries - q0) - [&] {
          int64_t c = 0;
          for (const auto& sl : s->slots) c += sl->busy ? (int64_t)sl->reqs.size() : 0;
          return c;
        }();
        if (finished >= n) break;
        if (s->queries == before && inflight == 0 && next < n) {
          const double gap = arrival_s[next] - s->now();  // idle: wait for the next arrival
          if (gap > 3e-4) std::this_thread::sleep_for(std::chrono::duration<double>(gap - 2e-4));
        } else if (s->queries == before) {
          std::this_thread::yield();
        }
      }
    } catch (...) {
      s->trace_ids = nullptr;
      s->trace_dists = nullptr;
      s->trace_latency = nullptr;
      throw;
    }
    s->trace_ids = nullptr;
    s->trace_dists = nullptr;
    s->trace_latency = nullptr;
    s->next_id = id0;
  });
}

int bpq_server_get_stats(const bpq_server* s, bpq_server_stats* out) {
  return guarded([&] {
    BPQ_CHECK(s && out, BPQ_EINVAL, "NULL pointer");
    out->batches = s->batches;
    out->queries = s->queries;
    out->max_in_flight = s->max_in_flight;
    int64_t p = 0;
    for (const auto& q : s->pending) p += (int64_t)q.size();
    out->pending = p;
    out->slot_workspace_bytes = s->slots.empty() ? 0 : (int64_t)s->slots[0]->ws_bytes;
  });
}

void bpq_server_free(bpq_server* s) {
  if (!s) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(s->ix->device);
  release(s);
  delete s;
  if (prev >= 0) cudaSetDevice(prev);
}

}  // extern "C"
