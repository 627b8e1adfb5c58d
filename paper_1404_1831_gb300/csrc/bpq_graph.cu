// A search captured once as a CUDA graph and replayed: the whole bpq_search
// pipeline of one batch shape (query tables, traversal, HBPQ tables, scan or
// work-queue scan with its merge, every memset and the budget copy) becomes one
// graph launch, which removes the per-kernel launch cost that dominates small
// batches.  The graph reads the queries from, and writes the results to, the
// device buffers given at creation (static I/O buffers: the caller writes new
// queries there before a launch); per-query budgets are read at each launch from
// page-locked memory the graph owns, so they can change between launches up to
// the L_max of the capture.  The scan schedule (work-item size) is the one in
// force at capture, including a bpq_autotune choice for the batch's class.
#include <vector>

#include "bpq_internal.cuh"

struct bpq_graph {
  const bpq_index* ix = nullptr;
  int64_t nq = 0, L_max = 0, L_stride = 0;
  int32_t k = 0, scorer = 0;
  bpq::DevBuf ws;
  int32_t* L_pin = nullptr;
  std::vector<int64_t> L64;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

void release(bpq_graph* g) {
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->cap) cudaStreamDestroy(g->cap);
  if (g->L_pin) cudaFreeHost(g->L_pin);
  g->exec = nullptr;
  g->graph = nullptr;
  g->cap = nullptr;
  g->L_pin = nullptr;
}

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

}  // namespace

extern "C" {

int bpq_graph_create(bpq_graph** out, const bpq_index* ix, const float* queries_dev, int64_t nq,
                     const int64_t* L_host, int64_t L_stride, int32_t k, int32_t scorer, int32_t* ids_dev,
                     float* dists_dev) {
  return guarded([&] {
    BPQ_CHECK(out && ix && queries_dev && ids_dev && dists_dev && L_host, BPQ_EINVAL, "NULL pointer");
    *out = nullptr;
    BPQ_CHECK(ix->n_pending == 0, BPQ_ESTATE, "points were added since the last bpq_finalize");
    BPQ_CHECK(nq >= 1, BPQ_EINVAL, "nq must be >= 1");
    BPQ_CHECK(L_stride == 0 || L_stride == 1, BPQ_EINVAL, "L_stride must be 0 or 1");
    Guard gd(ix->device);
    auto* g = new bpq_graph();
    try {
      g->ix = ix;
      g->nq = nq;
      g->k = k;
      g->scorer = scorer;
      g->L_stride = L_stride;
      const int64_t n = L_stride ? nq : 1;
      g->L64.assign(L_host, L_host + n);
      for (int64_t v : g->L64) {
        BPQ_CHECK(v >= 1 && v < ((int64_t)1 << 31), BPQ_EINVAL, "every L must be in [1, 2^31)");
        g->L_max = std::max(g->L_max, v);
      }
      BPQ_CUDA(cudaMallocHost(&g->L_pin, (size_t)nq * 4));
      for (int64_t i = 0; i < nq; ++i) g->L_pin[i] = (int32_t)g->L64[L_stride ? i : 0];
      g->ws.alloc(bpq_search_workspace_size(ix, nq, g->L_max, k, scorer));
      BPQ_CUDA(cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking));
      // one uncaptured run (argument checks, function attributes), then the capture
      bpq::run_queries(*ix, queries_dev, nq, g->L64.data(), L_stride, k, scorer, ids_dev, dists_dev, nullptr, 0,
                       nullptr, nullptr, g->ws.p, g->ws.bytes, g->cap, L_stride ? g->L_pin : nullptr);
      BPQ_CUDA(cudaStreamSynchronize(g->cap));
      BPQ_CUDA(cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal));
      try {
        bpq::run_queries(*ix, queries_dev, nq, g->L64.data(), L_stride, k, scorer, ids_dev, dists_dev, nullptr, 0,
                         nullptr, nullptr, g->ws.p, g->ws.bytes, g->cap, L_stride ? g->L_pin : nullptr);
      } catch (...) {
        cudaGraph_t dropped = nullptr;
        cudaStreamEndCapture(g->cap, &dropped);
        if (dropped) cudaGraphDestroy(dropped);
        throw;
      }
      BPQ_CUDA(cudaStreamEndCapture(g->cap, &g->graph));
      BPQ_CUDA(cudaGraphInstantiate(&g->exec, g->graph, 0));
    } catch (...) {
      release(g);
      delete g;
      throw;
    }
    *out = g;
  });
}

int bpq_graph_set_budgets(bpq_graph* g, const int64_t* L_host) {
  return guarded([&] {
    BPQ_CHECK(g && L_host, BPQ_EINVAL, "NULL pointer");
    BPQ_CHECK(g->L_stride == 1, BPQ_EINVAL, "the graph was captured with one budget for every query");
    for (int64_t i = 0; i < g->nq; ++i)
      BPQ_CHECK(L_host[i] >= 1 && L_host[i] <= g->L_max, BPQ_EINVAL, "every L must be in [1, the capture's L_max]");
    for (int64_t i = 0; i < g->nq; ++i) g->L_pin[i] = (int32_t)L_host[i];
  });
}

int bpq_graph_launch(bpq_graph* g, void* stream) {
  return guarded([&] {
    BPQ_CHECK(g && g->exec, BPQ_EINVAL, "NULL graph");
    Guard gd(g->ix->device);
    BPQ_CUDA(cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)));
  });
}

void bpq_graph_free(bpq_graph* g) {
  if (!g) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(g->ix->device);
  if (g->cap) cudaStreamSynchronize(g->cap);
  release(g);
  delete g;
  if (prev >= 0) cudaSetDevice(prev);
}

}  // extern "C"
