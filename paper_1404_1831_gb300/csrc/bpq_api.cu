// C ABI entry points of libbpq (declared in include/bpq.h): index lifecycle,
// workspace layout and the query pipeline
//   tables (K1/K2) -> traversal (K4) -> scan + top-k (K5/K6)
// enqueued on the caller's stream, chunk by chunk when the workspace is small.
#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "bpq_internal.cuh"

namespace bpq {
bool ids_nonnegative(const int32_t* ids, int64_t n, cudaStream_t st);
}

using namespace bpq;

namespace {

thread_local std::string g_last_error;

template <typename F>
int guard(F&& f) {
  try {
    g_last_error.clear();
    f();
    return BPQ_OK;
  } catch (const Error& e) {
    g_last_error = e.what();
    return e.code;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return BPQ_ENOMEM;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return BPQ_EINVAL;
  }
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    BPQ_CUDA(cudaGetDevice(&prev));
    if (prev != dev) BPQ_CUDA(cudaSetDevice(dev));
  }
  ~DeviceGuard() {
    int cur = -1;
    if (cudaGetDevice(&cur) == cudaSuccess && cur != prev && prev >= 0) cudaSetDevice(prev);
  }
};

void check_params(const bpq_params* p) {
  BPQ_CHECK(p, BPQ_EINVAL, "params is NULL");
  BPQ_CHECK(p->ksub == KSUB, BPQ_EINVAL, "ksub must be 256");
  BPQ_CHECK(p->D > 0 && p->D % 2 == 0, BPQ_EINVAL, "D must be positive and even");
  BPQ_CHECK(p->M > 0 && p->M % 2 == 0 && (p->D / 2) % (p->M / 2) == 0, BPQ_EINVAL,
            "M must be even with D/M dividing D/2");
  BPQ_CHECK(p->T >= 1 && p->T <= MAX_T, BPQ_EINVAL, "T must be in [1, 4096]");
  BPQ_CHECK(p->variant == BPQ_VARIANT_GLOBAL || p->variant == BPQ_VARIANT_LOCAL, BPQ_EINVAL, "bad variant");
  BPQ_CHECK(p->kmeans_iters >= 0 && p->kmeans_iters <= 1000, BPQ_EINVAL, "kmeans_iters out of range");
  BPQ_CHECK(p->opq == 0 || p->opq == 1, BPQ_EINVAL, "opq must be 0 or 1");
  BPQ_CHECK(!p->opq || p->variant == BPQ_VARIANT_GLOBAL, BPQ_EINVAL, "OPQ rotations are built for the global codebooks");
  BPQ_CHECK(scan_supported(p->D, p->M), BPQ_EINVAL,
            "this build supports (D, M) in {(128, 8), (128, 16), (384, 8), (32, 8), (8, 8)}");
}

bpq_index* new_index(const bpq_params* p, int device) {
  check_params(p);
  int ndev = 0;
  BPQ_CUDA(cudaGetDeviceCount(&ndev));
  BPQ_CHECK(device >= 0 && device < ndev, BPQ_EINVAL, "bad device ordinal");
  auto* ix = new bpq_index();
  ix->p = *p;
  ix->device = device;
  ix->h = p->D / 2;
  ix->s = p->D / p->M;
  ix->m2 = p->M / 2;
  BPQ_CUDA(cudaDeviceGetAttribute(&ix->sm_count, cudaDevAttrMultiProcessorCount, device));
  return ix;
}

void empty_lists(bpq_index& ix, cudaStream_t st) {
  const int64_t nc = (int64_t)ix.p.T * ix.p.T + 1;
  ix.offsets.alloc(nc * 4);
  BPQ_CUDA(cudaMemsetAsync(ix.offsets.p, 0, nc * 4, st));
  ix.n_points = ix.n_nonempty = ix.max_cell = 0;
}

size_t cb_floats_R(const bpq_params& p) { return (size_t)p.M * KSUB * (p.D / p.M); }
size_t cb_floats_local(const bpq_params& p) { return (size_t)p.T * (p.M / 2) * KSUB * (p.D / p.M); }

// ---------------------------------------------------------------------------
// Workspace layout for a chunk of nq queries.
// ---------------------------------------------------------------------------
bool uses_lut(int scorer);

// The HBPQ table form (BPQ_SCORER_HBPQ, k <= 128) adds per query its table slots
// and bitmaps, per half-cell the bitmap of visiting queries, and the tables.
bool hbpq_tables_used(int scorer, int k) { return scorer == BPQ_SCORER_HBPQ && k <= 128; }

// Table slots expected for a query at budget L: about 4 sqrt(L / rho) + 32 distinct
// rows and columns (the visited cells of a query fill a region of the key grid a
// few times wider than sqrt(#cells) in each direction; rho = points per non-empty
// cell), at most 2T.  A query whose slots do not fit is scored by the O(D) form.
double hbpq_slots_per_query(const bpq_index& ix, double L) {
  if (ix.hb_slots_per_query > 0.0) return ix.hb_slots_per_query;
  const double rho = std::max(1.0, (double)ix.n_points / (double)std::max<int64_t>(1, ix.n_nonempty));
  return std::min(2.0 * ix.p.T, 4.0 * std::ceil(std::sqrt(std::max(1.0, L / rho))) + 32.0);
}

// Table offsets are 32-bit float indices in the scan.
int64_t hbpq_slot_limit(const bpq_index& ix) { return (((int64_t)1 << 32) - 1) / ((int64_t)ix.m2 * KSUB); }

struct Layout {
  size_t status, qcounter, L, d1, d2, lut, cells, ncells, npoints, total;
  size_t hb_qbase, hb_qrows, hb_qbits, hb_hmap, hb_ctr, hb_fb, hb_tab;
  size_t wq_ctr, wq_items, wq_merges, wq_pids, wq_pdists;  // work-queue scan
  size_t rq_c, rq_r;  // OPQ: rot0 q and B rot0 q of the chunk's queries
  size_t fb_list, fb_n, fb_handed;  // the traversal's handed-over queries (overlapped passes)
  bool overlap;
  int64_t cap, hb_slots;
  bool wq;
};

// The persistent work-queue form of the segment scans (FBPQ per-point and the
// HBPQ table form, k <= 128) when a work-item size W > 0 is in force.
bool work_queue_used(int W, int scorer, int k) {
  return W > 0 && k <= 128 && (scorer == BPQ_SCORER_FBPQ || scorer == BPQ_SCORER_HBPQ);
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

Layout layout(const bpq_index& ix, int64_t nq, int64_t L_max, int scorer, bool with_cells, int k = 1,
              double hb_per_query = 0.0, int work_W = -1) {
  if (work_W < 0) work_W = ix.scan_work_W;
  Layout l{};
  size_t o = 0;
  l.status = o;
  o = align_up(o + 4);
  l.qcounter = o;
  o = align_up(o + 4);
  l.L = o;
  o = align_up(o + (size_t)nq * 4);
  l.d1 = o;
  o = align_up(o + (size_t)nq * ix.p.T * 4);
  l.d2 = o;
  o = align_up(o + (size_t)nq * ix.p.T * 4);
  l.lut = o;
  if (uses_lut(scorer) && with_cells) o = align_up(o + (size_t)nq * ix.p.M * KSUB * 4);
  // visited cells per query: at most the non-empty cells the traversal sees (the
  // whole index's for a point shard)
  const int64_t nonempty = ix.goffsets.p ? ix.g_nonempty : ix.n_nonempty;
  l.cap = std::max<int64_t>(1, std::min<int64_t>(L_max, std::max<int64_t>(nonempty, 1)));
  l.cells = o;
  if (with_cells) o = align_up(o + (size_t)nq * l.cap * sizeof(bpq_cell));
  l.ncells = o;
  o = align_up(o + (size_t)nq * 4);
  l.npoints = o;
  o = align_up(o + (size_t)nq * 8);
  if (ix.opq) {
    l.rq_c = o;
    o = align_up(o + (size_t)nq * ix.p.D * 4);
    l.rq_r = o;
    o = align_up(o + (size_t)nq * ix.p.D * 4);
  }
  if (with_cells && hbpq_tables_used(scorer, k)) {
    const int TW = (ix.p.T + 31) / 32;
    if (hb_per_query <= 0.0) hb_per_query = hbpq_slots_per_query(ix, (double)L_max);
    l.hb_slots = std::min<int64_t>(hbpq_slot_limit(ix), (int64_t)std::ceil(hb_per_query * (double)nq));
    l.hb_qbase = o;
    o = align_up(o + (size_t)nq * 4);
    l.hb_qrows = o;
    o = align_up(o + (size_t)nq * 4);
    l.hb_qbits = o;
    o = align_up(o + (size_t)nq * 2 * TW * 4);
    l.hb_hmap = o;
    o = align_up(o + (size_t)2 * ix.p.T * ((nq + 31) / 32) * 4);
    l.hb_ctr = o;
    o = align_up(o + 16);
    l.hb_fb = o;
    o = align_up(o + (size_t)nq * 4);
    l.hb_tab = o;
    o = align_up(o + (size_t)l.hb_slots * ix.m2 * KSUB * 4);
  }
  l.wq = with_cells && work_queue_used(work_W, scorer, k);
  // FBPQ segment scan: the traversal's CTA pass and the scan of the queries it
  // takes run beside the scan of the others
  l.overlap = with_cells && scorer == BPQ_SCORER_FBPQ && k <= 128 && !l.wq && ix.p.T <= 1024 && !ix.goffsets.p;
  if (l.overlap) {
    l.fb_n = o;
    o = align_up(o + 4);
    l.fb_list = o;
    o = align_up(o + (size_t)nq * 4);
    l.fb_handed = o;
    o = align_up(o + (size_t)nq);
  }
  if (l.wq) {
    const size_t parts = (size_t)nq * SCAN_MAX_ITEMS;
    l.wq_ctr = o;
    o = align_up(o + 16);
    l.wq_items = o;
    o = align_up(o + parts * 16);
    l.wq_merges = o;
    o = align_up(o + (size_t)nq * 16);
    l.wq_pids = o;
    o = align_up(o + parts * k * 4);
    l.wq_pdists = o;
    o = align_up(o + parts * k * 4);
  }
  l.total = o;
  return l;
}

int64_t read_L(const int64_t* L_host, int64_t L_stride, int64_t nq, std::vector<int32_t>* per_query) {
  BPQ_CHECK(L_host, BPQ_EINVAL, "L is NULL");
  BPQ_CHECK(L_stride == 0 || L_stride == 1, BPQ_EINVAL, "L_stride must be 0 or 1");
  int64_t L_max = 0;
  const int64_t n = L_stride ? nq : 1;
  if (per_query && L_stride) per_query->resize(nq);
  for (int64_t i = 0; i < n; ++i) {
    const int64_t v = L_host[i];
    BPQ_CHECK(v >= 1 && v < ((int64_t)1 << 31), BPQ_EINVAL, "every L must be in [1, 2^31)");
    L_max = std::max(L_max, v);
    if (per_query && L_stride) (*per_query)[i] = (int32_t)v;
  }
  return L_max;
}

// The traversal's cell counts and mean points per non-empty cell: the whole
// index's for a point shard, else the index's own.
const uint32_t* traversal_offsets(const bpq_index& ix) {
  return ix.goffsets.p ? ix.goffsets.as<uint32_t>() : ix.offsets.as<uint32_t>();
}
float traversal_rho(const bpq_index& ix) {
  if (ix.goffsets.p) return (float)((double)ix.g_points / (double)std::max<int64_t>(1, ix.g_nonempty));
  return (float)((double)ix.n_points / (double)std::max<int64_t>(1, ix.n_nonempty));
}

void check_searchable(const bpq_index* ix) {
  BPQ_CHECK(ix, BPQ_EINVAL, "index is NULL");
  BPQ_CHECK(ix->n_pending == 0, BPQ_ESTATE, "points were added since the last bpq_finalize");
}

ScanArgs scan_args(const bpq_index& ix, const float* q, int64_t nq, const float* lut, const bpq_cell* cells,
                   const int32_t* ncells, int32_t cap, int k, int32_t* ids, float* dists, int32_t* counter) {
  ScanArgs sa{};
  sa.cells = cells;
  sa.ncells = ncells;
  sa.cap = cap;
  sa.nq = nq;
  sa.T = ix.p.T;
  sa.M = ix.p.M;
  sa.D = ix.p.D;
  sa.k = k;
  sa.lut = lut;
  sa.X1 = ix.X1.as<float>();
  sa.X2 = ix.X2.as<float>();
  sa.cross = ix.cross.as<float>();
  sa.queries = q;
  sa.C1 = ix.opq ? ix.C1r.as<float>() : ix.C1.as<float>();  // the reconstruction's centroids
  sa.C2 = ix.opq ? ix.C2r.as<float>() : ix.C2.as<float>();  // (residual space with OPQ)
  sa.R = ix.R.as<float>();
  sa.Q = ix.Q.as<float>();
  sa.S = ix.S.as<float>();
  sa.codes = ix.codes.as<uint8_t>();
  sa.ids = ix.ids.as<int32_t>();
  sa.out_ids = ids;
  sa.out_dists = dists;
  sa.qcounter = counter;
  sa.sm_count = ix.sm_count;
  return sa;
}

bool uses_lut(int scorer) { return scorer == BPQ_SCORER_FBPQ || scorer == BPQ_SCORER_FBPQ_TABLES; }

void check_scorer(const bpq_index& ix, int scorer) {
  BPQ_CHECK(scorer >= BPQ_SCORER_FBPQ && scorer <= BPQ_SCORER_HBPQ_RECON, BPQ_EINVAL, "bad scorer");
  if (scorer == BPQ_SCORER_HBPQ || scorer == BPQ_SCORER_HBPQ_RECON)
    BPQ_CHECK(ix.p.variant == BPQ_VARIANT_LOCAL, BPQ_EINVAL, "the HBPQ scorer needs local codebooks");
  else
    BPQ_CHECK(ix.p.variant == BPQ_VARIANT_GLOBAL, BPQ_EINVAL, "FBPQ and reconstruction scorers need global codebooks");
}

}  // namespace

// Runs tables + traversal (+ scan when ids/dists are given) over the queries in
// chunks that fit the workspace.  L32_pinned (optional, per-query budgets only):
// the same budgets as int32 in page-locked host memory, copied from there so that
// no pageable copy stalls the host on the stream.
namespace {

// A second stream per (device, caller stream) for the overlapped passes, with
// the fork and join events; created on first use and kept for the process.
struct AuxStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr, lut = nullptr;
  std::mutex m;  // one caller at a time enqueues the fork ... join sequence
};

AuxStream* aux_stream(cudaStream_t st) {
  static std::mutex pool_m;
  static std::map<std::pair<int, cudaStream_t>, std::unique_ptr<AuxStream>> pool;
  int dev = 0;
  BPQ_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> g(pool_m);
  auto it = pool.find({dev, st});
  if (it != pool.end()) return it->second.get();
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  BPQ_CUDA(cudaStreamIsCapturing(st, &cs));
  if (cs != cudaStreamCaptureStatusNone || pool.size() >= 256) return nullptr;  // no new stream: one pass after the other
  auto a = std::make_unique<AuxStream>();
  BPQ_CUDA(cudaStreamCreateWithFlags(&a->s, cudaStreamNonBlocking));
  BPQ_CUDA(cudaEventCreateWithFlags(&a->fork, cudaEventDisableTiming));
  BPQ_CUDA(cudaEventCreateWithFlags(&a->join, cudaEventDisableTiming));
  BPQ_CUDA(cudaEventCreateWithFlags(&a->lut, cudaEventDisableTiming));
  AuxStream* r = a.get();
  pool.emplace(std::make_pair(dev, st), std::move(a));
  return r;
}

}  // namespace

void bpq::run_queries(const bpq_index& ix, const float* q, int64_t nq, const int64_t* L_host, int64_t L_stride,
                      int k, int scorer, int32_t* out_ids, float* out_dists, bpq_cell* user_cells, int32_t user_cap,
                      int32_t* user_ncells, int64_t* user_npoints, void* ws, size_t ws_bytes, cudaStream_t st,
                      const int32_t* L32_pinned) {
  const bool scan = user_cells == nullptr;
  std::vector<int32_t> Lq;
  const int64_t L_max = read_L(L_host, L_stride, nq, &Lq);
  if (scan) {
    BPQ_CHECK(k >= 1 && k <= MAX_K, BPQ_EINVAL, "k must be in [1, 1024]");
    check_scorer(ix, scorer);
  } else {
    BPQ_CHECK(user_cap >= 1, BPQ_EINVAL, "cap must be >= 1");
  }
  if (nq <= 0) return;
  BPQ_CHECK(q, BPQ_EINVAL, "queries is NULL");
  BPQ_CHECK(ws, BPQ_EINVAL, "workspace is NULL");
  if (scan)
    BPQ_CHECK(out_ids && out_dists, BPQ_EINVAL, "output pointers are NULL");
  else
    BPQ_CHECK(user_ncells && user_npoints, BPQ_EINVAL, "bad traversal outputs");
  const bool hb = scan && hbpq_tables_used(scorer, k);
  // HBPQ table slots per query: the mean of the per-query expectation
  double hb_per_query = 0.0;
  if (hb) {
    if (L_stride) {
      for (int32_t v : Lq) hb_per_query += hbpq_slots_per_query(ix, (double)v);
      hb_per_query /= (double)nq;
    } else {
      hb_per_query = hbpq_slots_per_query(ix, (double)L_max);
    }
  }
  // work-item size: the autotuner's choice for this batch class, else the index's setting
  int work_W = ix.scan_work_W;
  if (scan && !ix.tuned_W.empty()) {
    double Lm = (double)L_max;
    if (L_stride) {
      Lm = 0.0;
      for (int32_t v : Lq) Lm += v;
      Lm /= (double)nq;
    }
    const auto it = ix.tuned_W.find(tune_key(scorer, k, nq, Lm));
    if (it != ix.tuned_W.end()) work_W = it->second;
  }
  auto lay = [&](int64_t n) { return layout(ix, n, L_max, scorer, scan, k, hb_per_query, work_W); };
  // largest chunk that fits the workspace (and, for HBPQ, whose table offsets fit 32 bits)
  auto fits = [&](int64_t n) {
    return lay(n).total <= ws_bytes && !(hb && hb_per_query * (double)n > (double)hbpq_slot_limit(ix));
  };
  int64_t chunk = nq;
  if (!fits(chunk)) {
    int64_t lo = 0, hi = nq;
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) / 2;
      if (fits(mid)) lo = mid; else hi = mid;
    }
    chunk = lo;
  }
  BPQ_CHECK(chunk >= 1, BPQ_ECAPACITY, "workspace too small for one query");
  const Layout l = lay(chunk);
  char* w = static_cast<char*>(ws);
  BPQ_CUDA(cudaMemsetAsync(w + l.status, 0, 4, st));
  const float rho = traversal_rho(ix);
  for (int64_t c0 = 0; c0 < nq; c0 += chunk) {
    const int64_t nc = std::min(chunk, nq - c0);
    const float* qc = q + c0 * ix.p.D;
    float* d1 = reinterpret_cast<float*>(w + l.d1);
    float* d2 = reinterpret_cast<float*>(w + l.d2);
    float* lut = (scan && uses_lut(scorer)) ? reinterpret_cast<float*>(w + l.lut) : nullptr;
    // OPQ: the coarse tables and the traversal use rot0 q, the PQ table and the
    // reconstruction scorer B rot0 q (with the rotated centroids)
    const float* qcoarse = qc;
    const float* qres = qc;
    if (ix.opq) {
      float* rc = reinterpret_cast<float*>(w + l.rq_c);
      float* rr = reinterpret_cast<float*>(w + l.rq_r);
      rotate_queries(ix, qc, nc, rc, rr, st);
      qcoarse = rc;
      qres = rr;
    }
    // FBPQ segment scan: the PQ table is built on the second stream beside the
    // coarse tables and the traversal (only the scans read it)
    AuxStream* aux = (scan && l.overlap) ? aux_stream(st) : nullptr;
    std::unique_lock<std::mutex> aux_lock;  // held from the fork to the join
    int32_t* status = reinterpret_cast<int32_t*>(w + l.status);
    if (aux && lut) {
      aux_lock = std::unique_lock<std::mutex>(aux->m);
      BPQ_CUDA(cudaEventRecord(aux->fork, st));
      BPQ_CUDA(cudaStreamWaitEvent(aux->s, aux->fork, 0));
      launch_query_tables(ix, qcoarse, nc, nullptr, nullptr, lut, aux->s, status, qres);
      BPQ_CUDA(cudaEventRecord(aux->lut, aux->s));
      launch_query_tables(ix, qcoarse, nc, d1, d2, nullptr, st, status, qres);
    } else {
      aux = nullptr;
      launch_query_tables(ix, qcoarse, nc, d1, d2, lut, st, status, qres);
    }
    TraverseArgs ta{};
    ta.d1 = d1;
    ta.d2 = d2;
    ta.offsets = traversal_offsets(ix);
    if (L_stride) {
      BPQ_CUDA(cudaMemcpyAsync(w + l.L, (L32_pinned ? L32_pinned : Lq.data()) + c0, nc * 4, cudaMemcpyHostToDevice, st));
      ta.L = reinterpret_cast<const int32_t*>(w + l.L);
    } else {
      ta.L = nullptr;
      ta.L_scalar = (int32_t)L_host[0];
    }
    ta.T = ix.p.T;
    ta.rho = rho;
    ta.ordered = scan ? 0 : 1;
    ta.status = reinterpret_cast<int32_t*>(w + l.status);
    ta.nq = nc;
    if (scan) {
      ta.cap = (int32_t)l.cap;
      ta.cells = reinterpret_cast<bpq_cell*>(w + l.cells);
      ta.ncells = reinterpret_cast<int32_t*>(w + l.ncells);
      ta.npoints = reinterpret_cast<int64_t*>(w + l.npoints);
    } else {
      ta.cap = user_cap;
      ta.cells = user_cells + c0 * user_cap;
      ta.ncells = user_ncells + c0;
      ta.npoints = user_npoints + c0;
    }
    ScanArgs sa = scan_args(ix, qres, nc, lut, ta.cells, ta.ncells, ta.cap, k, out_ids + c0 * k,
                            out_dists + c0 * k, reinterpret_cast<int32_t*>(w + l.qcounter));
    if (aux) {
      // the warp pass lists the queries it hands over; the CTA pass for them, then
      // their scan, run on the second stream (after the PQ table) beside the scan
      // of the other queries
      ta.fb_n = reinterpret_cast<int32_t*>(w + l.fb_n);
      ta.fb_list = reinterpret_cast<int32_t*>(w + l.fb_list);
      ta.handed = reinterpret_cast<uint8_t*>(w + l.fb_handed);
      BPQ_CUDA(cudaMemsetAsync(ta.fb_n, 0, 4, st));
      if (launch_traverse_warp(ta, st)) {
        BPQ_CUDA(cudaEventRecord(aux->fork, st));
        BPQ_CUDA(cudaStreamWaitEvent(aux->s, aux->fork, 0));
        launch_traverse_marked(ta, aux->s);
        ScanArgs sb = sa;
        sb.sel = ta.fb_list;
        sb.sel_n = ta.fb_n;
        launch_scan(sb, scorer, aux->s);
        BPQ_CUDA(cudaStreamWaitEvent(st, aux->lut, 0));
        sa.skip = ta.handed;
        launch_scan(sa, scorer, st);
        BPQ_CUDA(cudaEventRecord(aux->join, aux->s));
        BPQ_CUDA(cudaStreamWaitEvent(st, aux->join, 0));
      } else {
        BPQ_CUDA(cudaStreamWaitEvent(st, aux->lut, 0));
        launch_scan(sa, scorer, st);  // the CTA pass took every query
      }
      aux_lock.unlock();
      continue;
    }
    launch_traverse(ta, st);
    if (ix.goffsets.p) launch_localize_cells(ta, ix.offsets.as<uint32_t>(), st);
    if (!scan) continue;
    if (hb) {
      // per-(query, visited half-cell) tables on the tensor cores, then the M-lookup scan
      HbpqArgs h{};
      h.cells = ta.cells;
      h.ncells = ta.ncells;
      h.cap = ta.cap;
      h.nq = nc;
      h.T = ix.p.T;
      h.M = ix.p.M;
      h.D = ix.p.D;
      h.queries = qc;
      h.qbase = reinterpret_cast<int32_t*>(w + l.hb_qbase);
      h.qrows = reinterpret_cast<int32_t*>(w + l.hb_qrows);
      h.qbits = reinterpret_cast<uint32_t*>(w + l.hb_qbits);
      h.hmap = reinterpret_cast<uint32_t*>(w + l.hb_hmap);
      h.slot_counter = reinterpret_cast<unsigned long long*>(w + l.hb_ctr);
      h.fb_count = reinterpret_cast<int32_t*>(w + l.hb_ctr + 8);
      h.fallback = reinterpret_cast<int32_t*>(w + l.hb_fb);
      h.slot_cap = l.hb_slots;
      h.tables = reinterpret_cast<float*>(w + l.hb_tab);
      h.status = reinterpret_cast<int32_t*>(w + l.status);
      BPQ_CUDA(cudaMemsetAsync(w + l.hb_hmap, 0, (size_t)2 * ix.p.T * ((nc + 31) / 32) * 4, st));
      BPQ_CUDA(cudaMemsetAsync(w + l.hb_ctr, 0, 16, st));
      launch_hbpq_pairs(h, st);
      launch_hbpq_tables(ix, h, st);
      sa.hb_qbase = h.qbase;
      sa.hb_qrows = h.qrows;
      sa.hb_qbits = h.qbits;
      sa.hb_tables = h.tables;
      sa.qlist = h.fallback;
      sa.qlist_n = h.fb_count;
    }
    if (l.wq) {
      sa.work_W = work_W;
      int32_t* ctr = reinterpret_cast<int32_t*>(w + l.wq_ctr);
      sa.n_items = ctr;
      sa.item_counter = ctr + 1;
      sa.part_counter = ctr + 2;
      sa.n_merges = ctr + 3;
      sa.items = reinterpret_cast<int4*>(w + l.wq_items);
      sa.merges = reinterpret_cast<int4*>(w + l.wq_merges);
      sa.part_ids = reinterpret_cast<int32_t*>(w + l.wq_pids);
      sa.part_dists = reinterpret_cast<float*>(w + l.wq_pdists);
    }
    launch_scan(sa, scorer, st);
  }
}

namespace {

// ---------------------------------------------------------------------------
// bpq_search_shortlist: the bpq_search layout plus the reduced-precision tables
// (sized for the 2-byte FP16 form; the int8 form uses the first half), their
// steps and the shortlists.
// ---------------------------------------------------------------------------
struct ShortlistLayout {
  Layout base;
  size_t lutr, scale, sl, hint, total;
};

ShortlistLayout shortlist_layout(const bpq_index& ix, int64_t nq, int64_t L_max, int S) {
  ShortlistLayout l{};
  l.base = layout(ix, nq, L_max, BPQ_SCORER_FBPQ, true);
  size_t o = l.base.total;
  l.lutr = o;
  o = align_up(o + (size_t)nq * ix.p.M * KSUB * 2);
  l.scale = o;
  o = align_up(o + (size_t)nq * 4);
  l.sl = o;
  o = align_up(o + (size_t)nq * S * 8);
  l.hint = o;
  o = align_up(o + position_hint_count(ix.n_points) * 4);
  l.total = o;
  return l;
}

void run_shortlist(const bpq_index& ix, const float* q, int64_t nq, const int64_t* L_host, int64_t L_stride, int k,
                   int S, bool f16, int32_t* out_ids, float* out_dists, void* ws, size_t ws_bytes, cudaStream_t st) {
  std::vector<int32_t> Lq;
  const int64_t L_max = read_L(L_host, L_stride, nq, &Lq);
  BPQ_CHECK(k >= 1 && S >= k && S <= MAX_K, BPQ_EINVAL, "need 1 <= k <= shortlist <= 1024");
  check_scorer(ix, BPQ_SCORER_FBPQ);
  BPQ_CHECK(ix.p.D == 128 && (ix.p.M == 8 || ix.p.M == 16), BPQ_EINVAL,
            "the reduced-precision shortlist is built for D = 128, M = 8 or 16");
  if (nq <= 0) return;
  BPQ_CHECK(q && ws && out_ids && out_dists, BPQ_EINVAL, "NULL pointer");
  int64_t chunk = nq;
  if (shortlist_layout(ix, chunk, L_max, S).total > ws_bytes) {
    int64_t lo = 0, hi = nq;
    while (hi - lo > 1) {
      const int64_t mid = (lo + hi) / 2;
      if (shortlist_layout(ix, mid, L_max, S).total <= ws_bytes) lo = mid; else hi = mid;
    }
    chunk = lo;
  }
  BPQ_CHECK(chunk >= 1, BPQ_ECAPACITY, "workspace too small for one query");
  const ShortlistLayout l = shortlist_layout(ix, chunk, L_max, S);
  char* w = static_cast<char*>(ws);
  BPQ_CUDA(cudaMemsetAsync(w + l.base.status, 0, 4, st));
  const float rho = traversal_rho(ix);
  // the re-score's cell hints of the list positions (every chunk uses them)
  launch_position_hints(ix.offsets.as<uint32_t>(), (int64_t)ix.p.T * ix.p.T, ix.n_points,
                        reinterpret_cast<uint32_t*>(w + l.hint), st);
  for (int64_t c0 = 0; c0 < nq; c0 += chunk) {
    const int64_t nc = std::min(chunk, nq - c0);
    const float* qc = q + c0 * ix.p.D;
    float* d1 = reinterpret_cast<float*>(w + l.base.d1);
    float* d2 = reinterpret_cast<float*>(w + l.base.d2);
    float* lut = reinterpret_cast<float*>(w + l.base.lut);
    void* lutr = w + l.lutr;
    float* scale = reinterpret_cast<float*>(w + l.scale);
    uint64_t* sl = reinterpret_cast<uint64_t*>(w + l.sl);
    const float* qcoarse = qc;
    const float* qres = qc;
    if (ix.opq) {
      float* rc = reinterpret_cast<float*>(w + l.base.rq_c);
      float* rr = reinterpret_cast<float*>(w + l.base.rq_r);
      rotate_queries(ix, qc, nc, rc, rr, st);
      qcoarse = rc;
      qres = rr;
    }
    launch_query_tables(ix, qcoarse, nc, d1, d2, lut, st, nullptr, qres);
    launch_quant_lut(lut, ix.p.M, nc, lutr, scale, f16, st);
    TraverseArgs ta{};
    ta.d1 = d1;
    ta.d2 = d2;
    ta.offsets = traversal_offsets(ix);
    if (L_stride) {
      BPQ_CUDA(cudaMemcpyAsync(w + l.base.L, Lq.data() + c0, nc * 4, cudaMemcpyHostToDevice, st));
      ta.L = reinterpret_cast<const int32_t*>(w + l.base.L);
    } else {
      ta.L = nullptr;
      ta.L_scalar = (int32_t)L_host[0];
    }
    ta.T = ix.p.T;
    ta.rho = rho;
    ta.ordered = 0;
    ta.status = reinterpret_cast<int32_t*>(w + l.base.status);
    ta.nq = nc;
    ta.cap = (int32_t)l.base.cap;
    ta.cells = reinterpret_cast<bpq_cell*>(w + l.base.cells);
    ta.ncells = reinterpret_cast<int32_t*>(w + l.base.ncells);
    ta.npoints = reinterpret_cast<int64_t*>(w + l.base.npoints);
    launch_traverse(ta, st);
    if (ix.goffsets.p) launch_localize_cells(ta, ix.offsets.as<uint32_t>(), st);
    ScanArgs sa = scan_args(ix, qc, nc, lut, ta.cells, ta.ncells, ta.cap, S, nullptr, nullptr,
                            reinterpret_cast<int32_t*>(w + l.base.qcounter));
    sa.lut8 = static_cast<const uint8_t*>(lutr);
    sa.lut16 = static_cast<const uint16_t*>(lutr);
    sa.lut_scale = scale;
    sa.sl_out = sl;
    sa.status = ta.status;
    launch_scan_reduced(sa, f16, st);
    RescoreArgs r{};
    r.sl = sl;
    r.S = S;
    r.k = k;
    r.T = ix.p.T;
    r.M = ix.p.M;
    r.nq = nc;
    r.d1 = d1;
    r.d2 = d2;
    r.lut = lut;
    r.offsets = ix.offsets.as<uint32_t>();
    r.hint = reinterpret_cast<const uint32_t*>(w + l.hint);
    r.codes = ix.codes.as<uint8_t>();
    r.cross = ix.cross.as<float>();
    r.ids = ix.ids.as<int32_t>();
    r.out_ids = out_ids + c0 * k;
    r.out_dists = out_dists + c0 * k;
    launch_rescore(r, st);
  }
}

// ---------------------------------------------------------------------------
// File format: magic, version, params, n_points, then sections
// (u64 size, bytes, u64 FNV-1a checksum).
// ---------------------------------------------------------------------------
const char MAGIC[8] = {'B', 'P', 'Q', 'I', 'D', 'X', 0, 1};

uint64_t fnv1a(const void* data, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(data);
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

struct File {
  FILE* f = nullptr;
  ~File() {
    if (f) fclose(f);
  }
};

void write_section(FILE* f, const void* dev, size_t bytes) {
  std::vector<unsigned char> host(bytes);
  if (bytes) BPQ_CUDA(cudaMemcpy(host.data(), dev, bytes, cudaMemcpyDeviceToHost));
  uint64_t n = bytes, h = fnv1a(host.data(), bytes);
  BPQ_CHECK(fwrite(&n, 8, 1, f) == 1 && (bytes == 0 || fwrite(host.data(), 1, bytes, f) == bytes) &&
                fwrite(&h, 8, 1, f) == 1,
            BPQ_EIO, "write failed");
}

void write_host_section(FILE* f, const void* data, size_t bytes) {
  uint64_t n = bytes, h = fnv1a(data, bytes);
  BPQ_CHECK(fwrite(&n, 8, 1, f) == 1 && (bytes == 0 || fwrite(data, 1, bytes, f) == bytes) && fwrite(&h, 8, 1, f) == 1,
            BPQ_EIO, "write failed");
}

void read_host_section(FILE* f, std::vector<double>& dst, size_t count) {
  uint64_t n = 0, h = 0;
  BPQ_CHECK(fread(&n, 8, 1, f) == 1 && n == count * 8, BPQ_ECORRUPT, "index file section has the wrong size");
  dst.resize(count);
  BPQ_CHECK((count == 0 || fread(dst.data(), 8, count, f) == count) && fread(&h, 8, 1, f) == 1, BPQ_ECORRUPT,
            "truncated index file");
  BPQ_CHECK(h == fnv1a(dst.data(), count * 8), BPQ_ECORRUPT, "index file checksum mismatch");
}

void read_section(FILE* f, DevBuf& dst, size_t bytes) {
  uint64_t n = 0, h = 0;
  BPQ_CHECK(fread(&n, 8, 1, f) == 1, BPQ_ECORRUPT, "truncated index file");
  BPQ_CHECK(n == bytes, BPQ_ECORRUPT, "index file section has the wrong size");
  std::vector<unsigned char> host(bytes);
  BPQ_CHECK((bytes == 0 || fread(host.data(), 1, bytes, f) == bytes) && fread(&h, 8, 1, f) == 1, BPQ_ECORRUPT,
            "truncated index file");
  BPQ_CHECK(h == fnv1a(host.data(), bytes), BPQ_ECORRUPT, "index file checksum mismatch");
  dst.alloc(bytes);
  if (bytes) BPQ_CUDA(cudaMemcpy(dst.p, host.data(), bytes, cudaMemcpyHostToDevice));
}

bpq_index* load_file(const char* path, int device) {
  File fh;
  fh.f = fopen(path, "rb");
  BPQ_CHECK(fh.f, BPQ_EIO, std::string("cannot open ") + path);
  char magic[8];
  uint32_t version = 0;
  bpq_params p{};
  int64_t n = 0;
  BPQ_CHECK(fread(magic, 8, 1, fh.f) == 1 && memcmp(magic, MAGIC, 8) == 0, BPQ_ECORRUPT, "not a bpq index file");
  BPQ_CHECK(fread(&version, 4, 1, fh.f) == 1 && (version == 1 || version == 2), BPQ_ECORRUPT,
            "unsupported index file version");
  // version 1 files end the params before the opq field
  const size_t psize = version == 1 ? offsetof(bpq_params, opq) : sizeof(p);
  BPQ_CHECK(fread(&p, psize, 1, fh.f) == 1 && fread(&n, 8, 1, fh.f) == 1, BPQ_ECORRUPT, "truncated header");
  try {
    check_params(&p);
  } catch (const Error& e) {
    throw Error(BPQ_ECORRUPT, std::string("bad params in index file: ") + e.what());
  }
  BPQ_CHECK(n >= 0 && n < ((int64_t)1 << 32) - 1, BPQ_ECORRUPT, "bad point count");
  bpq_index* ix = new_index(&p, device);
  try {
    DeviceGuard dg(device);
    const size_t hf = (size_t)p.T * (p.D / 2);
    read_section(fh.f, ix->C1, hf * 4);
    read_section(fh.f, ix->C2, hf * 4);
    read_section(fh.f, ix->R, cb_floats_R(p) * 4);
    if (p.variant == BPQ_VARIANT_LOCAL) {
      read_section(fh.f, ix->Q, cb_floats_local(p) * 4);
      read_section(fh.f, ix->S, cb_floats_local(p) * 4);
    }
    if (p.opq) {
      std::vector<double> r0, r1, r2;
      read_host_section(fh.f, r0, (size_t)p.D * p.D);
      read_host_section(fh.f, r1, (size_t)(p.D / 2) * (p.D / 2));
      read_host_section(fh.f, r2, (size_t)(p.D / 2) * (p.D / 2));
      set_opq_rotations(*ix, r0.data(), r1.data(), r2.data(), 0);
    }
    read_section(fh.f, ix->offsets, ((size_t)p.T * p.T + 1) * 4);
    read_section(fh.f, ix->codes, (size_t)n * p.M);
    read_section(fh.f, ix->ids, (size_t)n * 4);
    // consistency of the offsets with the point count, and the cell statistics
    std::vector<uint32_t> off((size_t)p.T * p.T + 1);
    BPQ_CUDA(cudaMemcpy(off.data(), ix->offsets.p, off.size() * 4, cudaMemcpyDeviceToHost));
    BPQ_CHECK(off[0] == 0 && off.back() == (uint64_t)n, BPQ_ECORRUPT, "offsets do not match the point count");
    int64_t nonempty = 0, maxc = 0;
    for (size_t c = 0; c + 1 < off.size(); ++c) {
      BPQ_CHECK(off[c + 1] >= off[c], BPQ_ECORRUPT, "offsets are not monotone");
      const int64_t cnt = off[c + 1] - off[c];
      nonempty += cnt > 0;
      maxc = std::max(maxc, cnt);
    }
    ix->n_points = n;
    ix->n_nonempty = nonempty;
    ix->max_cell = maxc;
    build_fbpq_tables(*ix, 0);
    build_hbpq_tables(*ix, 0);
    build_point_cross(*ix, 0);
    BPQ_CUDA(cudaDeviceSynchronize());
  } catch (...) {
    delete ix;
    throw;
  }
  return ix;
}

}  // namespace

void bpq::set_last_error(const std::string& msg) { g_last_error = msg; }

uint64_t bpq::tune_key(int scorer, int k, int64_t nq, double L_mean) {
  const uint64_t lq = (uint64_t)std::floor(std::log2((double)std::max<int64_t>(nq, 1)));
  const uint64_t lL = (uint64_t)std::floor(std::log2(std::max(1.0, L_mean)));
  return ((uint64_t)scorer << 24) | ((uint64_t)(k <= 32) << 20) | (lq << 8) | lL;
}

extern "C" {

const char* bpq_last_error(void) { return g_last_error.c_str(); }

int bpq_create(bpq_index** out, const bpq_params* p, const float* C1_host, const float* C2_host,
               const float* R_host, const float* Q_host, const float* S_host, int device) {
  return guard([&] {
    BPQ_CHECK(out, BPQ_EINVAL, "out is NULL");
    *out = nullptr;
    BPQ_CHECK(C1_host && C2_host && R_host, BPQ_EINVAL, "codebook pointer is NULL");
    bpq_index* ix = new_index(p, device);
    try {
      DeviceGuard dg(device);
      if (p->variant == BPQ_VARIANT_LOCAL) BPQ_CHECK(Q_host && S_host, BPQ_EINVAL, "local codebooks are NULL");
      const size_t hf = (size_t)p->T * (p->D / 2);
      ix->C1.alloc(hf * 4);
      ix->C2.alloc(hf * 4);
      ix->R.alloc(cb_floats_R(*p) * 4);
      BPQ_CUDA(cudaMemcpy(ix->C1.p, C1_host, hf * 4, cudaMemcpyHostToDevice));
      BPQ_CUDA(cudaMemcpy(ix->C2.p, C2_host, hf * 4, cudaMemcpyHostToDevice));
      BPQ_CUDA(cudaMemcpy(ix->R.p, R_host, cb_floats_R(*p) * 4, cudaMemcpyHostToDevice));
      if (p->variant == BPQ_VARIANT_LOCAL) {
        ix->Q.alloc(cb_floats_local(*p) * 4);
        ix->S.alloc(cb_floats_local(*p) * 4);
        BPQ_CUDA(cudaMemcpy(ix->Q.p, Q_host, cb_floats_local(*p) * 4, cudaMemcpyHostToDevice));
        BPQ_CUDA(cudaMemcpy(ix->S.p, S_host, cb_floats_local(*p) * 4, cudaMemcpyHostToDevice));
      }
      build_fbpq_tables(*ix, 0);
      build_hbpq_tables(*ix, 0);
      empty_lists(*ix, 0);
      BPQ_CUDA(cudaDeviceSynchronize());
    } catch (...) {
      delete ix;
      throw;
    }
    *out = ix;
  });
}

int bpq_train_load(bpq_index** out, const bpq_params* p, const float* learn_dev, int64_t n_learn,
                   const char* path, int device, void* stream) {
  return guard([&] {
    BPQ_CHECK(out, BPQ_EINVAL, "out is NULL");
    *out = nullptr;
    if (!learn_dev) {
      BPQ_CHECK(path, BPQ_EINVAL, "neither learn vectors nor a path were given");
      *out = load_file(path, device);
      return;
    }
    bpq_index* ix = new_index(p, device);
    try {
      DeviceGuard dg(device);
      cudaStream_t st = static_cast<cudaStream_t>(stream);
      train_codebooks(*ix, learn_dev, n_learn, st);
      build_fbpq_tables(*ix, st);
      build_hbpq_tables(*ix, st);
      empty_lists(*ix, st);
      BPQ_CUDA(cudaStreamSynchronize(st));
    } catch (...) {
      delete ix;
      throw;
    }
    *out = ix;
  });
}

int bpq_encode(const bpq_index* ix, const float* x_dev, int64_t n, int32_t* cell_out_dev, uint8_t* codes_out_dev,
               void* stream) {
  return guard([&] {
    BPQ_CHECK(ix, BPQ_EINVAL, "index is NULL");
    BPQ_CHECK(n >= 0, BPQ_EINVAL, "n < 0");
    if (n == 0) return;
    BPQ_CHECK(x_dev && cell_out_dev && codes_out_dev, BPQ_EINVAL, "NULL pointer");
    DeviceGuard dg(ix->device);
    launch_encode(*ix, x_dev, n, cell_out_dev, codes_out_dev, static_cast<cudaStream_t>(stream));
  });
}

int bpq_reconstruction_error(const bpq_index* ix, const float* x_dev, int64_t n, const int32_t* cells_dev,
                             const uint8_t* codes_dev, float* err_dev, void* stream) {
  return guard([&] {
    BPQ_CHECK(ix, BPQ_EINVAL, "index is NULL");
    BPQ_CHECK(n >= 0, BPQ_EINVAL, "n < 0");
    if (n == 0) return;
    BPQ_CHECK(n < ((int64_t)1 << 26) * 8, BPQ_EINVAL, "too many points in one call");
    BPQ_CHECK(x_dev && cells_dev && codes_dev && err_dev, BPQ_EINVAL, "NULL pointer");
    DeviceGuard dg(ix->device);
    launch_reconstruction_error(*ix, x_dev, n, cells_dev, codes_dev, err_dev, static_cast<cudaStream_t>(stream));
  });
}

int bpq_add(bpq_index* ix, const float* x_dev, int64_t n, const int32_t* ids_dev, void* stream) {
  return guard([&] {
    BPQ_CHECK(ix, BPQ_EINVAL, "index is NULL");
    BPQ_CHECK(n >= 0, BPQ_EINVAL, "n < 0");
    if (n == 0) return;
    BPQ_CHECK(x_dev, BPQ_EINVAL, "x is NULL");
    BPQ_CHECK(ix->n_points + ix->n_pending + n < ((int64_t)1 << 32) - 1, BPQ_EINVAL, "too many points");
    DeviceGuard dg(ix->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (ids_dev) BPQ_CHECK(ids_nonnegative(ids_dev, n, st), BPQ_EINVAL, "ids must be >= 0");
    const int M = ix->p.M;
    const int64_t need = ix->n_pending + n;
    if (need > ix->pend_cap) {
      const int64_t cap = std::max<int64_t>(need, 2 * ix->pend_cap);
      DevBuf c, k, d;
      c.alloc(cap * 4);
      k.alloc(cap * M);
      d.alloc(cap * 4);
      if (ix->n_pending) {
        BPQ_CUDA(cudaMemcpyAsync(c.p, ix->pend_cells.p, ix->n_pending * 4, cudaMemcpyDeviceToDevice, st));
        BPQ_CUDA(cudaMemcpyAsync(k.p, ix->pend_codes.p, ix->n_pending * M, cudaMemcpyDeviceToDevice, st));
        BPQ_CUDA(cudaMemcpyAsync(d.p, ix->pend_ids.p, ix->n_pending * 4, cudaMemcpyDeviceToDevice, st));
        BPQ_CUDA(cudaStreamSynchronize(st));
      }
      std::swap(c.p, ix->pend_cells.p);
      std::swap(c.bytes, ix->pend_cells.bytes);
      std::swap(k.p, ix->pend_codes.p);
      std::swap(k.bytes, ix->pend_codes.bytes);
      std::swap(d.p, ix->pend_ids.p);
      std::swap(d.bytes, ix->pend_ids.bytes);
      ix->pend_cap = cap;
    }
    launch_encode(*ix, x_dev, n, ix->pend_cells.as<int32_t>() + ix->n_pending,
                  ix->pend_codes.as<uint8_t>() + ix->n_pending * M, st);
    int32_t* idp = ix->pend_ids.as<int32_t>() + ix->n_pending;
    if (ids_dev)
      BPQ_CUDA(cudaMemcpyAsync(idp, ids_dev, n * 4, cudaMemcpyDeviceToDevice, st));
    else
      fill_sequential_ids(idp, n, ix->n_added, st);
    ix->n_pending += n;
    ix->n_added += n;
  });
}

int bpq_finalize(bpq_index* ix, void* stream) {
  return guard([&] {
    BPQ_CHECK(ix, BPQ_EINVAL, "index is NULL");
    DeviceGuard dg(ix->device);
    finalize_lists(*ix, static_cast<cudaStream_t>(stream));
    ix->goffsets.release();  // the shard's lists changed: its whole-index counts must be set again
    ix->g_points = ix->g_nonempty = 0;
  });
}

int bpq_set_global_counts(bpq_index* ix, const int64_t* counts_host) {
  return guard([&] {
    check_searchable(ix);
    DeviceGuard dg(ix->device);
    if (!counts_host) {
      ix->goffsets.release();
      ix->g_points = ix->g_nonempty = 0;
      return;
    }
    const int64_t nc = (int64_t)ix->p.T * ix->p.T;
    BPQ_CHECK(ix->offsets.p, BPQ_ESTATE, "the index has no lists: call bpq_finalize first");
    std::vector<uint32_t> loff((size_t)nc + 1);
    BPQ_CUDA(cudaMemcpy(loff.data(), ix->offsets.p, loff.size() * 4, cudaMemcpyDeviceToHost));
    std::vector<uint32_t> g((size_t)nc + 1);
    int64_t total = 0, nonempty = 0;
    uint32_t run = 0;
    for (int64_t c = 0; c < nc; ++c) {
      const int64_t v = counts_host[c];
      BPQ_CHECK(v >= 0 && v < ((int64_t)1 << 32), BPQ_EINVAL, "every count must be in [0, 2^32)");
      BPQ_CHECK(v >= (int64_t)(loff[c + 1] - loff[c]), BPQ_EINVAL,
                "a cell holds more points in this shard than in the whole index");
      BPQ_CHECK(total <= INT64_MAX - v, BPQ_EINVAL, "the counts overflow");
      g[c] = run;
      run += (uint32_t)v;  // modulo 2^32: differences of neighbours are the counts
      total += v;
      nonempty += v > 0;
    }
    g[nc] = run;
    DevBuf d;
    d.alloc(g.size() * 4);
    BPQ_CUDA(cudaMemcpy(d.p, g.data(), g.size() * 4, cudaMemcpyHostToDevice));
    std::swap(ix->goffsets.p, d.p);
    std::swap(ix->goffsets.bytes, d.bytes);
    ix->g_points = total;
    ix->g_nonempty = nonempty;
  });
}

int bpq_query_tables(const bpq_index* ix, const float* q, int64_t nq, float* d1, float* d2, float* lut,
                     void* stream) {
  return guard([&] {
    BPQ_CHECK(ix, BPQ_EINVAL, "index is NULL");
    BPQ_CHECK(nq >= 0, BPQ_EINVAL, "nq < 0");
    if (nq == 0) return;
    BPQ_CHECK(q && d1 && d2, BPQ_EINVAL, "NULL pointer");
    DeviceGuard dg(ix->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t step = 65535LL * 64;
    for (int64_t c0 = 0; c0 < nq; c0 += step) {
      const int64_t nc = std::min(step, nq - c0);
      const float* qcoarse = q + c0 * ix->p.D;
      const float* qres = qcoarse;
      DevBuf rc, rr;
      if (ix->opq) {  // rot0 q for the coarse tables, B rot0 q for the PQ table
        rc.alloc((size_t)nc * ix->p.D * 4);
        rr.alloc((size_t)nc * ix->p.D * 4);
        rotate_queries(*ix, qcoarse, nc, rc.as<float>(), rr.as<float>(), st);
        qcoarse = rc.as<float>();
        qres = rr.as<float>();
      }
      launch_query_tables(*ix, qcoarse, nc, d1 + c0 * ix->p.T, d2 + c0 * ix->p.T,
                          lut ? lut + c0 * ix->p.M * KSUB : nullptr, st, nullptr, qres);
      if (ix->opq) BPQ_CUDA(cudaStreamSynchronize(st));  // the rotated copies are released here
    }
  });
}

size_t bpq_search_workspace_size(const bpq_index* ix, int64_t nq, int64_t L_max, int32_t k, int32_t scorer) {
  if (!ix || nq < 0 || L_max < 1) return 0;
  // room for the work-queue form whenever the index may use it (its setting or a tuned class)
  int W = ix->scan_work_W;
  for (const auto& e : ix->tuned_W) W = std::max(W, e.second);
  return layout(*ix, std::max<int64_t>(nq, 1), L_max, scorer, true, k, 0.0, W).total;
}

int bpq_traverse(const bpq_index* ix, const float* q, int64_t nq, const int64_t* L_host, int64_t L_stride,
                 int32_t cap, bpq_cell* cells, int32_t* ncells, int64_t* npoints, void* ws, size_t ws_bytes,
                 void* stream) {
  return guard([&] {
    check_searchable(ix);
    BPQ_CHECK(nq >= 0, BPQ_EINVAL, "nq < 0");
    BPQ_CHECK(cells || nq == 0, BPQ_EINVAL, "cells is NULL");
    DeviceGuard dg(ix->device);
    run_queries(*ix, q, nq, L_host, L_stride, 1, BPQ_SCORER_FBPQ, nullptr, nullptr, cells, cap, ncells, npoints,
                ws, ws_bytes, static_cast<cudaStream_t>(stream));
  });
}

int bpq_search(const bpq_index* ix, const float* q, int64_t nq, const int64_t* L_host, int64_t L_stride,
               int32_t k, int32_t scorer, int32_t* ids, float* dists, void* ws, size_t ws_bytes, void* stream) {
  return guard([&] {
    check_searchable(ix);
    BPQ_CHECK(nq >= 0, BPQ_EINVAL, "nq < 0");
    DeviceGuard dg(ix->device);
    run_queries(*ix, q, nq, L_host, L_stride, k, scorer, ids, dists, nullptr, 0, nullptr, nullptr, ws, ws_bytes,
                static_cast<cudaStream_t>(stream));
  });
}

size_t bpq_search_shortlist_workspace_size(const bpq_index* ix, int64_t nq, int64_t L_max, int32_t shortlist) {
  if (!ix || nq < 0 || L_max < 1 || shortlist < 1 || shortlist > MAX_K) return 0;
  return shortlist_layout(*ix, std::max<int64_t>(nq, 1), L_max, shortlist).total;
}

int bpq_search_shortlist(const bpq_index* ix, const float* q, int64_t nq, const int64_t* L_host, int64_t L_stride,
                         int32_t k, int32_t shortlist, int32_t lut_precision, int32_t* ids, float* dists, void* ws,
                         size_t ws_bytes, void* stream) {
  return guard([&] {
    check_searchable(ix);
    BPQ_CHECK(nq >= 0, BPQ_EINVAL, "nq < 0");
    BPQ_CHECK(lut_precision == BPQ_LUT_I8 || lut_precision == BPQ_LUT_F16, BPQ_EINVAL,
              "lut_precision must be BPQ_LUT_I8 or BPQ_LUT_F16");
    DeviceGuard dg(ix->device);
    run_shortlist(*ix, q, nq, L_host, L_stride, k, shortlist, lut_precision == BPQ_LUT_F16, ids, dists, ws, ws_bytes,
                  static_cast<cudaStream_t>(stream));
  });
}

int bpq_scan(const bpq_index* ix, const float* q, int64_t nq, const float* lut, const bpq_cell* cells,
             const int32_t* ncells, int32_t cap, int32_t k, int32_t scorer, int32_t* ids, float* dists,
             int32_t* counter, void* stream) {
  return guard([&] {
    check_searchable(ix);
    BPQ_CHECK(nq >= 0, BPQ_EINVAL, "nq < 0");
    if (nq == 0) return;
    BPQ_CHECK(k >= 1 && k <= MAX_K, BPQ_EINVAL, "k must be in [1, 1024]");
    check_scorer(*ix, scorer);
    BPQ_CHECK(cells && ncells && ids && dists && counter && cap >= 1, BPQ_EINVAL, "bad argument");
    BPQ_CHECK(!uses_lut(scorer) || lut, BPQ_EINVAL, "FBPQ needs the query tables");
    BPQ_CHECK(uses_lut(scorer) || q, BPQ_EINVAL, "reconstruction needs the queries");
    DeviceGuard dg(ix->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DevBuf rr;
    if (ix->opq && !uses_lut(scorer)) {  // the reconstruction scorer works in the residual space
      rr.alloc((size_t)nq * ix->p.D * 4);
      rotate_for_index(*ix, q, nq, nullptr, rr.as<float>(), st);
      q = rr.as<float>();
    }
    launch_scan(scan_args(*ix, q, nq, lut, cells, ncells, cap, k, ids, dists, counter), scorer, st);
    if (rr.p) BPQ_CUDA(cudaStreamSynchronize(st));
  });
}

int bpq_search_status(const bpq_index* ix, void* ws, void* stream) {
  return guard([&] {
    BPQ_CHECK(ix && ws, BPQ_EINVAL, "NULL pointer");
    DeviceGuard dg(ix->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int32_t s = 0;
    BPQ_CUDA(cudaMemcpyAsync(&s, ws, 4, cudaMemcpyDeviceToHost, st));  // status is the first word
    BPQ_CUDA(cudaStreamSynchronize(st));
    BPQ_CHECK((s & STATUS_TIMEOUT) == 0, BPQ_ETIMEOUT,
              "a bounded wait on a tensor-core table tile gave up (the tile was recomputed on the CUDA cores)");
    BPQ_CHECK((s & STATUS_OVERFLOW) == 0, BPQ_ECAPACITY, "a query overflowed a fixed-size buffer (band or cell list)");
  });
}

int bpq_search_host(bpq_index* ix, const float* q_host, int64_t nq, const int64_t* L_host, int64_t L_stride,
                    int32_t k, int32_t scorer, int32_t* ids_host, float* dists_host, void* stream) {
  return guard([&] {
    check_searchable(ix);
    BPQ_CHECK(nq >= 0 && q_host && ids_host && dists_host, BPQ_EINVAL, "bad argument");
    BPQ_CHECK(k >= 1 && k <= MAX_K, BPQ_EINVAL, "k must be in [1, 1024]");
    if (nq == 0) return;
    DeviceGuard dg(ix->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t L_max = read_L(L_host, L_stride, nq, nullptr);
    const size_t want = std::min<size_t>(layout(*ix, nq, L_max, scorer, true, k).total, (size_t)4 << 30);
    const size_t one = layout(*ix, 1, L_max, scorer, true, k).total;
    ix->host_ws.ensure(std::max(want, one));
    ix->host_q.ensure((size_t)nq * ix->p.D * 4);
    ix->host_ids.ensure((size_t)nq * k * 4);
    ix->host_dists.ensure((size_t)nq * k * 4);
    BPQ_CUDA(cudaMemcpyAsync(ix->host_q.p, q_host, (size_t)nq * ix->p.D * 4, cudaMemcpyHostToDevice, st));
    run_queries(*ix, ix->host_q.as<float>(), nq, L_host, L_stride, k, scorer, ix->host_ids.as<int32_t>(),
                ix->host_dists.as<float>(), nullptr, 0, nullptr, nullptr, ix->host_ws.p, ix->host_ws.bytes, st);
    BPQ_CUDA(cudaMemcpyAsync(ids_host, ix->host_ids.p, (size_t)nq * k * 4, cudaMemcpyDeviceToHost, st));
    BPQ_CUDA(cudaMemcpyAsync(dists_host, ix->host_dists.p, (size_t)nq * k * 4, cudaMemcpyDeviceToHost, st));
    BPQ_CUDA(cudaStreamSynchronize(st));
  });
}

int bpq_set_hbpq_table_budget(bpq_index* ix, double slots_per_query) {
  return guard([&] {
    BPQ_CHECK(ix, BPQ_EINVAL, "index is NULL");
    BPQ_CHECK(std::isfinite(slots_per_query) && slots_per_query >= 0.0, BPQ_EINVAL,
              "slots per query must be finite and >= 0");
    ix->hb_slots_per_query = slots_per_query;
  });
}

int bpq_autotune(bpq_index* ix, const float* q, int64_t nq, const int64_t* L_host, int64_t L_stride, int32_t k,
                 int32_t scorer, int32_t* ids, float* dists, void* stream, int32_t* chosen_out) {
  return guard([&] {
    check_searchable(ix);
    BPQ_CHECK(nq >= 1 && q && ids && dists, BPQ_EINVAL, "bad argument");
    BPQ_CHECK(k >= 1 && k <= MAX_K, BPQ_EINVAL, "k must be in [1, 1024]");
    check_scorer(*ix, scorer);
    DeviceGuard dg(ix->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<int32_t> Lq;
    const int64_t L_max = read_L(L_host, L_stride, nq, &Lq);
    double Lm = (double)L_max;
    if (L_stride) {
      Lm = 0.0;
      for (int32_t v : Lq) Lm += v;
      Lm /= (double)nq;
    }
    const uint64_t key = tune_key(scorer, k, nq, Lm);
    ix->tuned_W.erase(key);
    const int32_t cand[] = {0, 4096, 8192, 16384, 32768};
    // one workspace that holds the batch in one chunk with either schedule
    DevBuf wsb;
    wsb.alloc(layout(*ix, nq, L_max, scorer, true, k, 0.0, work_queue_used(1, scorer, k) ? 1 : 0).total);
    void* ws = wsb.p;
    const size_t ws_bytes = wsb.bytes;
    cudaEvent_t e0, e1;
    BPQ_CUDA(cudaEventCreate(&e0));
    BPQ_CUDA(cudaEventCreate(&e1));
    int32_t best = 0;
    float best_ms = 0.f;
    const int32_t saved = ix->scan_work_W;
    try {
      for (int32_t W : cand) {
        if (W > 0 && !work_queue_used(W, scorer, k)) continue;
        if (layout(*ix, nq, L_max, scorer, true, k, 0.0, W).total > ws_bytes) continue;  // must run in one chunk
        ix->scan_work_W = W;
        std::vector<float> t;
        for (int r = 0; r < 4; ++r) {  // the first run of a configuration is a warm-up
          BPQ_CUDA(cudaEventRecord(e0, st));
          run_queries(*ix, q, nq, L_host, L_stride, k, scorer, ids, dists, nullptr, 0, nullptr, nullptr, ws, ws_bytes,
                      st);
          BPQ_CUDA(cudaEventRecord(e1, st));
          BPQ_CUDA(cudaEventSynchronize(e1));
          float ms = 0.f;
          BPQ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
          if (r > 0) t.push_back(ms);
        }
        std::sort(t.begin(), t.end());
        const float med = t[t.size() / 2];
        if (W == 0 || med < best_ms) {
          best = W;
          best_ms = med;
        }
      }
    } catch (...) {
      ix->scan_work_W = saved;
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      throw;
    }
    ix->scan_work_W = saved;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ix->tuned_W[key] = best;
    if (chosen_out) *chosen_out = best;
  });
}

int bpq_set_rotations(bpq_index* ix, const double* R0, const double* R1, const double* R2) {
  return guard([&] {
    BPQ_CHECK(ix && R0 && R1 && R2, BPQ_EINVAL, "NULL pointer");
    BPQ_CHECK(ix->p.opq, BPQ_EINVAL, "the index was made without OPQ (params.opq = 0)");
    BPQ_CHECK(ix->n_points == 0 && ix->n_pending == 0, BPQ_ESTATE, "rotations must be set before points are added");
    DeviceGuard dg(ix->device);
    set_opq_rotations(*ix, R0, R1, R2, 0);
    build_fbpq_tables(*ix, 0);
    BPQ_CUDA(cudaDeviceSynchronize());
  });
}

int bpq_get_rotations(const bpq_index* ix, double* R0, double* R1, double* R2) {
  return guard([&] {
    BPQ_CHECK(ix && R0 && R1 && R2, BPQ_EINVAL, "NULL pointer");
    BPQ_CHECK(ix->opq, BPQ_ESTATE, "the index has no rotations");
    std::copy(ix->h_rot0.begin(), ix->h_rot0.end(), R0);
    std::copy(ix->h_rot1.begin(), ix->h_rot1.end(), R1);
    std::copy(ix->h_rot2.begin(), ix->h_rot2.end(), R2);
  });
}

int bpq_set_scan_work_size(bpq_index* ix, int32_t candidates_per_item) {
  return guard([&] {
    BPQ_CHECK(ix, BPQ_EINVAL, "index is NULL");
    BPQ_CHECK(candidates_per_item >= 0, BPQ_EINVAL, "candidates per item must be >= 0");
    ix->scan_work_W = candidates_per_item;
  });
}

int bpq_get_info(const bpq_index* ix, bpq_info* out) {
  return guard([&] {
    BPQ_CHECK(ix && out, BPQ_EINVAL, "NULL pointer");
    out->n_points = ix->n_points;
    out->n_pending = ix->n_pending;
    out->n_nonempty = ix->n_nonempty;
    out->max_cell = ix->max_cell;
    out->device_bytes = (int64_t)(ix->C1.bytes + ix->C2.bytes + ix->R.bytes + ix->Q.bytes + ix->S.bytes +
                                  ix->X1.bytes + ix->X2.bytes + ix->offsets.bytes + ix->codes.bytes +
                                  ix->ids.bytes + ix->cross.bytes + ix->pend_cells.bytes + ix->pend_codes.bytes +
                                  ix->pend_ids.bytes + ix->C1b.bytes + ix->C2b.bytes + ix->Rb.bytes + ix->n1.bytes +
                                  ix->n2.bytes + ix->nR.bytes + ix->Qb.bytes + ix->Sb.bytes + ix->E1.bytes +
                                  ix->E2.bytes + ix->rot0t.bytes + ix->rotBt.bytes + ix->rotPt.bytes +
                                  ix->C1r.bytes + ix->C2r.bytes + ix->rot0tf.bytes + ix->rotPtf.bytes);
    out->params = ix->p;
  });
}

int bpq_get_arrays(const bpq_index* ix, bpq_arrays* out) {
  return guard([&] {
    BPQ_CHECK(ix && out, BPQ_EINVAL, "NULL pointer");
    out->C1 = ix->C1.as<float>();
    out->C2 = ix->C2.as<float>();
    out->R = ix->R.as<float>();
    out->Q = ix->Q.as<float>();
    out->S = ix->S.as<float>();
    out->X1 = ix->X1.as<float>();
    out->X2 = ix->X2.as<float>();
    out->offsets = ix->offsets.as<uint32_t>();
    out->codes = ix->codes.as<uint8_t>();
    out->ids = ix->ids.as<int32_t>();
    out->cross = ix->cross.as<float>();
  });
}

int bpq_save(const bpq_index* ix, const char* path) {
  return guard([&] {
    check_searchable(ix);
    BPQ_CHECK(path, BPQ_EINVAL, "path is NULL");
    DeviceGuard dg(ix->device);
    BPQ_CUDA(cudaDeviceSynchronize());
    File fh;
    fh.f = fopen(path, "wb");
    BPQ_CHECK(fh.f, BPQ_EIO, std::string("cannot open ") + path + " for writing");
    const uint32_t version = 2;
    const int64_t n = ix->n_points;
    BPQ_CHECK(fwrite(MAGIC, 8, 1, fh.f) == 1 && fwrite(&version, 4, 1, fh.f) == 1 &&
                  fwrite(&ix->p, sizeof(ix->p), 1, fh.f) == 1 && fwrite(&n, 8, 1, fh.f) == 1,
              BPQ_EIO, "write failed");
    write_section(fh.f, ix->C1.p, ix->C1.bytes);
    write_section(fh.f, ix->C2.p, ix->C2.bytes);
    write_section(fh.f, ix->R.p, ix->R.bytes);
    if (ix->p.variant == BPQ_VARIANT_LOCAL) {
      write_section(fh.f, ix->Q.p, ix->Q.bytes);
      write_section(fh.f, ix->S.p, ix->S.bytes);
    }
    if (ix->p.opq) {
      BPQ_CHECK(ix->opq, BPQ_ESTATE, "an OPQ index needs its rotations (bpq_set_rotations) before it is saved");
      write_host_section(fh.f, ix->h_rot0.data(), ix->h_rot0.size() * 8);
      write_host_section(fh.f, ix->h_rot1.data(), ix->h_rot1.size() * 8);
      write_host_section(fh.f, ix->h_rot2.data(), ix->h_rot2.size() * 8);
    }
    write_section(fh.f, ix->offsets.p, ((size_t)ix->p.T * ix->p.T + 1) * 4);
    write_section(fh.f, ix->codes.p, (size_t)n * ix->p.M);
    write_section(fh.f, ix->ids.p, (size_t)n * 4);
    BPQ_CHECK(fflush(fh.f) == 0, BPQ_EIO, "write failed");
  });
}

void bpq_free(bpq_index* ix) {
  if (!ix) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(ix->device);
  delete ix;
  if (prev >= 0) cudaSetDevice(prev);
}

}  // extern "C"
