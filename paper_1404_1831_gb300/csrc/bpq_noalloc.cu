// bpq_search_noalloc: bpq_search for callers that cannot allocate device memory.
//
// Some programs that embed this library own all of the GPU's memory through
// their own pool or budget, and others run latency-critical loops in which a
// cudaMalloc / cudaFree (which may synchronize the whole device) is not
// acceptable.  Such callers cannot provide the workspace bpq_search wants.  This
// entry point runs the same kernels (query tables, traversal, scan and top-k)
// but keeps their scratch data in one fixed array of device memory that is part
// of the library itself, so the call allocates nothing.
//
// The array (NOALLOC_SCRATCH_BYTES) is reserved on every GPU that loads the
// library, for as long as the process lives.  All calls share it and it keeps
// the previous call's contents, so two calls whose work overlaps on the GPU (on
// different streams, or from different threads without ordering) race on it.
#include <mutex>

#include "bpq_internal.cuh"

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = BPQ_NOALLOC_SCRATCH_BYTES;
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[MAX_DEVICES] = {};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device address of the scratch array on the current device.  Host code cannot
// use the array's name as an address, so it is looked up once per device.  The
// address belongs to the device's primary context (the one the CUDA runtime
// uses); it is not valid in another context of the same device, nor after
// cudaDeviceReset, and this entry point does not support either.
void* scratch_address(int device) {
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      throw bpq::Error(BPQ_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_noalloc_ptr[device] = p;
  }
  return g_noalloc_ptr[device];
}

struct Offsets {
  size_t status, counter, L, d1, d2, lut, cells, ncells, npoints, total;
  int64_t cap;
};

Offsets plan(const bpq_index& ix, int64_t nq, int64_t L_max, int scorer) {
  Offsets o{};
  size_t at = 0;
  auto take = [&](size_t bytes) {
    size_t here = at;
    at = align256(at + bytes);
    return here;
  };
  o.cap = std::max<int64_t>(1, std::min<int64_t>(L_max, std::max<int64_t>(ix.n_nonempty, 1)));
  o.status = take(4);
  o.counter = take(4);
  o.L = take((size_t)nq * 4);
  o.d1 = take((size_t)nq * ix.p.T * 4);
  o.d2 = take((size_t)nq * ix.p.T * 4);
  const bool lut = scorer == BPQ_SCORER_FBPQ || scorer == BPQ_SCORER_FBPQ_TABLES;
  o.lut = take(lut ? (size_t)nq * ix.p.M * bpq::KSUB * 4 : 0);
  o.cells = take((size_t)nq * o.cap * sizeof(bpq_cell));
  o.ncells = take((size_t)nq * 4);
  o.npoints = take((size_t)nq * 8);
  o.total = at;
  return o;
}

// Failures are reported by return code only: filling in the message that
// bpq_last_error() returns could allocate host memory.
int fail(int code, const char*) { return code; }

}  // namespace

extern "C" int bpq_search_noalloc(const bpq_index* ix, const float* queries_dev, int64_t nq, const int64_t* L_host,
                                  int64_t L_stride, int32_t k, int32_t scorer, int32_t* ids_dev, float* dists_dev,
                                  int32_t* status_dev, void* stream) {
  if (!ix) return fail(BPQ_EINVAL, "index is NULL");
  if (ix->n_pending != 0) return fail(BPQ_ESTATE, "points were added since the last bpq_finalize");
  if (nq < 0) return fail(BPQ_EINVAL, "nq < 0");
  if (k < 1 || k > bpq::MAX_K) return fail(BPQ_EINVAL, "k must be in [1, 1024]");
  if (scorer < BPQ_SCORER_FBPQ || scorer > BPQ_SCORER_FBPQ_TABLES) return fail(BPQ_EINVAL, "bad scorer");
  if ((scorer == BPQ_SCORER_HBPQ) != (ix->p.variant == BPQ_VARIANT_LOCAL))
    return fail(BPQ_EINVAL, "scorer does not match the codebook variant");
  if (ix->opq) return fail(BPQ_EINVAL, "OPQ indexes need rotated query buffers: use bpq_search");
  if (ix->goffsets.p) return fail(BPQ_EINVAL, "point shards (whole-index counts set) are searched by bpq_search");
  if (!L_host || (L_stride != 0 && L_stride != 1)) return fail(BPQ_EINVAL, "L must be given with stride 0 or 1");
  int64_t L_max = 0;
  for (int64_t i = 0; i < (L_stride ? nq : 1); ++i) {
    if (L_host[i] < 1 || L_host[i] >= ((int64_t)1 << 31)) return fail(BPQ_EINVAL, "every L must be in [1, 2^31)");
    L_max = std::max(L_max, L_host[i]);
  }
  if (nq == 0) return BPQ_OK;
  if (!queries_dev || !ids_dev || !dists_dev) return fail(BPQ_EINVAL, "NULL pointer");
  if (ix->device < 0 || ix->device >= MAX_DEVICES) return fail(BPQ_EINVAL, "device ordinal out of range");
  const Offsets o = plan(*ix, nq, L_max, scorer);
  if (o.total > NOALLOC_SCRATCH_BYTES)
    return fail(BPQ_ECAPACITY, "the batch needs more scratch than the built-in array holds: split it");
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) return fail(BPQ_ECUDA, "cudaGetDevice failed");
  if (prev != ix->device && cudaSetDevice(ix->device) != cudaSuccess) return fail(BPQ_ECUDA, "cudaSetDevice failed");
  int rc = BPQ_OK;
  try {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char* w = static_cast<char*>(scratch_address(ix->device));
    BPQ_CUDA(cudaMemsetAsync(w + o.status, 0, 4, st));
    float* d1 = reinterpret_cast<float*>(w + o.d1);
    float* d2 = reinterpret_cast<float*>(w + o.d2);
    const bool uses_lut = scorer == BPQ_SCORER_FBPQ || scorer == BPQ_SCORER_FBPQ_TABLES;
    float* lut = uses_lut ? reinterpret_cast<float*>(w + o.lut) : nullptr;
    bpq::launch_query_tables(*ix, queries_dev, nq, d1, d2, lut, st);
    bpq::TraverseArgs ta{};
    ta.d1 = d1;
    ta.d2 = d2;
    ta.offsets = ix->offsets.as<uint32_t>();
    if (L_stride) {
      // per-query budgets go up through a small stack buffer: a copy from pageable
      // memory returns once the source has been staged, so the buffer is reused
      int32_t buf[1024];
      for (int64_t c0 = 0; c0 < nq; c0 += 1024) {
        const int64_t n = std::min<int64_t>(1024, nq - c0);
        for (int64_t i = 0; i < n; ++i) buf[i] = (int32_t)L_host[c0 + i];
        BPQ_CUDA(cudaMemcpyAsync(w + o.L + c0 * 4, buf, n * 4, cudaMemcpyHostToDevice, st));
      }
      ta.L = reinterpret_cast<const int32_t*>(w + o.L);
    } else {
      ta.L = nullptr;
      ta.L_scalar = (int32_t)L_host[0];
    }
    ta.T = ix->p.T;
    ta.cap = (int32_t)o.cap;
    ta.rho = (float)((double)ix->n_points / (double)std::max<int64_t>(1, ix->n_nonempty));
    ta.cells = reinterpret_cast<bpq_cell*>(w + o.cells);
    ta.ncells = reinterpret_cast<int32_t*>(w + o.ncells);
    ta.npoints = reinterpret_cast<int64_t*>(w + o.npoints);
    ta.status = reinterpret_cast<int32_t*>(w + o.status);
    ta.nq = nq;
    bpq::launch_traverse(ta, st);
    bpq::ScanArgs sa{};
    sa.cells = ta.cells;
    sa.ncells = ta.ncells;
    sa.cap = ta.cap;
    sa.nq = nq;
    sa.T = ix->p.T;
    sa.M = ix->p.M;
    sa.D = ix->p.D;
    sa.k = k;
    sa.lut = lut;
    sa.X1 = ix->X1.as<float>();
    sa.X2 = ix->X2.as<float>();
    sa.cross = ix->cross.as<float>();
    sa.queries = queries_dev;
    sa.C1 = ix->C1.as<float>();
    sa.C2 = ix->C2.as<float>();
    sa.R = ix->R.as<float>();
    sa.Q = ix->Q.as<float>();
    sa.S = ix->S.as<float>();
    sa.codes = ix->codes.as<uint8_t>();
    sa.ids = ix->ids.as<int32_t>();
    sa.out_ids = ids_dev;
    sa.out_dists = dists_dev;
    sa.qcounter = reinterpret_cast<int32_t*>(w + o.counter);
    sa.sm_count = ix->sm_count;
    bpq::launch_scan(sa, scorer, st);
    if (status_dev) BPQ_CUDA(cudaMemcpyAsync(status_dev, w + o.status, 4, cudaMemcpyDeviceToDevice, st));
  } catch (const bpq::Error& e) {
    rc = e.code;
  } catch (...) {  // nothing else may cross the C boundary (e.g. a failed mutex lock)
    rc = BPQ_ECUDA;
  }
  if (prev >= 0 && prev != ix->device) cudaSetDevice(prev);
  return rc;
}
