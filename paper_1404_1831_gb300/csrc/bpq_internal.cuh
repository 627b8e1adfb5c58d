// Internal declarations shared by the translation units of libbpq.
// Device helpers, launch wrappers and the index object.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <stdexcept>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/bpq.h"

namespace bpq {

constexpr int KSUB = 256;
constexpr int MAX_T = 4096;
constexpr int MAX_K = 1024;

// ---------------------------------------------------------------------------
// Errors: host code throws Error; the C ABI layer turns it into a return code.
// ---------------------------------------------------------------------------
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define BPQ_CUDA(call)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      throw ::bpq::Error(e_ == cudaErrorMemoryAllocation ? BPQ_ENOMEM : BPQ_ECUDA,           \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                \
  } while (0)

#define BPQ_CHECK(cond, code, msg)                                                           \
  do {                                                                                       \
    if (!(cond)) throw ::bpq::Error((code), (msg));                                          \
  } while (0)

inline void check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw Error(BPQ_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// ---------------------------------------------------------------------------
// Order-preserving map between float and uint32 (for sort keys): a < b as floats
// iff ord(a) < ord(b) as unsigned, for all non-NaN values.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t f2ord(float f) {
  uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t o) {
  uint32_t b = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
  return __uint_as_float(b);
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Block-wide bitonic sort (ascending) of n = power of two 64-bit keys in shared
// memory; all threads of the block must call it.
__device__ __forceinline__ void block_bitonic_sort(uint64_t* a, int n) {
  for (int size = 2; size <= n; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      __syncthreads();
      for (int t = threadIdx.x; t < (n >> 1); t += blockDim.x) {
        int lo = 2 * t - (t & (stride - 1));
        int hi = lo + stride;
        bool up = ((lo & size) == 0);
        uint64_t x = a[lo], y = a[hi];
        if ((x > y) == up) {
          a[lo] = y;
          a[hi] = x;
        }
      }
    }
  }
  __syncthreads();
}

// Warp-wide bitonic sort (ascending) of n = power of two keys in shared memory
// (n >= 64); only the calling warp touches `a`.
__device__ __forceinline__ void warp_bitonic_sort(uint64_t* a, int n) {
  const int lane = threadIdx.x & 31;
  for (int size = 2; size <= n; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      __syncwarp();
      for (int t = lane; t < (n >> 1); t += 32) {
        int lo = 2 * t - (t & (stride - 1));
        int hi = lo + stride;
        bool up = ((lo & size) == 0);
        uint64_t x = a[lo], y = a[hi];
        if ((x > y) == up) {
          a[lo] = y;
          a[hi] = x;
        }
      }
    }
  }
  __syncwarp();
}

// Histogram increment aggregated over the lanes of a warp that hit the same bin
// (one shared-memory atomic per distinct bin instead of one per lane).  Every
// lane of the warp must call it; lanes with valid == false add nothing.
__device__ __forceinline__ void warp_hist_add(uint32_t* hist, uint32_t bin, bool valid) {
  const uint32_t peers = __match_any_sync(0xffffffffu, valid ? bin : 0xffffffffu);
  if (valid && (peers & lanemask_lt()) == 0) atomicAdd(&hist[bin], (uint32_t)__popc(peers));
}

// Weighted version: adds w (< 2^32) of every lane to its bin, 64-bit totals.
__device__ __forceinline__ void warp_hist_add_w(unsigned long long* hist, uint32_t bin, uint32_t w, bool valid) {
  const uint32_t peers = __match_any_sync(0xffffffffu, valid ? bin : 0xffffffffu);
  const uint32_t ww = valid ? w : 0u;
  const uint32_t lo = __reduce_add_sync(peers, ww & 0xffffu);
  const uint32_t hi = __reduce_add_sync(peers, ww >> 16);
  if (valid && (peers & lanemask_lt()) == 0) atomicAdd(&hist[bin], (unsigned long long)lo + ((unsigned long long)hi << 16));
}

// Sum over the warp: one redux.sync for 32-bit integers, shuffles otherwise.
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  if constexpr (std::is_same<T, int>::value || std::is_same<T, unsigned>::value) {
    return __reduce_add_sync(0xffffffffu, v);
  } else {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  }
}

// ---------------------------------------------------------------------------
// Tensor-core operand layout (tcgen05): operands K-major in shared memory without
// swizzle, as 8-row x 16-byte core matrices; core (row group g, column group c) at
// byte 128 (g * KB + c), KB = K / 8 column groups.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t core_off(int r, int k, int KB) {
  return (uint32_t)((((r >> 3) * KB + (k >> 3)) * 128) + (r & 7) * 16 + (k & 7) * 2);
}

// Shared-memory matrix descriptor: start, leading (K) and stride (row-group)
// byte offsets, the fixed 0b001 at bits 46-48, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Bounded wait on phase `parity` of an mbarrier: 1 when the phase completed,
// 0 when `iters` polls went by first.
__device__ __forceinline__ uint32_t mbar_wait_bounded(uint64_t* mbar, uint32_t parity, int iters) {
  uint32_t ready = 0;
  for (int it = 0; it < iters && !ready; ++it)
    asm volatile("{\n.reg .pred P;\nmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\nselp.u32 %0, 1, 0, P;\n}\n"
                 : "=r"(ready) : "r"(smem_u32(mbar)), "r"(parity));
  return ready;
}

// ---------------------------------------------------------------------------
// Index object (host side).
// ---------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  void alloc(size_t b) {
    release();
    if (b == 0) return;
    cudaError_t e = cudaMalloc(&p, b);
    if (e != cudaSuccess) {
      p = nullptr;
      throw Error(BPQ_ENOMEM, std::string("cudaMalloc(") + std::to_string(b) + "): " + cudaGetErrorString(e));
    }
    bytes = b;
  }
  void ensure(size_t b) {
    if (b > bytes) alloc(b);
  }
  template <typename T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

}  // namespace bpq

struct bpq_index {
  bpq_params p{};
  int device = 0;
  int sm_count = 0;
  int h = 0, s = 0, m2 = 0;  // D/2, D/M, M/2
  bpq::DevBuf C1, C2, R, Q, S, X1, X2;
  // pending points (encoded, not yet in the lists)
  bpq::DevBuf pend_cells, pend_codes, pend_ids;
  int64_t n_pending = 0, pend_cap = 0;
  int64_t n_added = 0;  // for default ids
  // finalized lists
  bpq::DevBuf offsets, codes, ids;
  bpq::DevBuf cross;  // per point 2<c_ij, r> (global variant)
  // tensor-core operands of the query tables: BF16 copies of C1, C2 (T x kh) and
  // R (M x 256 x ks), K padded with zeros to kh = 16 ceil(D/32), ks = 16 ceil(D/M/16),
  // FP32 squared norms of their rows, and whether every copy is exact
  bpq::DevBuf C1b, C2b, Rb, n1, n2, nR;
  int kh = 0, ks = 0;
  bool coarse_bf16_exact = false, R_bf16_exact = false;
  // second BF16 planes v - bf16(v) (codewords of magnitude up to 2^16 are exact as
  // the sum of two planes, e.g. integer codebooks in OPQ-rotated spaces)
  bpq::DevBuf C1b2, C2b2, Rb2;
  bool coarse_bf16x2_exact = false, R_bf16x2_exact = false;
  // HBPQ table form (local variant): BF16 copies of the local codebooks Q, S
  // (T x M/2 x 256 x ks, K padded with zeros) and the query-independent part of
  // the per-half-cell tables, E1[i][k][t] = ||Q^i_k[t]||^2 + 2<c^1_i|k, Q^i_k[t]>
  // and E2 likewise with S^j, c^2_j (T x M/2 x 256 FP32 each)
  bpq::DevBuf Qb, Sb, E1, E2;
  bool local_bf16_exact = false;
  double hb_slots_per_query = 0.0;  // 0: automatic (bpq_set_hbpq_table_budget)
  // OPQ: rotations (host FP64 copies; device FP64 transposed blocks for rotate_rows:
  // rot0, B = blockdiag(rot1, rot2), P = B rot0) and the rotated coarse centroids B c
  bool opq = false;
  std::vector<double> h_rot0, h_rot1, h_rot2;
  bpq::DevBuf rot0t, rotBt, rotPt, C1r, C2r;
  bpq::DevBuf rot0tf, rotPtf;  // FP32 transposed rot0 and P for the query rotation
  int32_t scan_work_W = 0;          // candidates per work item of the scan; 0: one CTA per query
  // work-item sizes chosen by bpq_autotune, per batch class (scorer, k <= 32, log2 nq,
  // log2 mean L); a class found here overrides scan_work_W
  std::map<uint64_t, int32_t> tuned_W;
  int64_t n_points = 0, n_nonempty = 0, max_cell = 0;
  // point shard (bpq_set_global_counts): the whole index's per-cell counts as a
  // prefix modulo 2^32 (differences give the counts), its points and non-empty
  // cells; the traversal runs on these, the scan on the shard's own lists
  bpq::DevBuf goffsets;
  int64_t g_points = 0, g_nonempty = 0;
  // workspace owned by bpq_search_host
  bpq::DevBuf host_ws, host_q, host_ids, host_dists;
};

namespace bpq {

// ---------------------------------------------------------------------------
// Launch wrappers (defined in the .cu files).
// ---------------------------------------------------------------------------

// Query tables (bpq_tables.cu).
// status: workspace status word (may be NULL); a tensor-core tile whose bounded
// wait gave up sets STATUS_TIMEOUT there and is recomputed on the CUDA cores.
// q_lut: the queries for the PQ table when they differ from q (OPQ: q~ = B rot0 q, q = rot0 q)
void launch_query_tables(const bpq_index& ix, const float* q, int64_t nq, float* d1, float* d2,
                         float* lut, cudaStream_t st, int32_t* status = nullptr, const float* q_lut = nullptr);
void build_fbpq_tables(bpq_index& ix, cudaStream_t st);

// Bits of the workspace status word.
constexpr int32_t STATUS_OVERFLOW = 1;  // a fixed-size buffer (traversal band) overflowed
constexpr int32_t STATUS_TIMEOUT = 2;   // a bounded device wait gave up

// HBPQ table form (bpq_hbpq.cu).
void build_hbpq_tables(bpq_index& ix, cudaStream_t st);
bool hbpq_tensor_shape(const bpq_index& ix);  // the tensor-core table kernel covers (D, M)
struct HbpqArgs {
  const bpq_cell* cells;
  const int32_t* ncells;
  int32_t cap;
  int64_t nq;
  int32_t T, M, D;
  const float* queries;   // nq x D
  // per query: first table slot (-1: did not fit, scored by the fallback), number of
  // distinct rows, and the row / column bitmaps (2 x ceil(T/32) words)
  int32_t* qbase;
  int32_t* qrows;
  uint32_t* qbits;
  // per half and half-cell: bitmap of the visiting queries (2 x T x ceil(nq/32) words, zeroed)
  uint32_t* hmap;
  unsigned long long* slot_counter;  // table slots taken (zeroed)
  int32_t* fb_count;      // queries handed to the fallback (zeroed)
  int32_t* fallback;      // nq: queries whose tables did not fit
  int64_t slot_cap;       // table slots in `tables`
  float* tables;          // slot_cap x M/2 x 256
  int32_t* status;
};
void launch_hbpq_pairs(const HbpqArgs& h, cudaStream_t st);
void launch_hbpq_tables(const bpq_index& ix, const HbpqArgs& h, cudaStream_t st);

// Traversal (bpq_traverse.cu).
struct TraverseArgs {
  const float* d1;
  const float* d2;
  const uint32_t* offsets;
  const int32_t* L;  // per query, or nullptr -> L_scalar
  int32_t L_scalar;
  int32_t T;
  int32_t cap;       // output cells per query
  float rho;         // mean points per non-empty cell (sizes the first band)
  int32_t ordered;   // 1: emit each band sorted by (key, cell id); 0: any order
  bpq_cell* cells;   // nq x cap
  int32_t* ncells;
  int64_t* npoints;
  int32_t* status;   // single word, set to 1 on overflow
  int64_t nq;
  // optional (T <= the warp path's limit): the warp kernel lists the queries it
  // hands over in fb_list[0 .. *fb_n) (*fb_n zeroed by the caller) and writes
  // handed[q] = 1 for them, 0 for the others; the CTA pass then takes the list
  int32_t* fb_list;
  int32_t* fb_n;
  uint8_t* handed;
};
void launch_traverse(const TraverseArgs& a, cudaStream_t st);
// The two passes of launch_traverse, for callers that overlap the second with
// other work: the warp pass returns false when the CTA pass already ran for
// every query (T above the warp path's limit) and there is no second pass.
bool launch_traverse_warp(const TraverseArgs& a, cudaStream_t st);
void launch_traverse_marked(const TraverseArgs& a, cudaStream_t st);
// Point shard: after a traversal on the whole index's counts, each visited cell
// gets the shard's list range (loff) and the cells the shard holds no point of
// are dropped, in order.
void launch_localize_cells(const TraverseArgs& a, const uint32_t* loff, cudaStream_t st);
int traverse_band_capacity();

// Scans (bpq_scan.cu).
struct ScanArgs {
  const bpq_cell* cells;
  const int32_t* ncells;
  int32_t cap;
  int64_t nq;
  int32_t T, M, D, k;
  const float* lut;      // nq x M x 256 (FBPQ)
  const float* X1;       // T x M/2 x 256
  const float* X2;
  const float* cross;    // per point 2<c_ij, r> (FBPQ)
  const float* queries;  // nq x D (recon / hbpq)
  const float* C1;
  const float* C2;
  const float* R;        // M x 256 x D/M
  const float* Q;        // T x M/2 x 256 x D/M (hbpq)
  const float* S;
  const uint8_t* codes;
  const int32_t* ids;
  int32_t* out_ids;
  float* out_dists;
  int32_t* qcounter;     // work counter for persistent kernels (zeroed by the launcher)
  int sm_count;
  // reduced-precision shortlist scan (bpq_search_shortlist): per-query table
  // (int8, or FP16 bits) and step, and the output: the k best
  // (ord(score) << 32 | list position) per query
  const uint8_t* lut8;     // nq x M x 256 (int8 form)
  const uint16_t* lut16;   // nq x M x 256 (fp16 form)
  const float* lut_scale;  // nq
  uint64_t* sl_out;        // nq x k (any order; EMPTY padded)
  int32_t* status;         // workspace status word (a bounded wait that gave up sets STATUS_TIMEOUT)
  // HBPQ table form: per-query slots and bitmaps (HbpqArgs) and the tables
  const int32_t* hb_qbase;
  const int32_t* hb_qrows;
  const uint32_t* hb_qbits;
  const float* hb_tables;
  // reconstruction scans: when set, only the queries qlist[0 .. *qlist_n) are scored
  const int32_t* qlist;
  const int32_t* qlist_n;
  // FBPQ segment scan (not the work-queue form): when sel is set, only the queries
  // sel[0 .. *sel_n) are scored; when skip is set, the queries with skip[q] != 0
  // are left alone (another launch scores them)
  const int32_t* sel;
  const int32_t* sel_n;
  const uint8_t* skip;
  // persistent work-queue scan (work_W > 0, segment scans only): items (q, first
  // cell, end cell, partial slot or -1), counters (zeroed by the launcher), merge
  // records (q, first slot, items) and the partial lists
  int32_t work_W;
  int4* items;
  int32_t* n_items;
  int32_t* item_counter;
  int32_t* part_counter;
  int4* merges;
  int32_t* n_merges;
  int32_t* part_ids;
  float* part_dists;
};
constexpr int SCAN_MAX_ITEMS = 16;  // work items per query at most
void launch_scan(const ScanArgs& a, int scorer, cudaStream_t st);
// Shortlist scan with the int8 (f16 = false) or FP16 table: sl_out[q][0..k) =
// the k best (score, position), EMPTY padded.
void launch_scan_reduced(const ScanArgs& a, bool f16, cudaStream_t st);
// Exact FBPQ re-score of the shortlist: per query, the k best (distance, id) of
// its S shortlisted positions (EMPTY entries skipped).
struct RescoreArgs {
  const uint64_t* sl;     // nq x S
  int32_t S, k, T, M;
  int64_t nq;
  const float* d1;        // nq x T
  const float* d2;
  const float* lut;       // nq x M x 256 (FP32)
  const uint32_t* offsets;  // T*T + 1
  const uint32_t* hint;     // position_hints: the cell of every 256th list position
  const uint8_t* codes;
  const float* cross;
  const int32_t* ids;
  int32_t* out_ids;
  float* out_dists;
};
void launch_rescore(const RescoreArgs& r, cudaStream_t st);
// hint[b] = the cell holding list position min(256 b, n - 1), b = 0 .. ceil(n / 256):
// the cell of position p then lies in [hint[p / 256], hint[p / 256 + 1]].
size_t position_hint_count(int64_t n_points);
void launch_position_hints(const uint32_t* offsets, int64_t ncells, int64_t n_points, uint32_t* hint, cudaStream_t st);
// Per-query reduced-precision table and step from the FP32 table (bpq_search_shortlist step 1).
// out: nq x M x 256 uint8 (int8 form) or FP16 bits (fp16 form).
void launch_quant_lut(const float* lut, int M, int64_t nq, void* out, float* scale, bool f16, cudaStream_t st);
bool scan_supported(int D, int M);  // (D, M) shapes the scan kernels are built for

// Text returned by bpq_last_error on the calling thread (bpq_api.cu).
void set_last_error(const std::string& msg);

// Batch class of the autotuner's table: scorer, k <= 32, floor(log2 nq), floor(log2 mean L).
uint64_t tune_key(int scorer, int k, int64_t nq, double L_mean);

// The search pipeline of bpq_search / bpq_traverse (bpq_api.cu).
void run_queries(const bpq_index& ix, const float* q, int64_t nq, const int64_t* L_host, int64_t L_stride,
                 int k, int scorer, int32_t* out_ids, float* out_dists, bpq_cell* user_cells, int32_t user_cap,
                 int32_t* user_ncells, int64_t* user_npoints, void* ws, size_t ws_bytes, cudaStream_t st,
                 const int32_t* L32_pinned = nullptr);

// OPQ (bpq_opq.cu).  rotate_rows: Y = R X per row within nblk diagonal blocks (Rt:
// the blocks transposed, FP64), FP64 accumulation, rounded half up or FP32.
void rotate_rows(const float* X, int64_t n, int D, const double* Rt, int nblk, bool round, float* Y, cudaStream_t st);
void set_opq_rotations(bpq_index& ix, const double* R0, const double* R1, const double* R2, cudaStream_t st);
// xc = rot0 x (coarse space), xr = B rot0 x (residual space); either may be NULL
void rotate_for_index(const bpq_index& ix, const float* x, int64_t n, float* xc, float* xr, cudaStream_t st);
// queries: qc = rot0 q, qr = B rot0 q in FP32 (both required)
void rotate_queries(const bpq_index& ix, const float* q, int64_t n, float* qc, float* qr, cudaStream_t st);
std::vector<double> opq_learn_rotation(const float* X, int64_t n, int64_t ld, int col, int d, int groups,
                                       cudaStream_t st);

// Index build (bpq_build.cu).
void launch_encode(const bpq_index& ix, const float* x, int64_t n, int32_t* cell, uint8_t* codes,
                   cudaStream_t st);
void finalize_lists(bpq_index& ix, cudaStream_t st);
void train_codebooks(bpq_index& ix, const float* learn, int64_t n, cudaStream_t st);
void fill_sequential_ids(int32_t* ids, int64_t n, int64_t start, cudaStream_t st);
void launch_reconstruction_error(const bpq_index& ix, const float* x, int64_t n, const int32_t* cells,
                                 const uint8_t* codes, float* err, cudaStream_t st);
void build_point_cross(bpq_index& ix, cudaStream_t st);  // per-point Eq. 9 cross terms

}  // namespace bpq
