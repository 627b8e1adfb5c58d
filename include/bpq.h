/*
 * bpq.h — C ABI of a GB300 (sm_103a) implementation of the query-time path of
 * bilayer product-quantization search: Babenko & Lempitsky, "Improving Bilayer
 * Product Quantization for Billion-Scale Approximate Nearest Neighbors in High
 * Dimensions" (arXiv:1404.1831).
 *
 * Notation (the paper's): D dimensions, split into two halves of D/2; coarse
 * codebooks C^1, C^2 of T codewords each define T*T cells W_ij (Eq. 4); every
 * point stores its cell and an M-byte PQ code of its displacement from the cell
 * centroid (Eqs. 6-7), with K = 256 codewords per sub-quantizer.  The PQ split is
 * aligned with the halves: M even, D/M divides D/2.
 *
 * Conventions for every entry point:
 *  - Every call returns int: BPQ_OK (0) or a negative BPQ_E* code; the message
 *    of the last failure on the calling thread is bpq_last_error().  No C++
 *    exception crosses this boundary.
 *  - Pointers named *_dev are device pointers on the index's device; *_host are
 *    host pointers.  The caller owns every buffer it passes and the library
 *    never frees them.  The index owns its codebooks, tables and lists.
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  It is borrowed; work is enqueued on it and nothing synchronizes
 *    unless the entry point says so.
 *  - Matrices are row-major and dense: n x D float32 points/queries, etc.
 *  - Point ids are int32 >= 0; -1 marks an empty result slot.
 */
#ifndef BPQ_H_
#define BPQ_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
enum {
  BPQ_OK = 0,
  BPQ_EINVAL = -1,     /* invalid argument (null pointer, bad size, bad id, ...) */
  BPQ_ENOMEM = -2,     /* device or host allocation failed */
  BPQ_EIO = -3,        /* file could not be read or written */
  BPQ_ECORRUPT = -4,   /* index file failed its header or checksum test */
  BPQ_ETIMEOUT = -5,   /* a bounded device wait gave up */
  BPQ_ECUDA = -6,      /* a CUDA runtime call failed */
  BPQ_ECAPACITY = -7,  /* a fixed-size buffer (workspace, band, output) is too small */
  BPQ_ESTATE = -8      /* call out of order (e.g. search before bpq_finalize) */
};

/* Codebook variants. */
enum {
  BPQ_VARIANT_GLOBAL = 0, /* Multi-D-ADC codebooks: global R_1..R_M (§2.3.1); FBPQ and
                             reconstruction scoring */
  BPQ_VARIANT_LOCAL = 1   /* HBPQ: per-half-cell local codebooks Q^i_k, S^j_k (§3.2) */
};

/* Candidate scorers. */
enum {
  BPQ_SCORER_FBPQ = 0,  /* Eq. 8: per-query lookup tables reused in every cell (§3.1);
                           the query-independent cross term 2<c_ij, r> of Eq. 9 is
                           precomputed per point at index build, so a candidate
                           costs M table lookups plus one stored scalar */
  BPQ_SCORER_RECON = 1, /* Multi-D-ADC: per-cell query displacement and explicit
                           reconstruction, O(D) per candidate (§2.3.3) */
  BPQ_SCORER_HBPQ = 2,  /* HBPQ distance (§3.2: reconstruction with the local codebooks
                           Q^i_k, S^j_k of the cell's half-cells), evaluated through
                           per-(query, visited half-cell) tables built on the tensor
                           cores: A_i[k][t] = ||Q^i_k[t]||^2 + 2<c^1_i|k, Q^i_k[t]>
                           - 2<q_k, Q^i_k[t]> (B_j likewise), so a candidate costs M
                           lookups: d1[i] + d2[j] + sum_k A_i[k][c_k] + sum_k B_j[k][c_{M/2+k}].
                           An exact regrouping of the O(D) distance.  For k > 128, and
                           for queries whose tables do not fit the workspace, the O(D)
                           form below is used. */
  BPQ_SCORER_FBPQ_TABLES = 3, /* Eq. 8 with Eq. 9 evaluated from the T*M*K cross tables of
                           §3.3 at query time: 2M table lookups per candidate */
  BPQ_SCORER_HBPQ_RECON = 4 /* HBPQ as the paper evaluates it (§3.2): explicit
                           reconstruction with the local codebooks, O(D) per candidate */
};

typedef struct bpq_index bpq_index;

typedef struct {
  int32_t D;            /* dimensionality; even */
  int32_t T;            /* coarse codewords per half, 1..4096 (T*T cells) */
  int32_t M;            /* PQ sub-quantizers; even, D/M must divide D/2, M*256 <= 8192 */
  int32_t ksub;         /* codewords per PQ codebook; must be 256 (one byte per index) */
  int32_t variant;      /* BPQ_VARIANT_* */
  int32_t kmeans_iters; /* Lloyd iterations for bpq_train_load */
  int32_t opq;          /* 1: OPQ rotations (the "optimized" OMulti-D-OADC of §2.3; global
                           variant only): rot0 (D x D) on vectors before the coarse
                           quantization, rot1 / rot2 (D/2 x D/2) on the displacement halves
                           before the residual PQ; 0: none */
} bpq_params;

typedef struct {
  int64_t n_points;        /* points in the finalized lists */
  int64_t n_pending;       /* points added since the last bpq_finalize */
  int64_t n_nonempty;      /* non-empty cells of the finalized lists */
  int64_t max_cell;        /* largest cell population */
  int64_t device_bytes;    /* device memory the index holds */
  bpq_params params;
} bpq_info;

/* Read-only device views of the index arrays (valid until the next mutating call). */
typedef struct {
  const float* C1;      /* T x D/2 */
  const float* C2;      /* T x D/2 */
  const float* R;       /* M x 256 x D/M (global variant) */
  const float* Q;       /* T x M/2 x 256 x D/M (local variant, else NULL) */
  const float* S;       /* T x M/2 x 256 x D/M (local variant, else NULL) */
  const float* X1;      /* T x M/2 x 256: 2<c^1_i block k, R_k[t]>, k < M/2 (Eq. 9) */
  const float* X2;      /* T x M/2 x 256: 2<c^2_j block k, R_{M/2+k}[t]> (Eq. 9) */
  const uint32_t* offsets; /* T*T + 1 start positions of the cells (§2.3.2) */
  const uint8_t* codes; /* n_points x M, cell-contiguous */
  const int32_t* ids;   /* n_points, ascending inside each cell */
  const float* cross;   /* n_points: 2<c_ij, r> of each point (Eq. 9 cross term; global
                           variant, else NULL) */
} bpq_arrays;

/* One visited cell, as bpq_traverse writes it. */
typedef struct {
  uint32_t cell;   /* i*T + j */
  uint32_t begin;  /* first list position of the cell */
  uint32_t count;  /* points of the cell (> 0) */
  float key;       /* d1[i] + d2[j] in FP32 */
} bpq_cell;

/* Text of the last error on the calling thread ("" if none). */
const char* bpq_last_error(void);

/*
 * bpq_create — index from given codebooks (copied from host memory).
 *  C1_host, C2_host: T x D/2 coarse codebooks C^1, C^2 (§2.3.1).
 *  R_host: M x 256 x D/M residual codebooks R_1..R_M (§2.3.1); required for both
 *          variants (the local variant uses it only as its global fallback).
 *  Q_host, S_host: T x M/2 x 256 x D/M local codebooks Q^i_k, S^j_k (§3.2, Eq. 11);
 *          required for BPQ_VARIANT_LOCAL, ignored otherwise.
 * Builds the query-independent FBPQ tables X1, X2 (Eq. 9, §3.3) on the device.
 * Errors: BPQ_EINVAL for a bad shape or null pointer, BPQ_ENOMEM, BPQ_ECUDA.
 */
int bpq_create(bpq_index** out, const bpq_params* p, const float* C1_host, const float* C2_host,
               const float* R_host, const float* Q_host, const float* S_host, int device);

/*
 * bpq_train_load — train a new index on the GPU, or load one from a file.
 *  If learn_dev != NULL: learns C^1, C^2 by K-means on the point halves, then
 *  R_1..R_M by K-means on the displacements from the cell centroids (§2.3.1),
 *  and for BPQ_VARIANT_LOCAL the local codebooks of every half-cell (§3.2,
 *  Eqs. 10-11).  learn_dev: n_learn x D float32, device, integer-valued in
 *  [-2^20, 2^20] (K-means sums are exact int64 and every centroid is the mean
 *  rounded half up to an integer); n_learn >= max(T, 256).  K-means starts from
 *  the first T (or 256) learn vectors; local codebooks start from the global ones.
 *  Real-valued data: train on round(x * s) for a scale s of your choice, and add
 *  and search vectors scaled the same way (searches then report distances times
 *  s^2); or build the index from your own codebooks with bpq_create, which takes
 *  real-valued codebooks.  Queries and added points may be real-valued either way
 *  (query tiles that BF16 cannot hold exactly are tabulated in FP32).
 *  Synchronizes the stream before returning.
 *  Otherwise loads path (written by bpq_save) onto `device`.
 * Errors: BPQ_EINVAL (bad params, non-integer data), BPQ_EIO, BPQ_ECORRUPT,
 *         BPQ_ENOMEM, BPQ_ECUDA.
 */
int bpq_train_load(bpq_index** out, const bpq_params* p, const float* learn_dev, int64_t n_learn,
                   const char* path, int device, void* stream);

/*
 * bpq_encode — cell and PQ code of n points (§2.3.2, Eqs. 6-7; HBPQ Eq. 12),
 * without adding them.  x_dev: n x D float32.  cell_out_dev: n int32 (i*T + j).
 * codes_out_dev: n x M uint8.  Ties go to the lowest codeword index.
 */
int bpq_encode(const bpq_index* idx, const float* x_dev, int64_t n, int32_t* cell_out_dev,
               uint8_t* codes_out_dev, void* stream);

/*
 * bpq_reconstruction_error — squared encoding error ||x - xhat||^2 of n points
 * (§4.2, Fig. errors), xhat being the reconstruction of Eq. 7 (global variant)
 * or of §3.2 (local codebooks of the cell's half-cells) from the given cell and
 * code.  x_dev: n x D float32; cells_dev, codes_dev: as bpq_encode writes them
 * (cell ids in [0, T*T), codes M bytes per point); err_dev: n float32.  The
 * average over a dataset is the paper's average encoding error.
 */
int bpq_reconstruction_error(const bpq_index* idx, const float* x_dev, int64_t n, const int32_t* cells_dev,
                             const uint8_t* codes_dev, float* err_dev, void* stream);

/*
 * bpq_add — encode n points and append them to the pending set.  ids_dev: n
 * int32 >= 0 (NULL = consecutive ids starting at the number of points added so
 * far).  The points become searchable after bpq_finalize.  Total points < 2^32.
 */
int bpq_add(bpq_index* idx, const float* x_dev, int64_t n, const int32_t* ids_dev, void* stream);

/*
 * bpq_finalize — build the inverted multi-index lists (§2.3.2): all points of a
 * cell contiguous, cells in id order, ids ascending inside a cell, plus the
 * T*T + 1 cell start offsets.  Merges pending points into existing lists.
 * Synchronizes the stream before returning.
 */
int bpq_finalize(bpq_index* idx, void* stream);

/*
 * bpq_set_global_counts — make this index a point shard of a larger index (the
 * layout for an index that does not fit one GPU; queries are independent,
 * §2.3.3, so the shards need no exchange but the final merge).  counts_host:
 * T*T int64, the number of points of each cell (i*T + j) in the WHOLE index (the
 * sum of every shard's counts).  From then on every search of this index
 * traverses the cells with these counts -- the stopping rule "the visited cells
 * hold at least L points" of §2.3.3 is the whole index's, so every shard visits
 * the same cells and reports the same L' -- and scores only the points this
 * shard holds; the k best of each shard, merged by (distance, id), are exactly
 * the whole index's answer.  NULL clears the setting.  Call after bpq_finalize
 * (which clears it, as the shard's lists change); not saved by bpq_save.
 * Errors: BPQ_ESTATE before bpq_finalize; BPQ_EINVAL for a count outside
 * [0, 2^32) or below this shard's count of the same cell.
 * bpq_search_noalloc rejects a shard.
 */
int bpq_set_global_counts(bpq_index* idx, const int64_t* counts_host);

/*
 * bpq_query_tables — per-query tables of §3.1 for nq queries (queries_dev:
 * nq x D float32): d1_dev, d2_dev: nq x T squared distances ||q^1 - c^1_i||^2,
 * ||q^2 - c^2_j||^2 (Eqs. 2-3); lut_dev (may be NULL): nq x M x 256 entries
 * ||R_k[t]||^2 - 2<q_k, R_k[t]> (the query terms of Eq. 8 with the codeword norms
 * of Eq. 9).
 */
int bpq_query_tables(const bpq_index* idx, const float* queries_dev, int64_t nq, float* d1_dev,
                     float* d2_dev, float* lut_dev, void* stream);

/*
 * Candidate budgets: L_host points to nq int64 values (L_stride == 1) or to one
 * value used for every query (L_stride == 0); every L must be in [1, 2^31).
 */

/* Device workspace bytes bpq_search / bpq_traverse need for nq queries at budget <= L_max. */
size_t bpq_search_workspace_size(const bpq_index* idx, int64_t nq, int64_t L_max, int32_t k,
                                 int32_t scorer);

/*
 * bpq_traverse — visit order of the inverted multi-index (§2.3.3): for each query,
 * the non-empty cells in non-decreasing d1[i] + d2[j] order, ties by cell id
 * (bpq_search visits the same cells but does not need them in order),
 * up to and including the first cell at which the visited points reach L (the
 * multi-sequence stopping rule; all cells if the index holds fewer points).
 * Empty cells consume order but hold no candidates, so they are not listed.
 *  cells_dev: nq x cap bpq_cell; ncells_dev: nq int32; npoints_dev: nq int64 (L').
 *  If a query visits more than cap non-empty cells its ncells is -1.
 *  workspace: bpq_search_workspace_size(idx, nq, max L, 1, BPQ_SCORER_FBPQ) bytes.
 */
int bpq_traverse(const bpq_index* idx, const float* queries_dev, int64_t nq, const int64_t* L_host,
                 int64_t L_stride, int32_t cap, bpq_cell* cells_dev, int32_t* ncells_dev,
                 int64_t* npoints_dev, void* workspace_dev, size_t workspace_bytes, void* stream);

/*
 * bpq_search — approximate k-NN (§2.3.3, §3.1, §3.2): for each query, the k
 * candidates of the visited cells with the smallest squared distance
 * ||q - x^||^2 (Eq. 8), ascending, ties by id; slots beyond the candidate count
 * hold id -1 and distance +inf.
 *  queries_dev: nq x D float32; k in [1, 1024]; scorer: BPQ_SCORER_*
 *  (FBPQ, FBPQ_TABLES and RECON need the global variant, HBPQ and HBPQ_RECON the
 *  local one).
 *  ids_dev: nq x k int32; dists_dev: nq x k float32.
 *  workspace_dev: at least bpq_search_workspace_size(idx, nq, max L, k, scorer)
 *  bytes, or fewer: queries are then processed in chunks that fit (at least one
 *  query must fit, else BPQ_ECAPACITY).
 * Asynchronous on stream; per-query failures of a fixed-size buffer (a cell tie
 * group larger than the traversal band) are reported by bpq_search_status.
 * With the FBPQ scorer and k <= 128, part of the work (the PQ table, and the
 * traversal and scan of the queries the common traversal path hands over) runs
 * on a second stream that joins `stream` before the call's work on it ends; that
 * stream and its events are created, per device and caller stream, on the first
 * such call outside a stream capture (a call under capture that finds none runs
 * everything on `stream`) and are kept until the process exits (they do not
 * survive cudaDeviceReset).
 */
int bpq_search(const bpq_index* idx, const float* queries_dev, int64_t nq, const int64_t* L_host,
               int64_t L_stride, int32_t k, int32_t scorer, int32_t* ids_dev, float* dists_dev,
               void* workspace_dev, size_t workspace_bytes, void* stream);

/*
 * bpq_search_shortlist — FBPQ search with a reduced-precision table and exact
 * re-scoring (a precision variant of §3.1; the paper scans with full-precision
 * tables).  Per query:
 *  1. the PQ table lut[k][t] of Eq. 8/9 is shifted per sub-quantizer by its
 *     minimum lo_k; with range = max_k(max_t lut[k][t] - lo_k), in IEEE FP32:
 *     BPQ_LUT_I8:  step s = range / 255 (s = 1 if range is 0),
 *                  q8[k][t] = round_half_even((lut[k][t] - lo_k) / s) in [0, 255];
 *     BPQ_LUT_F16: step s = the smallest power of two >= 1 with range <= 65504 s,
 *                  h[k][t] = the FP16 value nearest to (lut[k][t] - lo_k) / s
 *                  (ties to even; the scaling is exact);
 *  2. every candidate of the visited cells (the same cells as bpq_search) gets the
 *     score (key(i,j) + cross(p)) + s * part in FP32, in that order, with
 *     part = sum_k q8[k][c_k] (an exact integer) or the FP32 sum of the h[k][c_k]
 *     taken in sub-quantizer order k = 0 .. M-1 (the constant sum_k lo_k is left
 *     out), and the `shortlist` best by (score, position in the index lists) are
 *     kept;
 *  3. those are re-scored with the exact FBPQ distance (Eq. 8-9, as bpq_search)
 *     and the k best by (distance, id) are returned as by bpq_search.
 *  lut_precision: BPQ_LUT_I8 or BPQ_LUT_F16; shortlist in [k, 1024].
 *  Needs the global variant.  workspace: bpq_search_shortlist_workspace_size
 *  bytes or fewer (chunks, as bpq_search; the same size for both precisions).
 *  Asynchronous on stream.
 */
enum { BPQ_LUT_I8 = 1, BPQ_LUT_F16 = 2 };
size_t bpq_search_shortlist_workspace_size(const bpq_index* idx, int64_t nq, int64_t L_max, int32_t shortlist);
int bpq_search_shortlist(const bpq_index* idx, const float* queries_dev, int64_t nq, const int64_t* L_host,
                         int64_t L_stride, int32_t k, int32_t shortlist, int32_t lut_precision, int32_t* ids_dev,
                         float* dists_dev, void* workspace_dev, size_t workspace_bytes, void* stream);

/*
 * bpq_scan — the scan and top-k stage of bpq_search alone (§2.3.3 reranking,
 * §3.1, §3.2), on cells written by bpq_traverse: for each query the k smallest
 * (distance, id) over every point of its ncells_dev[q] visited cells.
 *  lut_dev: nq x M x 256 tables from bpq_query_tables (FBPQ scorers, else ignored);
 *  cells_dev: nq x cap; queries_dev: nq x D (reconstruction scorers);
 *  counter_dev: one int32 of device scratch (work counter of the persistent
 *  reconstruction kernels).  Outputs as bpq_search.  Asynchronous on stream.
 */
int bpq_scan(const bpq_index* idx, const float* queries_dev, int64_t nq, const float* lut_dev,
             const bpq_cell* cells_dev, const int32_t* ncells_dev, int32_t cap, int32_t k, int32_t scorer,
             int32_t* ids_dev, float* dists_dev, int32_t* counter_dev, void* stream);

/*
 * bpq_search_status — synchronizes the stream and returns BPQ_OK; BPQ_ETIMEOUT if
 * a bounded device wait of the last bpq_search / bpq_traverse on this workspace
 * gave up (a tensor-core table tile whose MMA did not signal completion; that tile
 * was recomputed on the CUDA cores, so the results are still complete); or
 * BPQ_ECAPACITY if a query overflowed a fixed-size buffer.
 */
int bpq_search_status(const bpq_index* idx, void* workspace_dev, void* stream);

/*
 * bpq_search_host — bpq_search with host buffers: copies queries_host (nq x D
 * float32) to the device, searches with a workspace the index owns, copies the
 * results to ids_host / dists_host (nq x k) and synchronizes the stream.
 */
int bpq_search_host(bpq_index* idx, const float* queries_host, int64_t nq, const int64_t* L_host,
                    int64_t L_stride, int32_t k, int32_t scorer, int32_t* ids_host,
                    float* dists_host, void* stream);

/*
 * bpq_search_noalloc — bpq_search without any device allocation, for callers
 * that cannot call cudaMalloc: programs whose device memory is all owned by
 * their own pool or budget, and latency-critical loops where a cudaMalloc /
 * cudaFree (which can synchronize the whole device) is not acceptable.  The
 * paper has no counterpart: this is a deployment convenience of this library.
 *  Same arguments and results as bpq_search, minus the workspace: the scratch
 *  data (query tables, visited-cell lists, counters) live in one fixed array of
 *  BPQ_NOALLOC_SCRATCH_BYTES of device memory inside the library, reserved on
 *  every GPU that loads the library until the process exits.
 *  A batch fits if bpq_search_workspace_size(idx, nq, max L, k, scorer) <=
 *  BPQ_NOALLOC_SCRATCH_BYTES; a larger batch returns BPQ_ECAPACITY before any
 *  GPU work (split the batch).  status_dev (may be NULL): one int32 of device
 *  memory that receives 0, or 1 if a query overflowed the traversal band.
 *  The first call on a device looks up the array's device address (one-time
 *  set-up), so make that first call before any stream capture.  That address
 *  belongs to the device's primary context: calls from another context of the
 *  device, or after cudaDeviceReset, are not supported.  Every call
 *  shares the array and it keeps the previous call's contents; calls whose GPU
 *  work overlaps (other streams, other threads) race on it, so order them.
 *  Per-query budgets (L_stride == 1) are copied from host memory with
 *  cudaMemcpyAsync.  Failures are reported by the return code only
 *  (bpq_last_error is not updated): BPQ_EINVAL, BPQ_ESTATE, BPQ_ECAPACITY,
 *  BPQ_ECUDA as for bpq_search.  Asynchronous on stream.
 */
#define BPQ_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20) /* 32 MiB */
int bpq_search_noalloc(const bpq_index* idx, const float* queries_dev, int64_t nq, const int64_t* L_host,
                       int64_t L_stride, int32_t k, int32_t scorer, int32_t* ids_dev, float* dists_dev,
                       int32_t* status_dev, void* stream);

/*
 * bpq_set_hbpq_table_budget — table slots reserved per query for the HBPQ table
 * form of bpq_search (BPQ_SCORER_HBPQ).  One slot is one (query, visited
 * half-cell) table of M/2 x 256 floats (4 KB at M = 8); a query visits one slot
 * per distinct row i and per distinct column j of its visited cells.  0 (the
 * default) reserves about 4 sqrt(L / rho) + 32 slots per query (rho = points per
 * non-empty cell, at most 2T).  A query whose slots do not fit the reserved area is
 * scored with the O(D) reconstruction instead, with the same results.  The value
 * also sizes bpq_search_workspace_size.  Errors: BPQ_EINVAL (NULL index, negative
 * or non-finite value).
 */
int bpq_set_hbpq_table_budget(bpq_index* idx, double slots_per_query);

/*
 * Continuous-batching server: a request loop over one resident index (serving
 * is not part of the paper, which measures one query at a time; every batch runs
 * the bpq_search pipeline of §2.3.3 / §3.1 / §3.2 unchanged, so each query's
 * answer equals bpq_search of that query alone).
 *
 * The server owns `slots` batches in flight, each with its own non-blocking CUDA
 * stream, a device workspace of device_bytes / slots bytes, device and page-locked
 * host buffers for max_batch queries, and a completion event.  Progress calls
 * retire finished slots (their results are then in host memory) and fill free
 * slots with batches of waiting requests, oldest first, enqueued asynchronously
 * (H2D copy, search, D2H copy); batches therefore overlap on the GPU.  A batch
 * admits requests only while bpq_search_workspace_size of the batch at its largest
 * L fits the slot's workspace (admission by device memory), and with
 * group_by_budget it takes requests of one budget class only (floor(log2 L)), so
 * short queries do not wait for the long queries of their batch.
 * A server is used from one host thread at a time; the index must outlive it and
 * must not be modified while it exists.
 */
typedef struct bpq_server bpq_server;
typedef struct {
  int32_t slots;           /* batches in flight, 1..64 */
  int32_t k;               /* results per query, 1..1024 */
  int32_t scorer;          /* BPQ_SCORER_* (matching the index's variant) */
  int32_t group_by_budget; /* 1: one budget class per batch; 0: first come first served */
  int64_t max_batch;       /* queries per batch, 1..2^20 */
  int64_t L_max;           /* the largest candidate budget a request may ask for */
  size_t device_bytes;     /* device memory for all slots' workspaces */
} bpq_server_config;
typedef struct {
  int64_t batches;         /* batches launched */
  int64_t queries;         /* queries launched */
  int64_t max_in_flight;   /* most batches in flight at once */
  int64_t pending;         /* requests waiting for a slot */
  int64_t slot_workspace_bytes;
} bpq_server_stats;

/* bpq_server_create — allocates the slots.  Errors: BPQ_EINVAL, BPQ_ESTATE
 * (unfinalized index), BPQ_ECAPACITY (device_bytes / slots cannot hold one query at
 * L_max), BPQ_ENOMEM, BPQ_ECUDA. */
int bpq_server_create(bpq_server** out, const bpq_index* idx, const bpq_server_config* cfg);
/* bpq_server_submit — queues n requests: queries_host n x D float32 (copied),
 * L_host n budgets in [1, L_max]; request numbers first_request_out .. + n - 1
 * (may be NULL).  Nothing is launched until bpq_server_progress. */
int bpq_server_submit(bpq_server* s, const float* queries_host, const int64_t* L_host, int64_t n,
                      int64_t* first_request_out);
/* bpq_server_progress — retires finished batches and launches waiting requests
 * into free slots.  wait != 0: if neither happened, blocks until one in-flight
 * batch finishes, then launches again. */
int bpq_server_progress(bpq_server* s, int32_t wait);
/* bpq_server_take — up to max_n finished requests, in completion order:
 * request numbers, ids / dists (max_n x k, as bpq_search), latency_s (may be NULL:
 * seconds from submission to the progress call that saw the batch finish);
 * *n_out = how many were written. */
int bpq_server_take(bpq_server* s, int64_t max_n, int64_t* request_out, int32_t* ids_out, float* dists_out,
                    double* latency_s_out, int64_t* n_out);
/* bpq_server_run_trace — serves a recorded arrival trace: request i (queries_host
 * row i, budget L_host[i]) arrives arrival_s[i] seconds (non-decreasing) after the
 * call starts; the server admits arrived requests, launches and retires batches as
 * above until all n are answered.  ids_out / dists_out: n x k rows in request
 * order; latency_s_out[i]: arrival to results in host memory.  Needs an idle
 * server.  Returns when every request is answered. */
int bpq_server_run_trace(bpq_server* s, const float* queries_host, const int64_t* L_host, const double* arrival_s,
                         int64_t n, int32_t* ids_out, float* dists_out, double* latency_s_out);
int bpq_server_get_stats(const bpq_server* s, bpq_server_stats* out);
/* bpq_server_free — waits for the slots' streams and releases the server (NULL is allowed). */
void bpq_server_free(bpq_server* s);

/*
 * bpq_set_scan_work_size — how bpq_search schedules the scan of the FBPQ and
 * HBPQ scorers (k <= 128).  0 (the default): one CTA per query.  W > 0: the
 * visited cells of each query are cut into contiguous work items of about W
 * candidates (at most 16 items per query), a persistent wave of CTAs takes the
 * items from a queue, and the partial top-k lists of a split query are merged by
 * (distance, id); the answers are the same.  Long queries then no longer set the
 * batch's tail.  bpq_autotune picks W by measurement.  Errors: BPQ_EINVAL.
 */
int bpq_set_scan_work_size(bpq_index* idx, int32_t candidates_per_item);

/*
 * bpq_autotune — picks the scan schedule of bpq_search for one batch class by
 * measurement: runs the batch (queries_dev, nq, budgets, k, scorer and outputs as
 * for bpq_search; the call allocates a workspace for the whole batch) with each
 * candidate work-item size W in {0, 4096, 8192, 16384, 32768} (0: one CTA per
 * query; W: the persistent work-queue scan of bpq_set_scan_work_size), four
 * timed runs each with CUDA events on `stream` (the first discarded), and keeps the
 * fastest for the class (scorer, k <= 32, floor(log2 nq), floor(log2 mean L)).
 * Later bpq_search calls of that class use it; other classes keep the index's
 * setting.  chosen_out (may be NULL) receives the chosen W.  Synchronizes the
 * stream.  The outputs hold the last run's (identical) answers.  (An engineering
 * step of this library; the paper has no scheduling.)
 */
int bpq_autotune(bpq_index* idx, const float* queries_dev, int64_t nq, const int64_t* L_host, int64_t L_stride,
                 int32_t k, int32_t scorer, int32_t* ids_dev, float* dists_dev, void* stream, int32_t* chosen_out);

/*
 * Search graphs: one batch shape of bpq_search captured as a CUDA graph and
 * replayed with one launch (every kernel, memset and budget copy of the
 * pipeline), for repeated batches of the same shape where per-kernel launch costs
 * matter.  bpq_graph_create captures the search of nq queries read from
 * queries_dev with results written to ids_dev / dists_dev (nq x k, as
 * bpq_search): those device buffers are fixed for the graph's lifetime (write new
 * queries into queries_dev before a launch).  The graph owns a workspace for the
 * whole batch and page-locked budgets: L_host / L_stride as bpq_search; with
 * per-query budgets (L_stride == 1), bpq_graph_set_budgets replaces them (values
 * in [1, the largest budget given at creation]), read by the next launches (do not
 * call it while a launch of the graph is in flight).  The scan schedule in force
 * at creation (bpq_set_scan_work_size, or a bpq_autotune choice for the class) is
 * captured.  bpq_graph_create runs the search once uncaptured and synchronizes;
 * bpq_graph_launch is asynchronous on `stream`.  The index must stay unchanged
 * while the graph exists.  Errors: BPQ_EINVAL, BPQ_ESTATE, BPQ_ENOMEM, BPQ_ECUDA.
 */
typedef struct bpq_graph bpq_graph;
int bpq_graph_create(bpq_graph** out, const bpq_index* idx, const float* queries_dev, int64_t nq,
                     const int64_t* L_host, int64_t L_stride, int32_t k, int32_t scorer, int32_t* ids_dev,
                     float* dists_dev);
int bpq_graph_set_budgets(bpq_graph* g, const int64_t* L_host);
int bpq_graph_launch(bpq_graph* g, void* stream);
void bpq_graph_free(bpq_graph* g);

/*
 * bpq_set_rotations — the OPQ rotations of an index made by bpq_create with
 * params.opq = 1 (its codebooks C^1, C^2 then live in the space of rot0 x and R_k in
 * the space of [rot1 d^1; rot2 d^2]); before any point is added.  R0: D x D, R1, R2:
 * D/2 x D/2, row-major FP64 host arrays (orthogonal; copied).  bpq_train_load with
 * params.opq = 1 learns them instead (parametric OPQ: covariance eigenvectors dealt
 * to the subspaces by balanced log-eigenvalue sums; the rotated learn vectors and
 * displacements are rounded half up before K-means).  Errors: BPQ_EINVAL, BPQ_ESTATE.
 */
int bpq_set_rotations(bpq_index* idx, const double* R0_host, const double* R1_host, const double* R2_host);
/* bpq_get_rotations — copies an OPQ index's rotations to host arrays (sizes as above). */
int bpq_get_rotations(const bpq_index* idx, double* R0_host, double* R1_host, double* R2_host);

/* bpq_info / bpq_arrays — sizes and read-only device views (see the structs). */
int bpq_get_info(const bpq_index* idx, bpq_info* out);
int bpq_get_arrays(const bpq_index* idx, bpq_arrays* out);

/* bpq_save — write codebooks, lists and a checksummed header to path (synchronizes). */
int bpq_save(const bpq_index* idx, const char* path);

/* bpq_free — release the index and its device memory (NULL is allowed). */
void bpq_free(bpq_index* idx);

#ifdef __cplusplus
}
#endif

#endif /* BPQ_H_ */
