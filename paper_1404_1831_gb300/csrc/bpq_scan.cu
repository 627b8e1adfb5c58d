// Candidate scans and top-k selection (§2.3.3 reranking, §3.1 FBPQ, §3.2 HBPQ).
//
// Input: the visited non-empty cells of each query (bpq_cell lists written by the
// traversal).  Every point of those cells is a candidate; the scan computes its
// approximate squared distance and keeps the k smallest (distance, id) pairs.
//
//  * FBPQ (§3.1): with the per-query tables in shared memory, a candidate with
//    code [r_1..r_M] in cell (i, j) costs M table lookups plus M lookups into the
//    query-independent cross tables (Eq. 9):
//       key(i,j) + sum_k ( lut[k][r_k] + X[k][r_k] ),  X = X1[i] for k < M/2, X2[j] else
//    where key(i, j) = d1[i] + d2[j] = ||q - [c^1_i; c^2_j]||^2.
//  * Reconstruction (Multi-D-ADC, §2.3.3): per visited cell the query displacement
//    q - [c^1_i; c^2_j] is staged in shared memory, and every candidate costs an
//    O(D) distance to its reconstructed displacement [R_1[r_1] .. R_M[r_M]].
//  * HBPQ (§3.2): the same O(D) reconstruction with the local codebooks Q^i_k and
//    S^j_k of the cell's two half-cells.
//
// Top-k: each warp keeps a sorted list of its best KP >= k composites
// (ord(distance) << 32 | id) in shared memory plus a buffer of new candidates;
// a full buffer is merged by a warp-wide bitonic sort.  A block-wide threshold
// (the smallest k-th best of any warp) filters candidates; ids are read only for
// candidates that pass it.  At the end the warp lists are merged by rank.
#include <cuda_fp16.h>

#include <algorithm>
#include <type_traits>

#include "bpq_internal.cuh"

namespace bpq {
namespace {

constexpr uint64_t EMPTY = ~0ull;

template <int KP>
struct WarpTopK {
  static constexpr int AREA = 2 * (KP > 64 ? KP : 64);
  static constexpr int BUF = AREA - KP;
  uint64_t* area;
  int nbuf;
  __device__ void init(uint64_t* a) {
    area = a;
    nbuf = 0;
    for (int i = threadIdx.x & 31; i < AREA; i += 32) area[i] = EMPTY;
    __syncwarp();
  }
  __device__ void flush(int k, unsigned long long* thr) {
    warp_bitonic_sort(area, AREA);
    for (int i = KP + (threadIdx.x & 31); i < AREA; i += 32) area[i] = EMPTY;
    nbuf = 0;
    __syncwarp();
    if ((threadIdx.x & 31) == 0) atomicMin(thr, (unsigned long long)area[k - 1]);
    __syncwarp();
  }
  // Warp-collective: every lane calls with its own (accept, composite).
  __device__ void offer(bool acc, uint64_t comp, int k, unsigned long long* thr) {
    const unsigned m = __ballot_sync(0xffffffffu, acc);
    if (!m) return;
    if (acc) area[KP + nbuf + __popc(m & lanemask_lt())] = comp;
    nbuf += __popc(m);
    if (nbuf > BUF - 32) {
      __syncwarp();
      flush(k, thr);
    }
  }
};

// Merge NW sorted warp lists (stride AREA, first KP entries) into the k best,
// written to out_ids / out_dists.  Ties between equal composites are broken by
// warp index, so every element gets a distinct rank.
__device__ void merge_lists(const uint64_t* areas, int NW, int KP, int AREA, int k, int32_t* out_ids,
                            float* out_dists) {
  const int total = NW * KP;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int w = e / KP, r = e % KP;
    const uint64_t x = areas[w * AREA + r];
    int rank = r;
    for (int w2 = 0; w2 < NW && rank < k; ++w2) {
      if (w2 == w) continue;
      const uint64_t* b = areas + w2 * AREA;
      int lo = 0, hi = KP;
      if (w2 < w) {
        while (lo < hi) {
          int mid = (lo + hi) >> 1;
          if (b[mid] <= x) lo = mid + 1; else hi = mid;
        }
      } else {
        while (lo < hi) {
          int mid = (lo + hi) >> 1;
          if (b[mid] < x) lo = mid + 1; else hi = mid;
        }
      }
      rank += lo;
    }
    if (rank < k) {
      out_ids[rank] = (x == EMPTY) ? -1 : (int32_t)(uint32_t)x;
      out_dists[rank] = (x == EMPTY) ? __int_as_float(0x7f800000) : ord2f((uint32_t)(x >> 32));
    }
  }
}

// Code words of one point: M bytes as M/4 32-bit words.
template <int M>
struct Code {
  uint32_t w[M / 4];
  __device__ __forceinline__ void load(const uint8_t* codes, uint32_t pos) {
    if constexpr (M == 4) {
      w[0] = __ldg(reinterpret_cast<const uint32_t*>(codes) + pos);
    } else if constexpr (M == 8) {
      uint2 v = __ldg(reinterpret_cast<const uint2*>(codes) + pos);
      w[0] = v.x;
      w[1] = v.y;
    } else {
      static_assert(M == 16, "M must be 4, 8 or 16");
      uint4 v = __ldg(reinterpret_cast<const uint4*>(codes) + pos);
      w[0] = v.x;
      w[1] = v.y;
      w[2] = v.z;
      w[3] = v.w;
    }
  }
  __device__ __forceinline__ uint32_t byte(int k) const { return (w[k >> 2] >> (8 * (k & 3))) & 0xffu; }
};

// Last index c in [0, n) with pref[c] <= f (pref strictly increasing, pref[0] = 0).
__device__ __forceinline__ int find_cell(const int* pref, int n, int f) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (pref[mid] <= f) lo = mid; else hi = mid;
  }
  return lo;
}

// Exclusive scan of one int per thread over the block (NT threads); returns the
// exclusive prefix and writes the total to *total.  Uses tmp[NT/32 + 1].
template <int NT>
__device__ int block_excl_scan(int x, int* tmp, int* total) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  int v = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, v, o);
    if (l >= o) v += y;
  }
  __syncthreads();
  if (l == 31) tmp[w] = v;
  __syncthreads();
  if (w == 0) {
    int t = (l < NT / 32) ? tmp[l] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, t, o);
      if (l >= o) t += y;
    }
    if (l < NT / 32) tmp[l] = t;
  }
  __syncthreads();
  *total = tmp[NT / 32 - 1];
  return v - x + (w > 0 ? tmp[w - 1] : 0);
}

// ---------------------------------------------------------------------------
// Block-wide top-k: accepted composites go to a shared buffer; when it fills up,
// a radix select on the distance bits finds the k-th smallest distance v_k of
// the buffer, everything above it is dropped and v_k becomes the threshold.
// The buffer therefore always holds every candidate that can still be in the
// top k (ties at v_k included); the final list is its exact (distance, id) sort.
// ---------------------------------------------------------------------------
template <int NT, int CAP_ = 2048>
struct BlockTopK {
  static constexpr int CAP = CAP_;  // buffer entries (a power of two); rounds add at most NT * ILP
  uint64_t* buf;    // CAP
  uint64_t* alt;    // CAP (compaction target)
  int* nbuf;        // shared counter
  unsigned long long* thr;  // shared threshold composite
  uint32_t* hist;   // 256 + 8 scratch
};

// k-th smallest value of the distance bits (high 32) among buf[0..n): 4 passes of
// 8-bit histograms.  All threads call; returns the value on every thread.
template <int NT>
__device__ uint32_t select_kth_hi(const uint64_t* buf, int n, int k, uint32_t* hist) {
  uint32_t prefix = 0, mask = 0;
  int rank = k;  // 1-based rank still to find among keys matching prefix
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int t = threadIdx.x; t < 256; t += NT) hist[t] = 0;
    __syncthreads();
    for (int e0 = 0; e0 < n; e0 += NT) {
      const int e = e0 + threadIdx.x;
      const uint32_t key = e < n ? (uint32_t)(buf[e] >> 32) : 0u;
      warp_hist_add(hist, (key >> shift) & 255u, e < n && (key & mask) == prefix);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      const int l = threadIdx.x;
      uint32_t c[8], tot = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        c[i] = hist[l * 8 + i];
        tot += c[i];
      }
      uint32_t incl = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (l >= o) incl += y;
      }
      uint32_t run = incl - tot;
      // the bin where the running count reaches `rank`
      const bool mine = run < (uint32_t)rank && (uint32_t)rank <= incl;
      if (mine) {
        int d = 0;
        while (run + c[d] < (uint32_t)rank) run += c[d++];
        hist[256] = (uint32_t)(l * 8 + d);
        hist[257] = run;
      }
    }
    __syncthreads();
    const uint32_t d = hist[256];
    rank -= (int)hist[257];
    prefix |= d << shift;
    mask |= 255u << shift;
    __syncthreads();
  }
  return prefix;
}

// Keep the entries whose distance bits are <= v (the k-th smallest): moves them
// to alt, swaps buffers.  Updates *nbuf and the threshold.
template <int NT, int CAP>
__device__ void block_topk_prune(BlockTopK<NT, CAP>& tk, int k) {
  const int n = *tk.nbuf;
  if (n <= k) {
    __syncthreads();
    return;
  }
  const uint32_t v = select_kth_hi<NT>(tk.buf, n, k, tk.hist);
  if (threadIdx.x == 0) tk.hist[258] = 0;
  __syncthreads();
  for (int e = threadIdx.x; e < n; e += NT) {
    const uint64_t x = tk.buf[e];
    if ((uint32_t)(x >> 32) <= v) tk.alt[atomicAdd(&tk.hist[258], 1u)] = x;
  }
  __syncthreads();
  const int kept = (int)tk.hist[258];
  uint64_t* t = tk.buf;
  tk.buf = tk.alt;
  tk.alt = t;
  if (kept > CAP / 2) {
    // a huge tie group at v: sort exactly and keep k
    int n2 = 1;
    while (n2 < kept) n2 <<= 1;
    for (int e = kept + threadIdx.x; e < n2; e += NT) tk.buf[e] = EMPTY;
    block_bitonic_sort(tk.buf, n2);
    if (threadIdx.x == 0) {
      *tk.nbuf = k;
      *tk.thr = tk.buf[k - 1];
    }
  } else if (threadIdx.x == 0) {
    *tk.nbuf = kept;
    *tk.thr = ((unsigned long long)v << 32) | 0xffffffffull;
  }
  __syncthreads();
}

// Final: exact (distance, id) order of the buffer, first k written out.
template <int NT, int CAP>
__device__ void block_topk_finish(BlockTopK<NT, CAP>& tk, int k, int32_t* out_ids, float* out_dists) {
  block_topk_prune<NT, CAP>(tk, k);
  const int n = *tk.nbuf;
  int n2 = 1;
  while (n2 < n) n2 <<= 1;
  for (int e = n + threadIdx.x; e < n2; e += NT) tk.buf[e] = EMPTY;
  block_bitonic_sort(tk.buf, n2);
  for (int r = threadIdx.x; r < k; r += NT) {
    const uint64_t x = r < n ? tk.buf[r] : EMPTY;
    out_ids[r] = (x == EMPTY) ? -1 : (int32_t)(uint32_t)x;
    out_dists[r] = (x == EMPTY) ? __int_as_float(0x7f800000) : ord2f((uint32_t)(x >> 32));
  }
}

// ---------------------------------------------------------------------------
// FBPQ scan variants:
//  FB_POINT : per-point cross term (one coalesced float per candidate)
//  FB_TABLES: cross terms gathered from the X1 / X2 tables (2M lookups)
//  FB_F16   : FP16 table (bpq_search_shortlist): score (key + cross) + s * the FP32
//             sum, in sub-quantizer order, of M FP16 entries; ranked as FB_Q8
//  FB_Q8    : int8 table (bpq_search_shortlist): score (key + cross) + s * sum of
//             M int8 entries, ranked by (score, list position); no id is read
// The round-based kernel below (one CTA per query) takes FB_TABLES and k > 128;
// the warp-segment kernel further down FB_POINT with k <= 128 and the shortlists.
// ---------------------------------------------------------------------------
enum { FB_POINT = 0, FB_TABLES = 1, FB_Q8 = 2, FB_F16 = 3 };

template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src),
                 "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Code words of one point as a single vector (M bytes).
template <int M>
using CodeVec = typename std::conditional<M == 16, uint4, uint2>::type;

//  Loads are pipelined: each thread copies the codes (and cross terms) of its
//  next round of ILP candidates into its own shared-memory slots with cp.async
//  while it scores the current round (two slot sets), so no register holds a
//  load in flight.
template <int M, int VAR, int ILP, int CAP, int SUB>
__global__ void __launch_bounds__(256) fbpq_scan_kernel(ScanArgs a) {
  static_assert(VAR == FB_POINT || VAR == FB_TABLES, "the shortlists run on the warp-segment scan");
  constexpr bool POINT = VAR != FB_TABLES;
  constexpr int NT = 256, NW = NT / 32, CH = NT, M2 = M / 2;
  constexpr int PER = SUB / NT;      // candidates per thread in the cell map of a slice
  using TK = BlockTopK<NT, CAP>;
  using CV = CodeVec<M>;
  extern __shared__ __align__(16) unsigned char smem[];
  float* lut = reinterpret_cast<float*>(smem);
  uint64_t* bufs = reinterpret_cast<uint64_t*>(lut + M * KSUB);  // 2 x CAP
  CV* sc = reinterpret_cast<CV*>(bufs + 2 * CAP);                 // [2][ILP][NT] staged codes
  float* sx = reinterpret_cast<float*>(sc + 2 * ILP * NT);        // [2][ILP][NT] staged cross terms
  uint8_t* cmap = reinterpret_cast<uint8_t*>(sx + (POINT ? 2 * ILP * NT : 0));  // SUB
  __shared__ uint32_t c_beg[CH];
  __shared__ uint32_t c_x1[POINT ? 1 : CH];
  __shared__ uint32_t c_x2[POINT ? 1 : CH];
  __shared__ float c_key[CH];
  __shared__ int c_pref[CH + 1];
  __shared__ int scan_tmp[NW + 1];
  __shared__ unsigned long long thr;
  __shared__ int nbuf;
  __shared__ uint32_t hist[260];
  const int lane = threadIdx.x & 31;
  const int k = a.k;

  for (int64_t q = blockIdx.x; q < a.nq; q += gridDim.x) {
    __syncthreads();
    {
      const float4* src = reinterpret_cast<const float4*>(a.lut + q * M * KSUB);
      for (int t = threadIdx.x; t < M * KSUB / 4; t += NT) reinterpret_cast<float4*>(lut)[t] = src[t];
    }
    TK tk{bufs, bufs + TK::CAP, &nbuf, &thr, hist};
    if (threadIdx.x == 0) {
      thr = EMPTY;
      nbuf = 0;
    }
    __syncthreads();  // every thread reads nbuf / thr, also when the query has no cells
    const int nc = max(0, a.ncells[q]);
    const bpq_cell* cl = a.cells + q * (int64_t)a.cap;
    for (int cs = 0; cs < nc; cs += CH) {
      const int nch = min(CH, nc - cs);
      int cnt = 0;
      if ((int)threadIdx.x < nch) {
        bpq_cell c = cl[cs + threadIdx.x];
        c_beg[threadIdx.x] = c.begin;
        c_key[threadIdx.x] = c.key;
        if (!POINT) {
          uint32_t i = c.cell / (uint32_t)a.T, j = c.cell % (uint32_t)a.T;
          c_x1[threadIdx.x] = i * M2 * KSUB;
          c_x2[threadIdx.x] = j * M2 * KSUB;
        }
        cnt = (int)c.count;
      }
      int total;
      int ex = block_excl_scan<NT>(cnt, scan_tmp, &total);
      if ((int)threadIdx.x < nch) c_pref[threadIdx.x] = ex;
      if (threadIdx.x == 0) c_pref[nch] = total;
      __syncthreads();
      const int P = total;
      for (int sub = 0; sub < P; sub += SUB) {
        // cell of every candidate of this slice: one search, then a walk
        {
          const int f0 = sub + threadIdx.x * PER;
          if (f0 < P) {
            int c = find_cell(c_pref, nch, f0);
            const int fe = min(P, f0 + PER);
            for (int f = f0; f < fe; ++f) {
              while (c_pref[c + 1] <= f) ++c;
              cmap[f - sub] = (uint8_t)c;
            }
          }
        }
        __syncthreads();
        const int Pe = min(P, sub + SUB);
        uint32_t pos_n[ILP];
        int cid_n[ILP];
        auto issue = [&](int b, int stg) {
#pragma unroll
          for (int u = 0; u < ILP; ++u) {
            const int f = b + u * NT + threadIdx.x;
            cid_n[u] = -1;
            if (f < Pe) {
              const int c = cmap[f - sub];
              cid_n[u] = c;
              pos_n[u] = c_beg[c] + (uint32_t)(f - c_pref[c]);
              cp_async<sizeof(CV)>(sc + (stg * ILP + u) * NT + threadIdx.x, a.codes + (size_t)pos_n[u] * M);
              if (POINT) cp_async<4>(sx + (stg * ILP + u) * NT + threadIdx.x, a.cross + pos_n[u]);
            }
          }
          cp_async_commit();
        };
        int stage = 0;
        issue(sub, 0);
        for (int base = sub; base < Pe; base += NT * ILP) {
          Code<M> code[ILP];
          float pc[ILP];
          int cidx[ILP];
          uint32_t pos[ILP];
#pragma unroll
          for (int u = 0; u < ILP; ++u) {
            cidx[u] = cid_n[u];
            pos[u] = pos_n[u];
          }
          if (base + NT * ILP < Pe) {
            issue(base + NT * ILP, stage ^ 1);
            cp_async_wait<1>();
          } else {
            cp_async_wait<0>();
          }
#pragma unroll
          for (int u = 0; u < ILP; ++u) {
            if (cidx[u] >= 0) {
              const CV v = sc[(stage * ILP + u) * NT + threadIdx.x];
              if constexpr (M == 16) {
                code[u].w[0] = v.x;
                code[u].w[1] = v.y;
                code[u].w[2] = v.z;
                code[u].w[3] = v.w;
              } else {
                code[u].w[0] = v.x;
                code[u].w[1] = v.y;
              }
              if (POINT) pc[u] = sx[(stage * ILP + u) * NT + threadIdx.x];
            }
          }
          stage ^= 1;
          const unsigned long long th = *(volatile unsigned long long*)&thr;
          const uint32_t th_hi = (uint32_t)(th >> 32);
#pragma unroll
          for (int u = 0; u < ILP; ++u) {
            bool acc = false;
            uint64_t comp = 0;
            if (cidx[u] >= 0) {
              const int c = cidx[u];
              float part;
              if (POINT) {
                part = pc[u];
#pragma unroll
                for (int kk = 0; kk < M; ++kk) part += lut[kk * KSUB + code[u].byte(kk)];
              } else {
                part = 0.f;
                const float* x1 = a.X1 + c_x1[c];
                const float* x2 = a.X2 + c_x2[c];
#pragma unroll
                for (int kk = 0; kk < M; ++kk) {
                  const uint32_t b = code[u].byte(kk);
                  const float xv = (kk < M2) ? __ldg(x1 + kk * KSUB + b) : __ldg(x2 + (kk - M2) * KSUB + b);
                  part += lut[kk * KSUB + b] + xv;
                }
              }
              const float dist = c_key[c] + part;
              const uint32_t o = f2ord(dist);
              if (o <= th_hi) {
                comp = ((uint64_t)o << 32) | (uint32_t)__ldg(a.ids + pos[u]);
                acc = comp <= th;
              }
            }
            const unsigned m = __ballot_sync(0xffffffffu, acc);
            if (m) {
              int at = 0;
              if (lane == 0) at = atomicAdd(&nbuf, __popc(m));
              at = __shfl_sync(0xffffffffu, at, 0);
              if (acc) tk.buf[at + __popc(m & lanemask_lt())] = comp;
            }
          }
          __syncthreads();
          if (nbuf > CAP - NT * ILP) block_topk_prune<NT, CAP>(tk, k);
        }
        __syncthreads();
      }
    }
    block_topk_finish<NT, CAP>(tk, k, a.out_ids + q * k, a.out_dists + q * k);
  }
}

// ---------------------------------------------------------------------------
// FBPQ scan, warp-segment form (per-point cross terms, k <= 128).
//
// One CTA per query.  The query's cells are taken in chunks of CH; the
// candidates of a chunk (the concatenation of its cells' list ranges) are split
// into NW contiguous segments, one per warp.  A warp walks its segment 32U
// consecutive candidates per step (U per lane): the cells of the step's
// candidates come from OR-reductions of the cell boundaries that fall inside
// the step's window, and the codes and cross terms of a step are loaded D steps
// ahead into registers (coalesced: consecutive candidates of a cell are
// consecutive list positions).
//
// Top-k: a candidate whose distance passes the block threshold goes to its
// warp's buffer as (ord(distance) << 32 | list position).  A full buffer is cut
// to the entries with distance <= v, a value with at least k entries at or
// below it (a count bisection, stopped once k .. k + 32 remain), and the block
// threshold drops to min(threshold, v): at least k candidates of the query lie
// at or below every warp's v, so no candidate above it can rank, and ties at v
// stay accepted.  At the end the entries within the threshold are gathered, cut
// the same way over the block, given their ids (the only id reads) and ranked
// exactly by (distance, id).
// ---------------------------------------------------------------------------
constexpr uint32_t NO_POS = 0xffffffffu;

// A cut value v for a warp buffer of n entries (k < n <= 256): at least k
// entries have distance bits <= v, and no more than k + 32 unless the bisection
// reaches the exact k-th smallest value first.  Bisection on the distance bits,
// counting with each lane's eight keys held in registers.
__device__ uint32_t warp_cut(const uint64_t* wb, int n, int k) {
  const int lane = threadIdx.x & 31;
  uint32_t h[8];
  uint32_t mn = 0xffffffffu, mx = 0u;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int e = lane + 32 * i;
    h[i] = 0xffffffffu;
    if (e < n) {
      h[i] = (uint32_t)(wb[e] >> 32);
      mn = min(mn, h[i]);
      mx = max(mx, h[i]);
    }
  }
  mn = __reduce_min_sync(0xffffffffu, mn);
  mx = __reduce_max_sync(0xffffffffu, mx);
  // count(<= hi) >= k; count(<= lo) < k (lo = mn - 1 as a 64-bit value)
  long long lo = (long long)mn - 1, hi = mx;
  while (hi - lo > 1) {
    const uint32_t mid = (uint32_t)(lo + ((hi - lo) >> 1));
    int c = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) c += (h[i] <= mid) ? 1 : 0;
    c = warp_sum(c);
    if (c >= k) {
      hi = mid;
      if (c <= k + 32) break;
    } else {
      lo = mid;
    }
  }
  return (uint32_t)hi;
}

// Warp-wide bitonic sort (ascending) of n = power of two 64-bit keys with 32-bit
// payloads in shared memory.
__device__ void warp_bitonic_sort_kv(uint64_t* a, uint32_t* p, int n) {
  const int lane = threadIdx.x & 31;
  for (int size = 2; size <= n; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      __syncwarp();
      for (int t = lane; t < (n >> 1); t += 32) {
        const int lo = 2 * t - (t & (stride - 1)), hi = lo + stride;
        const bool up = (lo & size) == 0;
        const uint64_t x = a[lo], y = a[hi];
        if ((x > y) == up) {
          a[lo] = y;
          a[hi] = x;
          const uint32_t u = p[lo];
          p[lo] = p[hi];
          p[hi] = u;
        }
      }
    }
  }
  __syncwarp();
}

// Cuts a full warp buffer (n entries, k < n <= KW) to the entries with distance
// <= the k-th smallest distance v and lowers the block threshold to v.  If ties
// at v keep more than half the buffer, the buffer is ranked exactly by
// (distance, id) and cut to k.  Returns the new count.
template <int KW>
__device__ int warp_prune(uint64_t* wb, int n, int k, uint32_t* hist, unsigned long long* thr, const int32_t* ids) {
  static_assert(KW == 256, "the cut keeps eight entries per lane");
  const int lane = threadIdx.x & 31;
  uint32_t v = warp_cut(wb, n, k);
  int kept = 0;
  for (int e0 = 0; e0 < n; e0 += 32) {
    const int e = e0 + lane;
    uint64_t x = 0;
    bool keep = false;
    if (e < n) {
      x = wb[e];
      keep = (uint32_t)(x >> 32) <= v;
    }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    __syncwarp();  // this step's entries are read before any is overwritten
    if (keep) wb[kept + __popc(m & lanemask_lt())] = x;
    kept += __popc(m);
  }
  __syncwarp();
  if (kept > KW / 2) {  // a large tie group at v: rank by (distance, id), keep k
    for (int e = lane; e < KW; e += 32) {
      if (e < kept) {
        const uint64_t x = wb[e];
        const uint32_t pos = (uint32_t)x;
        hist[e] = pos;
        wb[e] = (x & 0xffffffff00000000ull) | (uint32_t)__ldg(ids + pos);
      } else {
        wb[e] = EMPTY;
      }
    }
    warp_bitonic_sort_kv(wb, hist, KW);
    for (int e = lane; e < k; e += 32) wb[e] = (wb[e] & 0xffffffff00000000ull) | hist[e];
    kept = k;
    __syncwarp();
    v = (uint32_t)(wb[k - 1] >> 32);
  }
  if (lane == 0) atomicMin(thr, ((unsigned long long)v << 32) | 0xffffffffull);
  __syncwarp();
  return kept;
}

// The block form of warp_cut over a[0..n) (k < n <= 8 * NT): at least k
// entries have distance bits <= the result, and no more than k + 32 unless the
// bisection reaches the exact k-th smallest value first.  `red` holds 2 * NT / 32
// ints (alternating halves, one barrier per count).
template <int NT>
__device__ uint32_t block_cut(const uint64_t* a, int n, int k, int* red) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t h[8];
  uint32_t mn = 0xffffffffu, mx = 0u;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int e = threadIdx.x + NT * i;
    h[i] = 0xffffffffu;
    if (e < n) {
      h[i] = (uint32_t)(a[e] >> 32);
      mn = min(mn, h[i]);
      mx = max(mx, h[i]);
    }
  }
  mn = __reduce_min_sync(0xffffffffu, mn);
  mx = __reduce_max_sync(0xffffffffu, mx);
  if (lane == 0) {
    red[w] = (int)mn;
    red[NW + w] = (int)mx;
  }
  __syncthreads();
#pragma unroll
  for (int x = 0; x < NW; ++x) {
    mn = min(mn, (uint32_t)red[x]);
    mx = max(mx, (uint32_t)red[NW + x]);
  }
  __syncthreads();
  long long lo = (long long)mn - 1, hi = mx;
  int par = 0;
  while (hi - lo > 1) {
    const uint32_t mid = (uint32_t)(lo + ((hi - lo) >> 1));
    int c = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) c += (h[i] <= mid) ? 1 : 0;
    c = warp_sum(c);
    if (lane == 0) red[par * NW + w] = c;
    __syncthreads();
    c = 0;
#pragma unroll
    for (int x = 0; x < NW; ++x) c += red[par * NW + x];
    par ^= 1;
    if (c >= k) {
      hi = mid;
      if (c <= k + 32) break;
    } else {
      lo = mid;
    }
  }
  return (uint32_t)hi;
}

// Shortlists (bpq_search_shortlist): the S best (score, list position) composites
// of a query.  S is up to 1024, more than a warp buffer holds, so the warps move
// their buffered entries into one block buffer of BBC entries, one warp at a
// time (a lock in shared memory); when it nears its capacity that warp cuts it
// to the entries at or below a value v with at least S entries <= v (sl_cut_value:
// a sampled guess checked by one count, else a count bisection) and lowers the
// block threshold to (v, any position).  If a tie group at v still fills the
// buffer, the cut is exact on the whole composite.

// Entries of bb[0 .. n) with bits <= v kept in place (v on the whole composite
// when `whole`, else on the score bits).  Warp-wide; returns the new count.
__device__ int sl_compact(uint64_t* bb, int n, uint64_t v, bool whole) {
  const int lane = threadIdx.x & 31;
  int kept = 0;
  for (int e0 = 0; e0 < n; e0 += 32) {
    const int e = e0 + lane;
    uint64_t x = 0;
    bool keep = false;
    if (e < n) {
      x = bb[e];
      keep = whole ? x <= v : (x >> 32) <= v;
    }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    __syncwarp();  // this step's entries are read before any is overwritten
    if (keep) bb[kept + __popc(m & lanemask_lt())] = x;
    kept += __popc(m);
  }
  __syncwarp();
  return kept;
}

// Number of entries of bb[0 .. n) with score bits <= hi (hi_eq: == hi) and
// position bits <= lo_max.  Warp-wide.
__device__ int sl_count(const uint64_t* bb, int n, uint32_t hi, bool hi_eq, long long lo_max) {
  const int lane = threadIdx.x & 31;
  int c = 0;
  for (int e = lane; e < n; e += 32) {
    const uint64_t x = bb[e];
    const uint32_t h = (uint32_t)(x >> 32);
    c += ((hi_eq ? h == hi : h <= hi) && (long long)(uint32_t)x <= lo_max) ? 1 : 0;
  }
  return warp_sum(c);
}

// Bitonic sort (ascending) of 256 keys held by one warp, eight per lane (element
// lane * 8 + i in x[i]); pairs closer than 8 are in the same lane, farther pairs
// are exchanged with shuffles.
__device__ __forceinline__ void warp_sort256(uint32_t (&x)[8]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int size = 2; size <= 256; size <<= 1) {
#pragma unroll
    for (int j = size >> 1; j > 0; j >>= 1) {
      if (j < 8) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int p = i ^ j;
          if (p > i) {
            const bool up = (((lane * 8 + i) & size) == 0);
            const uint32_t a = x[i], b = x[p];
            const bool sw = (a > b) == up;
            x[i] = sw ? b : a;
            x[p] = sw ? a : b;
          }
        }
      } else {
        const int lj = j / 8;
        const bool lower = (lane & lj) == 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const uint32_t o = __shfl_xor_sync(0xffffffffu, x[i], lj);
          const bool up = (((lane * 8 + i) & size) == 0);
          x[i] = (lower == up) ? min(x[i], o) : max(x[i], o);
        }
      }
    }
  }
}

// The cut of a full block buffer (n > S entries): a score value v with
// S <= count(<= v) and, unless a tie group at v is larger, count(<= v) <= keep.
// A guess from a sorted sample of 256 entries (aimed at S + 96 entries) is
// checked with one count; a guess outside [S, keep] is refined by bisection
// between it and the buffer's extreme.
__device__ __noinline__ uint32_t sl_cut_value(const uint64_t* bb, int n, int S, int keep) {
  const int lane = threadIdx.x & 31;
  uint32_t x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = (uint32_t)(bb[(int)(((long long)(lane * 8 + i) * n) >> 8)] >> 32);
  warp_sort256(x);
  const int r = min(255, (int)(((long long)(S + 96) * 256 + n - 1) / n));
  const uint32_t g = __shfl_sync(0xffffffffu, x[r & 7], r >> 3);
  const int cg = sl_count(bb, n, g, false, 0xffffffffll);
  if (cg >= S && cg <= keep) return g;
  long long lo, hi;  // count(<= hi) >= S > count(<= lo)
  if (cg < S) {
    uint32_t mx = 0u;
    for (int e = lane; e < n; e += 32) mx = max(mx, (uint32_t)(bb[e] >> 32));
    mx = __reduce_max_sync(0xffffffffu, mx);
    lo = g;
    hi = mx;
  } else {
    uint32_t mn = 0xffffffffu;
    for (int e = lane; e < n; e += 32) mn = min(mn, (uint32_t)(bb[e] >> 32));
    mn = __reduce_min_sync(0xffffffffu, mn);
    lo = (long long)mn - 1;
    hi = g;
  }
  while (hi - lo > 1) {
    const uint32_t mid = (uint32_t)(lo + ((hi - lo) >> 1));
    const int c = sl_count(bb, n, mid, false, 0xffffffffll);
    if (c >= S) {
      hi = mid;
      if (c <= keep) break;
    } else {
      lo = mid;
    }
  }
  return (uint32_t)hi;
}

template <int KW, int BBC>
__device__ void sl_flush(const uint64_t* wb, int wn, int S, uint64_t* bb, int* bb_n, int* lock,
                         unsigned long long* thr, int32_t* status) {
  const int lane = threadIdx.x & 31;
  int ok = 1;
  if (lane == 0) {
    long long spins = 0;
    while (atomicCAS(lock, 0, 1) != 0) {
      if (++spins > (1ll << 24)) {  // never expected: the holder is a warp of this CTA doing bounded work
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (!ok) {
    if (lane == 0 && status) atomicOr(status, STATUS_TIMEOUT);
    __syncwarp();
    return;
  }
  __threadfence_block();
  const unsigned long long th = *(volatile unsigned long long*)thr;
  int n = *(volatile int*)bb_n;
  for (int e0 = 0; e0 < wn; e0 += 32) {
    const int e = e0 + lane;
    const uint64_t x = e < wn ? wb[e] : EMPTY;
    const bool keep = e < wn && x <= th;
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    if (keep) bb[n + __popc(m & lanemask_lt())] = x;
    n += __popc(m);
  }
  __syncwarp();
  if (n > BBC - KW) {
    // keep at most half of the room above S, so that the next cut is some flushes away
    const uint32_t v = sl_cut_value(bb, n, S, S + (BBC - KW - S) / 2);
    unsigned long long nt = ((unsigned long long)v << 32) | 0xffffffffull;
    if (sl_count(bb, n, v, false, 0xffffffffll) > BBC - KW) {
      // a tie group at v: the exact S-th composite, bisecting the positions at v
      const int need = S - (v > 0 ? sl_count(bb, n, v - 1, false, 0xffffffffll) : 0);
      long long plo = -1, phi = 0xffffffffll;  // count(pos <= phi) >= need > count(pos <= plo)
      while (phi - plo > 1) {
        const long long mid = plo + ((phi - plo) >> 1);
        if (sl_count(bb, n, v, true, mid) >= need) phi = mid; else plo = mid;
      }
      nt = ((unsigned long long)v << 32) | (uint32_t)phi;
      n = sl_compact(bb, n, nt, true);
    } else {
      n = sl_compact(bb, n, v, false);
    }
    if (lane == 0 && nt < *(volatile unsigned long long*)thr) *(volatile unsigned long long*)thr = nt;
  }
  if (lane == 0) *(volatile int*)bb_n = n;
  __threadfence_block();
  __syncwarp();
  if (lane == 0) atomicExch(lock, 0);
}

// HB = true: the same scan for HBPQ's table form (§3.2): a candidate of cell (i, j)
// costs the M lookups key(i, j) + sum_k A_i[k][c_k] + sum_k B_j[k][c_{M/2+k}] into
// the per-(query, half-cell) tables built by the HBPQ table kernel (read through
// the cache from global memory; the table slots of the query come from its row
// and column bitmaps), and no cross term is read.
//
// RV = FB_Q8 / FB_F16: the shortlist scan (the reduced-precision table and score
// described with the variants above), with a block buffer of BBC entries (BBC - KW
// >= S + 32; a small one for short shortlists keeps eight CTAs per SM); the S best
// composites go to a.sl_out in any order.
template <int M, int NT, int D, int U, int KW, int CH, bool HB, bool WQ, int RV, int BBC>
__global__ void __launch_bounds__(NT, HB ? 5 : 8) fbpq_scan_seg_kernel(ScanArgs a) {
  constexpr int NW = NT / 32, R = CH / NT, M2 = M / 2;
  constexpr bool RED = RV == FB_Q8 || RV == FB_F16;
  static_assert(CH % NT == 0 && (KW == 256 || (RED && KW >= 64)),
                "shape (the exact prune keeps its payloads in the warp's 256 counters)");
  static_assert(RV == FB_POINT || (RED && !HB && !WQ && BBC > KW), "variant");
  static_assert(RED || BBC == 0, "the block buffer is the shortlists'");
  // the final sort pads the at most BBC - KW entries to the next power of two in place
  static_assert(BBC == 0 || (BBC & (BBC - 1)) == 0, "the block buffer's size is a power of two");
  // the query's table: FP32 (FBPQ), int8 or FP16 (shortlists); none (HB)
  constexpr int AREA0 = HB ? 0 : M * KSUB * (RV == FB_Q8 ? 1 : (RV == FB_F16 ? 2 : 4));
  constexpr int TWMAX = MAX_T / 32;
  using CV = CodeVec<M>;
  extern __shared__ __align__(16) unsigned char smem[];
  float* lut = reinterpret_cast<float*>(smem);                    // M x 256 (FBPQ)
  uint32_t* hbits = reinterpret_cast<uint32_t*>(smem + AREA0);    // HB: 2 x TWMAX row / column bitmap words
  int* hpre = reinterpret_cast<int*>(hbits + (HB ? 2 * TWMAX : 0));  // HB: 2 x TWMAX bits below each word
  uint64_t* wbuf = reinterpret_cast<uint64_t*>(hpre + (HB ? 2 * TWMAX : 0));  // NW x KW
  uint32_t* whist = reinterpret_cast<uint32_t*>(wbuf + NW * KW);  // NW x 256 (not the shortlists')
  int2* c_info = reinterpret_cast<int2*>(whist + (RED ? 0 : NW * 256));  // CH: (begin - first candidate, key bits)
  int* c_pref = reinterpret_cast<int*>(c_info + CH);              // CH + 1: first candidate of each cell
  uint2* c_tab = reinterpret_cast<uint2*>(c_pref + CH + 2);       // HB, CH: table offsets (A_i, B_j) in floats
  uint64_t* bb = reinterpret_cast<uint64_t*>(c_pref + CH + 2);    // RED, BBC: shortlist block buffer
  __shared__ int bb_n, bb_lock;
  __shared__ int scan_tmp[NW + 1];
  __shared__ int cut_red[2 * NW];
  __shared__ int fcount;
  __shared__ unsigned long long thr;
  __shared__ int64_t s_item;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int k = a.k;
  uint64_t* wb = wbuf + w * KW;
  uint32_t* hist = whist + w * 256;
  const char* lutb = reinterpret_cast<const char*>(lut);

  // One unit of work per iteration: a whole query (CTAs strided over the queries),
  // or with WQ a work item (q, cells c_lo .. c_hi - 1, partial slot) taken from
  // the queue (persistent CTAs); a split query's items write partial top-k lists
  // that merge_parts_kernel combines.
  for (int64_t iter = blockIdx.x;; iter += gridDim.x) {
    __syncthreads();  // the previous unit's final list (in the table area) is written out
    int64_t q, out_row;
    int c_lo = 0, c_hi;
    bool part = false;
    if constexpr (WQ) {
      if (threadIdx.x == 0) s_item = atomicAdd(a.item_counter, 1);
      __syncthreads();
      const int64_t it = s_item;
      if (it >= *a.n_items) break;
      const int4 itm = a.items[it];
      q = itm.x;
      c_lo = itm.y;
      c_hi = itm.z;
      part = itm.w >= 0;
      out_row = part ? itm.w : q;
    } else {
      if (a.sel) {
        if (iter >= *a.sel_n) break;
        q = a.sel[iter];
      } else {
        if (iter >= a.nq) break;
        q = iter;
        if (a.skip && a.skip[q]) continue;  // uniform across the CTA
      }
      c_hi = max(0, a.ncells[q]);
      out_row = q;
    }
    int32_t* o_ids = (part ? a.part_ids : a.out_ids) + out_row * k;
    float* o_dists = (part ? a.part_dists : a.out_dists) + out_row * k;
    int hb_base = 0, hb_rows = 0, TW = 0;
    if constexpr (HB) {
      hb_base = a.hb_qbase[q];
      if (hb_base < 0) continue;  // its tables did not fit: scored by the reconstruction fallback
      hb_rows = a.hb_qrows[q];
      TW = (a.T + 31) >> 5;
      const uint32_t* qb = a.hb_qbits + q * 2 * TW;
      for (int x = threadIdx.x; x < 2 * TW; x += NT) hbits[x] = qb[x];
      __syncthreads();
      for (int x = threadIdx.x; x < 2 * TW; x += NT) {
        const int h0 = x >= TW ? TW : 0;
        int p = 0;
        for (int y = h0; y < x; ++y) p += __popc(hbits[y]);
        hpre[x] = p;
      }
    } else {
      const uint4* src = RV == FB_Q8    ? reinterpret_cast<const uint4*>(a.lut8 + q * M * KSUB)
                         : RV == FB_F16 ? reinterpret_cast<const uint4*>(a.lut16 + q * M * KSUB)
                                        : reinterpret_cast<const uint4*>(a.lut + q * M * KSUB);
      for (int t = threadIdx.x; t < AREA0 / 16; t += NT) reinterpret_cast<uint4*>(lut)[t] = src[t];
    }
    const float scale = RED ? a.lut_scale[q] : 0.f;
    if (threadIdx.x == 0) {
      thr = EMPTY;
      bb_n = 0;
      bb_lock = 0;
    }
    int wn = 0;  // entries in this warp's buffer (uniform across the warp)
    const bpq_cell* cl = a.cells + q * (int64_t)a.cap;
    for (int cs = c_lo; cs < c_hi; cs += CH) {
      const int nch = min(CH, c_hi - cs);
      // first candidate of each cell of the chunk (thread t takes cells
      // tR .. tR + R - 1; the second read of a cell hits the cache)
      int loc = 0;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int t = threadIdx.x * R + r;
        if (t < nch) loc += (int)cl[cs + t].count;
      }
      __syncthreads();  // the previous chunk's cells are no longer read
      int total;
      int run = block_excl_scan<NT>(loc, scan_tmp, &total);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int t = threadIdx.x * R + r;
        if (t < nch) {
          const bpq_cell cc = cl[cs + t];
          c_pref[t] = run;
          c_info[t] = make_int2((int)cc.begin - run, __float_as_int(cc.key));
          if constexpr (HB) {
            const uint32_t i = cc.cell / (uint32_t)a.T, j = cc.cell - i * (uint32_t)a.T;
            const int ri = hpre[i >> 5] + __popc(hbits[i >> 5] & ((1u << (i & 31)) - 1u));
            const int rj = hpre[TW + (j >> 5)] + __popc(hbits[TW + (j >> 5)] & ((1u << (j & 31)) - 1u));
            c_tab[t] = make_uint2((uint32_t)(hb_base + ri) * (uint32_t)(M2 * KSUB),
                                  (uint32_t)(hb_base + hb_rows + rj) * (uint32_t)(M2 * KSUB));
          }
          run += (int)cc.count;
        }
      }
      if (threadIdx.x == 0) c_pref[nch] = total;
      __syncthreads();
      const int P = total;
      // FBPQ: each warp walks one contiguous quarter of the chunk.  HB: the warps
      // take the windows of 32U candidates in turn, so the CTA's warps work in the
      // same few cells at a time and their table lookups share the L1 cache.
      constexpr int WSTEP = HB ? NW : 1;
      const int s = HB ? 32 * U * w : (int)(((long long)P * w) / NW);
      const int e = HB ? P : (int)(((long long)P * (w + 1)) / NW);
      if (s < e) {
        int c = find_cell(c_pref, nch, s);  // cell of the next step's first candidate
        int f = s;                          // next step's first candidate
        const unsigned le = (2u << lane) - 1u;
        uint32_t spos[D][U];
        float skey[D][U], sx[D][U];
        int scl[D][U];
        CV scode[D][U];
        // a step: candidates f + 32u + lane (u < U); the cell starts that fall in
        // half h of the window [f, f + 32U) set bits of msk[h]
        auto issue = [&](int d) {
#pragma unroll
          for (int u = 0; u < U; ++u) spos[d][u] = NO_POS;
          if (f < e) {
            if constexpr (HB) c = find_cell(c_pref, nch, f);
            unsigned bits[U];
#pragma unroll
            for (int h = 0; h < U; ++h) bits[h] = 0u;
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int i = c + 1 + 32 * u + lane;
              const int o = (i <= nch ? c_pref[i] : 0x7fffffff) - f;  // >= 1 + 32u
              const int hh = o >> 5;  // the window half the boundary falls in (>= U: none)
              const unsigned bit = 1u << (o & 31);
#pragma unroll
              for (int h = u; h < U; ++h) bits[h] |= (hh == h) ? bit : 0u;
            }
            int below = c;
#pragma unroll
            for (int h = 0; h < U; ++h) {
              const unsigned msk = __reduce_or_sync(0xffffffffu, bits[h]);
              const int fl = f + 32 * h + lane;
              if (fl < e) {
                const int cell = below + __popc(msk & le);
                const int2 inf = c_info[cell];
                const uint32_t pos = (uint32_t)(fl + inf.x);
                spos[d][h] = pos;
                skey[d][h] = __int_as_float(inf.y);
                scode[d][h] = __ldg(reinterpret_cast<const CV*>(a.codes) + pos);
                if constexpr (HB)
                  scl[d][h] = cell;
                else
                  sx[d][h] = __ldg(a.cross + pos);
              }
              below += __popc(msk);
            }
            c = below;
            if (c + 1 <= nch && c_pref[c + 1] == f + 32 * U) ++c;
            f += 32 * U * WSTEP;
          }
        };
#pragma unroll
        for (int d = 0; d < D; ++d) issue(d);
        for (int left = (e - s + 32 * U * WSTEP - 1) / (32 * U * WSTEP); left > 0; left -= D) {
          const unsigned long long th = *(volatile unsigned long long*)&thr;
          const uint32_t th_hi = (uint32_t)(th >> 32);
#pragma unroll
          for (int d = 0; d < D; ++d) {
            uint32_t o[U];
            bool acc[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
              acc[u] = false;
              o[u] = 0;
              if (spos[d][u] != NO_POS) {
                float part = (HB || RED) ? 0.f : sx[d][u];
                uint32_t wd[M / 4];
                if constexpr (M == 16) {
                  wd[0] = scode[d][u].x;
                  wd[1] = scode[d][u].y;
                  wd[2] = scode[d][u].z;
                  wd[3] = scode[d][u].w;
                } else {
                  wd[0] = scode[d][u].x;
                  wd[1] = scode[d][u].y;
                }
                if constexpr (HB) {
                  const uint2 tb = c_tab[scl[d][u]];
#pragma unroll
                  for (int kk = 0; kk < M; ++kk) {
                    const uint32_t c = (wd[kk >> 2] >> (8 * (kk & 3))) & 0xffu;
                    part += __ldg(a.hb_tables + (kk < M2 ? tb.x : tb.y) + (kk % M2) * KSUB + c);
                  }
                } else if constexpr (RV == FB_Q8) {
                  int isum = 0;  // exact integer sum of the int8 entries
#pragma unroll
                  for (int kk = 0; kk < M; ++kk)
                    isum += (int)*reinterpret_cast<const uint8_t*>(lutb + kk * KSUB + ((wd[kk >> 2] >> (8 * (kk & 3))) & 0xffu));
                  part = __fmul_rn(scale, (float)isum);
                } else if constexpr (RV == FB_F16) {
                  float hs = 0.f;  // FP32 additions in sub-quantizer order
#pragma unroll
                  for (int kk = 0; kk < M; ++kk) {
                    const uint32_t off = ((wd[kk >> 2] >> (8 * (kk & 3))) & 0xffu) << 1;
                    hs = __fadd_rn(hs, __half2float(*reinterpret_cast<const __half*>(lutb + kk * (KSUB * 2) + off)));
                  }
                  part = __fmul_rn(scale, hs);
                } else {
#pragma unroll
                  for (int kk = 0; kk < M; ++kk) {
                    const uint32_t off = ((wd[kk >> 2] >> (8 * (kk & 3))) & 0xffu) << 2;
                    part += *reinterpret_cast<const float*>(lutb + kk * (KSUB * 4) + off);
                  }
                }
                if constexpr (RED) {  // (key + cross) + s * part, that order, no fused multiply-add
                  o[u] = f2ord(__fadd_rn(__fadd_rn(skey[d][u], sx[d][u]), part));
                  acc[u] = (((uint64_t)o[u] << 32) | spos[d][u]) <= th;
                } else {
                  o[u] = f2ord(skey[d][u] + part);
                  acc[u] = o[u] <= th_hi;
                }
              }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const unsigned m = __ballot_sync(0xffffffffu, acc[u]);
              if (m) {
                if (acc[u]) wb[wn + __popc(m & lanemask_lt())] = ((uint64_t)o[u] << 32) | spos[d][u];
                wn += __popc(m);
                if (wn > KW - 32) {
                  __syncwarp();
                  if constexpr (RED) {
                    sl_flush<KW, BBC>(wb, wn, k, bb, &bb_n, &bb_lock, &thr, a.status);
                    wn = 0;
                  } else {
                    wn = warp_prune<KW>(wb, wn, k, hist, &thr, a.ids);
                  }
                }
              }
            }
            issue(d);
          }
        }
      }
    }
    if constexpr (RED) {
      // final (shortlist): the last entries of every warp into the block buffer
      // (it then holds at most BBC - KW), sorted when more than S: the S smallest
      // composites are the shortlist
      if (wn > 0) sl_flush<KW, BBC>(wb, wn, k, bb, &bb_n, &bb_lock, &thr, a.status);
      __syncthreads();
      const int n = bb_n;
      uint64_t* out = a.sl_out + out_row * k;
      if (n > k) {
        int n2 = 1;
        while (n2 < n) n2 <<= 1;
        for (int x = n + threadIdx.x; x < n2; x += NT) bb[x] = EMPTY;
        block_bitonic_sort(bb, n2);
      }
      for (int r = threadIdx.x; r < k; r += NT) out[r] = r < n ? bb[r] : EMPTY;
      continue;
    } else {
    // final: the entries within the block threshold are gathered into the table
    // area (it holds every buffer), cut near the k best distances, given their
    // ids (read only here) and ranked exactly by (distance, id)
    static_assert(NW * KW * 8 <= (HB ? CH * 8 + (CH + 2) * 4 + CH * 8 : AREA0),
                  "the final area holds every buffered entry");
    __syncthreads();
    const uint32_t th_hi = (uint32_t)(thr >> 32);
    int mine = 0;
    for (int e0 = 0; e0 < wn; e0 += 32) {
      const int e = e0 + lane;
      mine += __popc(__ballot_sync(0xffffffffu, e < wn && (uint32_t)(wb[e] >> 32) <= th_hi));
    }
    if (lane == 0) scan_tmp[w] = mine;
    if (threadIdx.x == 0) fcount = 0;
    __syncthreads();
    int base = 0, n = 0;
#pragma unroll
    for (int x = 0; x < NW; ++x) {
      base += (x < w) ? scan_tmp[x] : 0;
      n += scan_tmp[x];
    }
    // the table (FBPQ) or the chunk's cell arrays (HB) are no longer read
    uint64_t* fin = HB ? reinterpret_cast<uint64_t*>(c_info) : reinterpret_cast<uint64_t*>(lut);
    for (int e0 = 0; e0 < wn; e0 += 32) {
      const int e = e0 + lane;
      const uint64_t x = e < wn ? wb[e] : EMPTY;
      const bool keep = e < wn && (uint32_t)(x >> 32) <= th_hi;
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (keep) fin[base + __popc(m & lanemask_lt())] = x;
      base += __popc(m);
    }
    __syncthreads();
    const uint32_t v = (n > k) ? block_cut<NT>(fin, n, k, cut_red) : 0xffffffffu;
    for (int t = threadIdx.x; t < n; t += NT) {
      const uint64_t x = fin[t];
      if ((uint32_t)(x >> 32) <= v)
        wbuf[atomicAdd(&fcount, 1)] = (x & 0xffffffff00000000ull) | (uint32_t)__ldg(a.ids + (uint32_t)x);
    }
    __syncthreads();
    const int m = fcount;
    for (int t = threadIdx.x; t < m; t += NT) {  // rank among the survivors; equal composites (a
      const uint64_t x = wbuf[t];                 // point added twice under one id) by position
      int r = 0;
      for (int j = 0; j < m; ++j) r += (wbuf[j] < x || (wbuf[j] == x && j < t)) ? 1 : 0;
      if (r < k) {
        o_ids[r] = (int32_t)(uint32_t)x;
        o_dists[r] = ord2f((uint32_t)(x >> 32));
      }
    }
    for (int r = m + threadIdx.x; r < k; r += NT) {
      o_ids[r] = -1;
      o_dists[r] = __int_as_float(0x7f800000);
    }
    }
  }
}

// ---------------------------------------------------------------------------
// Work items for the persistent scan: one warp per query cuts its visited cells
// into contiguous ranges of about W candidates (cell c goes to range
// floor(start_c / W'), start_c = the candidates before it, W' = max(W,
// ceil(P / MAX_ITEMS)) for a query of P candidates), so that no unit of work is
// much longer than W and the queue finishes evenly whatever the budgets.  A query
// of one range writes its final list; a split query's ranges write partial
// lists in consecutive slots and the query is listed for the merge.
// ---------------------------------------------------------------------------
constexpr int MAX_ITEMS = SCAN_MAX_ITEMS;

__global__ void __launch_bounds__(128) build_items_kernel(ScanArgs a, int32_t W) {
  __shared__ int bnd_s[4][MAX_ITEMS + 1];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t q = (int64_t)blockIdx.x * 4 + w;
  if (q >= a.nq) return;  // uniform over the warp
  if (a.hb_qbase && a.hb_qbase[q] < 0) return;  // scored by the HBPQ fallback
  const int nc = max(0, a.ncells[q]);
  const bpq_cell* cl = a.cells + q * (int64_t)a.cap;
  long long P = 0;
  for (int c = lane; c < nc; c += 32) P += cl[c].count;
  P = warp_sum(P);
  const long long Wq = max((long long)W, (P + MAX_ITEMS - 1) / MAX_ITEMS);
  int* bnd = bnd_s[w];  // first cell of each range
  int nb = 0;
  long long run = 0;
  int prev_j = -1;
  for (int c0 = 0; c0 < nc; c0 += 32) {
    const int c = c0 + lane;
    const long long cnt = c < nc ? (long long)cl[c].count : 0;
    long long incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const long long start = run + incl - cnt;
    const int j = c < nc ? (int)(start / Wq) : -1;
    const int jp = __shfl_up_sync(0xffffffffu, j, 1);
    const bool first = c < nc && (lane == 0 ? j != prev_j : j != jp);
    const unsigned m = __ballot_sync(0xffffffffu, first);
    if (first) bnd[nb + __popc(m & lanemask_lt())] = c;
    nb += __popc(m);
    prev_j = __shfl_sync(0xffffffffu, j, 31);
    run += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (nb == 0) bnd[nb++] = 0;  // a query without cells: one (empty) range pads its output
  __syncwarp();
  int base = 0, slot0 = -1;
  if (lane == 0) {
    base = atomicAdd(a.n_items, nb);
    if (nb > 1) {
      slot0 = atomicAdd(a.part_counter, nb);
      a.merges[atomicAdd(a.n_merges, 1)] = make_int4((int)q, slot0, nb, 0);
    }
  }
  base = __shfl_sync(0xffffffffu, base, 0);
  slot0 = __shfl_sync(0xffffffffu, slot0, 0);
  for (int b = lane; b < nb; b += 32)
    a.items[base + b] = make_int4((int)q, bnd[b], b + 1 < nb ? bnd[b + 1] : max(nc, 0), nb > 1 ? slot0 + b : -1);
}

// The k best (distance, id) of a split query's partial lists (all sorted, each
// the exact k best of its range), ascending; equal entries (a point added twice
// under one id) stay adjacent and both count.
__global__ void __launch_bounds__(256) merge_parts_kernel(ScanArgs a) {
  __shared__ uint64_t buf[MAX_ITEMS * 128];
  for (int64_t r = blockIdx.x; r < *a.n_merges; r += gridDim.x) {
    __syncthreads();
    const int4 mg = a.merges[r];
    const int q = mg.x, slot0 = mg.y, nb = mg.z, k = a.k;
    const int n = nb * k;
    int n2 = 64;
    while (n2 < n) n2 <<= 1;
    for (int e = threadIdx.x; e < n2; e += 256) {
      uint64_t x = EMPTY;
      if (e < n) {
        const int32_t id = a.part_ids[(int64_t)slot0 * k + e];
        if (id >= 0) x = ((uint64_t)f2ord(a.part_dists[(int64_t)slot0 * k + e]) << 32) | (uint32_t)id;
      }
      buf[e] = x;
    }
    block_bitonic_sort(buf, n2);
    for (int e = threadIdx.x; e < k; e += 256) {
      const uint64_t x = buf[e];
      a.out_ids[(int64_t)q * k + e] = x == EMPTY ? -1 : (int32_t)(uint32_t)x;
      a.out_dists[(int64_t)q * k + e] = x == EMPTY ? __int_as_float(0x7f800000) : ord2f((uint32_t)(x >> 32));
    }
  }
}

// ---------------------------------------------------------------------------
// Exact re-score of a shortlist (bpq_search_shortlist step 3): one CTA per
// query; each shortlisted list position finds its cell by binary search on the
// offsets, then its FBPQ distance (Eqs. 8-9) is formed exactly as in the FP32
// scan: key(i, j) + (cross(p) + lut[0][c_0] + ... + lut[M-1][c_{M-1}]).
// ---------------------------------------------------------------------------
template <int M>
__global__ void __launch_bounds__(256) rescore_kernel(RescoreArgs r) {
  constexpr int NT = 256, G = 4;
  __shared__ __align__(16) float lut[M * KSUB];
  __shared__ uint64_t buf[MAX_K];
  int n2 = 1;
  while (n2 < r.S) n2 <<= 1;
  for (int64_t q = blockIdx.x; q < r.nq; q += gridDim.x) {
    __syncthreads();  // the previous query's list is written out
    const float4* src = reinterpret_cast<const float4*>(r.lut + q * M * KSUB);
    for (int t = threadIdx.x; t < M * KSUB / 4; t += NT) reinterpret_cast<float4*>(lut)[t] = src[t];
    __syncthreads();
    // four shortlisted positions per thread at a time; the cell of each (the last
    // cell with offsets[cell] <= pos) is searched between the two hints around it,
    // the four searches in lockstep so that their dependent loads overlap
    for (int e0 = threadIdx.x; e0 < n2; e0 += G * NT) {
      uint32_t pos[G], lo[G], hi[G];
      bool ok[G];
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int e = e0 + g * NT;
        const uint64_t s = e < r.S ? r.sl[q * r.S + e] : EMPTY;
        ok[g] = s != EMPTY;
        pos[g] = (uint32_t)s;
        lo[g] = ok[g] ? __ldg(r.hint + (pos[g] >> 8)) : 0u;
        hi[g] = ok[g] ? __ldg(r.hint + (pos[g] >> 8) + 1) + 1u : 1u;
      }
      for (int step = 0; step < 32; ++step) {
        bool more = false;
#pragma unroll
        for (int g = 0; g < G; ++g) {
          if (hi[g] - lo[g] > 1) {
            const uint32_t mid = lo[g] + ((hi[g] - lo[g]) >> 1);
            if (__ldg(r.offsets + mid) <= pos[g]) lo[g] = mid; else hi[g] = mid;
            more = true;
          }
        }
        if (!more) break;
      }
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const int e = e0 + g * NT;
        if (e >= n2) continue;
        uint64_t x = EMPTY;
        if (ok[g]) {
          const uint32_t i = lo[g] / (uint32_t)r.T, j = lo[g] % (uint32_t)r.T;
          const float key = __fadd_rn(r.d1[q * r.T + i], r.d2[q * r.T + j]);
          Code<M> code;
          code.load(r.codes, pos[g]);
          float part = __ldg(r.cross + pos[g]);
#pragma unroll
          for (int kk = 0; kk < M; ++kk) part += lut[kk * KSUB + code.byte(kk)];
          x = ((uint64_t)f2ord(key + part) << 32) | (uint32_t)__ldg(r.ids + pos[g]);
        }
        buf[e] = x;
      }
    }
    block_bitonic_sort(buf, n2);  // (distance, id) order; the padding sorts last
    for (int t = threadIdx.x; t < r.k; t += NT) {
      const uint64_t x = buf[t];
      r.out_ids[q * r.k + t] = x == EMPTY ? -1 : (int32_t)(uint32_t)x;
      r.out_dists[q * r.k + t] = x == EMPTY ? __int_as_float(0x7f800000) : ord2f((uint32_t)(x >> 32));
    }
  }
}

// hint[b] = the last cell c with offsets[c] <= min(256 b, n - 1)
__global__ void position_hint_kernel(const uint32_t* __restrict__ offsets, int64_t ncells, int64_t n,
                                     int64_t nb, uint32_t* __restrict__ hint) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b > nb) return;
  const uint32_t x = (uint32_t)min(b * 256, n - 1);
  int64_t lo = 0, hi = ncells;
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (offsets[mid] <= x) lo = mid; else hi = mid;
  }
  hint[b] = (uint32_t)lo;
}

// ---------------------------------------------------------------------------
// Reconstruction scans (Multi-D-ADC and HBPQ): persistent CTAs, one query at a
// time per CTA.
// ---------------------------------------------------------------------------
// RG: the global codebooks R are read through the cache instead of being staged
// in shared memory (when they do not fit it, e.g. D/M = 48).
template <int M, int SUB, int KP, int NW, bool LOCAL, bool RG>
__global__ void __launch_bounds__(NW * 32) recon_scan_kernel(ScanArgs a) {
  constexpr int NT = NW * 32, D = M * SUB, H = D / 2, M2 = M / 2, CHR = 32, ILP = 2;
  constexpr int RS = SUB + 1;  // padded codeword stride
  constexpr int QS = D + 1;    // padded displacement stride
  using TK = WarpTopK<KP>;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* areas = reinterpret_cast<uint64_t*>(smem);
  float* rq = reinterpret_cast<float*>(areas + NW * TK::AREA);  // CHR x QS
  float* Rs = rq + CHR * QS;                                     // M x 256 x RS (global codebooks)
  __shared__ uint32_t c_beg[CHR];
  __shared__ uint32_t c_i[CHR];
  __shared__ uint32_t c_j[CHR];
  __shared__ int c_pref[CHR + 1];
  __shared__ int scan_tmp[NW + 1];
  __shared__ unsigned long long thr;
  __shared__ int64_t q_s;
  const int warp = threadIdx.x >> 5;
  const int k = a.k;
  if (!LOCAL && !RG) {
    for (int t = threadIdx.x; t < M * KSUB * SUB; t += NT) {
      const int row = t / SUB, d = t % SUB;
      Rs[row * RS + d] = a.R[t];
    }
  }
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      const int64_t t = atomicAdd(a.qcounter, 1);
      q_s = a.qlist ? (t < *a.qlist_n ? (int64_t)a.qlist[t] : a.nq) : t;
    }
    __syncthreads();
    const int64_t q = q_s;
    if (q >= a.nq) break;
    const float* qv = a.queries + q * D;
    TK tk;
    tk.init(areas + warp * TK::AREA);
    if (threadIdx.x == 0) thr = EMPTY;
    const int nc = max(0, a.ncells[q]);
    const bpq_cell* cl = a.cells + q * (int64_t)a.cap;
    for (int cs = 0; cs < nc; cs += CHR) {
      const int nch = min(CHR, nc - cs);
      int cnt = 0;
      if ((int)threadIdx.x < nch) {
        bpq_cell c = cl[cs + threadIdx.x];
        c_beg[threadIdx.x] = c.begin;
        c_i[threadIdx.x] = c.cell / (uint32_t)a.T;
        c_j[threadIdx.x] = c.cell % (uint32_t)a.T;
        cnt = (int)c.count;
      }
      int total;
      int ex = block_excl_scan<NT>(cnt, scan_tmp, &total);
      if ((int)threadIdx.x < nch) c_pref[threadIdx.x] = ex;
      __syncthreads();
      // query displacement from each cell centroid: q - [c^1_i; c^2_j]
      for (int t = threadIdx.x; t < nch * D; t += NT) {
        const int c = t / D, d = t % D;
        const float cen = (d < H) ? a.C1[(int64_t)c_i[c] * H + d] : a.C2[(int64_t)c_j[c] * H + d - H];
        rq[c * QS + d] = qv[d] - cen;
      }
      __syncthreads();
      const int P = total;
      for (int base = 0; base < P; base += NT * ILP) {
        Code<M> code[ILP];
        int cidx[ILP];
        uint32_t pos[ILP];
#pragma unroll
        for (int u = 0; u < ILP; ++u) {
          const int f = base + u * NT + threadIdx.x;
          cidx[u] = -1;
          if (f < P) {
            const int c = find_cell(c_pref, nch, f);
            cidx[u] = c;
            pos[u] = c_beg[c] + (uint32_t)(f - c_pref[c]);
            code[u].load(a.codes, pos[u]);
          }
        }
        const unsigned long long th = *(volatile unsigned long long*)&thr;
        const uint32_t th_hi = (uint32_t)(th >> 32);
#pragma unroll
        for (int u = 0; u < ILP; ++u) {
          bool acc = false;
          uint64_t comp = 0;
          if (cidx[u] >= 0) {
            const int c = cidx[u];
            const float* r = rq + c * QS;
            float dist = 0.f;
#pragma unroll
            for (int kk = 0; kk < M; ++kk) {
              const uint32_t b = code[u].byte(kk);
              if (LOCAL) {
                const float* w = (kk < M2)
                    ? a.Q + (((int64_t)c_i[c] * M2 + kk) * KSUB + b) * SUB
                    : a.S + (((int64_t)c_j[c] * M2 + kk - M2) * KSUB + b) * SUB;
#pragma unroll
                for (int d = 0; d < SUB; ++d) {
                  const float t = r[kk * SUB + d] - __ldg(w + d);
                  dist = fmaf(t, t, dist);
                }
              } else if (RG) {
                const float* w = a.R + ((int64_t)kk * KSUB + b) * SUB;
#pragma unroll
                for (int d = 0; d < SUB; ++d) {
                  const float t = r[kk * SUB + d] - __ldg(w + d);
                  dist = fmaf(t, t, dist);
                }
              } else {
                const float* w = Rs + (kk * KSUB + b) * RS;
#pragma unroll
                for (int d = 0; d < SUB; ++d) {
                  const float t = r[kk * SUB + d] - w[d];
                  dist = fmaf(t, t, dist);
                }
              }
            }
            const uint32_t o = f2ord(dist);
            if (o <= th_hi) {
              comp = ((uint64_t)o << 32) | (uint32_t)__ldg(a.ids + pos[u]);
              acc = comp < th;
            }
          }
          tk.offer(acc, comp, k, &thr);
        }
      }
      __syncthreads();
    }
    if (tk.nbuf > 0) tk.flush(k, &thr);
    __syncthreads();
    merge_lists(areas, NW, KP, TK::AREA, k, a.out_ids + q * k, a.out_dists + q * k);
  }
}

template <int M, int VAR, int ILP, int CAP, int SUB>
void run_fbpq_cfg(const ScanArgs& a, cudaStream_t st) {
  constexpr bool POINT = VAR != FB_TABLES;
  const size_t smem = (size_t)M * KSUB * 4 + (size_t)2 * CAP * 8 + (size_t)2 * ILP * 256 * sizeof(CodeVec<M>) +
                      (POINT ? (size_t)2 * ILP * 256 * 4 : 0) + SUB;
  auto kern = fbpq_scan_kernel<M, VAR, ILP, CAP, SUB>;
  BPQ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int grid = (int)std::min<int64_t>(a.nq, 1 << 20);
  kern<<<grid, 256, smem, st>>>(a);
  check_launch("fbpq scan kernel");
}

template <int M, int NT, int D, int U, int KW, int CH, bool HB, bool WQ, int RV = FB_POINT, int BBC = 0>
void run_fbpq_seg_t(const ScanArgs& a, cudaStream_t st) {
  constexpr int NW = NT / 32;
  constexpr size_t TAB = (size_t)M * KSUB * (RV == FB_Q8 ? 1 : (RV == FB_F16 ? 2 : 4));
  const size_t smem = (HB ? (size_t)4 * (MAX_T / 32) * 4 : TAB) + (size_t)NW * KW * 8 +
                      (BBC ? 0 : (size_t)NW * 256 * 4) + (size_t)CH * 8 + (size_t)(CH + 2) * 4 +
                      (HB ? (size_t)CH * 8 : 0) + (size_t)BBC * 8;
  auto kern = fbpq_scan_seg_kernel<M, NT, D, U, KW, CH, HB, WQ, RV, BBC>;
  BPQ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // HB reads its tables through L1: shared memory for five CTAs (132 KB), the rest as cache
  if (HB) BPQ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 57));
  if (WQ) {
    // persistent work-queue form: items, one resident wave of CTAs, merge of split queries
    BPQ_CHECK(a.items && a.n_items && a.item_counter && a.part_counter && a.merges && a.n_merges && a.part_ids &&
                  a.part_dists && a.k <= 128,
              BPQ_EINVAL, "work-queue scan: missing buffers or k > 128");
    BPQ_CUDA(cudaMemsetAsync(a.n_items, 0, 4 * sizeof(int32_t), st));  // n_items, item_counter, part_counter, n_merges
    build_items_kernel<<<(unsigned)((a.nq + 3) / 4), 128, 0, st>>>(a, a.work_W);
    check_launch("work item kernel");
    int per_sm = 0;
    BPQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
    const int grid = std::max(1, per_sm) * a.sm_count;
    kern<<<grid, NT, smem, st>>>(a);
    check_launch("fbpq segment scan kernel (work queue)");
    merge_parts_kernel<<<(unsigned)std::min<int64_t>(a.nq, (int64_t)a.sm_count * 4), 256, 0, st>>>(a);
    check_launch("partial list merge kernel");
    return;
  }
  // a selected list (its length is on the device): a few CTAs per SM, those past its end exit
  const int grid = (int)std::min<int64_t>(a.nq, a.sel ? (int64_t)8 * a.sm_count : (int64_t)1 << 20);
  kern<<<grid, NT, smem, st>>>(a);
  check_launch("fbpq segment scan kernel");
}

template <int M, int NT, int D, int U, int KW, int CH, bool HB = false>
void run_fbpq_seg(const ScanArgs& a, cudaStream_t st) {
  if (a.work_W > 0)
    run_fbpq_seg_t<M, NT, D, U, KW, CH, HB, true>(a, st);
  else
    run_fbpq_seg_t<M, NT, D, U, KW, CH, HB, false>(a, st);
}

// Per-point cross terms and k <= 128: the warp-segment scan.  Otherwise the
// round-based scan: k <= 128 with two candidates per thread per round and a
// 1024-entry top-k buffer (small shared memory, more CTAs per SM); larger k:
// four and 2048.
template <int M, int VAR>
void run_fbpq(const ScanArgs& a, cudaStream_t st) {
  if (VAR == FB_POINT && a.k <= 128)
    run_fbpq_seg<M, 128, 1, 4, 256, 512>(a, st);
  else if (a.k <= 128)
    run_fbpq_cfg<M, VAR, 2, 1024, 2048>(a, st);
  else
    run_fbpq_cfg<M, VAR, 4, 2048, 4096>(a, st);
}

template <int M, int SUB, int KP, bool LOCAL>
void run_recon(const ScanArgs& a, cudaStream_t st) {
  constexpr int NW = KP <= 128 ? 16 : (KP <= 256 ? 8 : (KP <= 512 ? 4 : 2));
  using TK = WarpTopK<KP>;
  // the global codebooks go to shared memory when they fit beside the rest
  constexpr size_t BASE = (size_t)NW * TK::AREA * 8 + (size_t)32 * (M * SUB + 1) * 4;
  constexpr bool RG = !LOCAL && BASE + (size_t)M * KSUB * (SUB + 1) * 4 > 200 * 1024;
  const size_t smem = BASE + ((LOCAL || RG) ? 0 : (size_t)M * KSUB * (SUB + 1) * 4);
  BPQ_CHECK(smem <= 227 * 1024, BPQ_EINVAL, "reconstruction scan: shape too large for shared memory");
  auto kern = recon_scan_kernel<M, SUB, KP, NW, LOCAL, RG>;
  BPQ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  BPQ_CUDA(cudaMemsetAsync(a.qcounter, 0, sizeof(int32_t), st));
  const int grid = (int)std::min<int64_t>(a.nq, (int64_t)a.sm_count);
  kern<<<grid, NW * 32, smem, st>>>(a);
  check_launch("reconstruction scan kernel");
}

// HBPQ: with the per-half-cell tables of the batch (a.hb_tables, k <= 128) the
// warp-segment scan with M lookups per candidate, then the O(D) reconstruction
// scan for the queries listed in a.qlist (their tables did not fit); without
// tables, the O(D) reconstruction for every query.
template <int M, int SUB, int KP>
void dispatch_scorer(const ScanArgs& a, int scorer, cudaStream_t st) {
  if (scorer == BPQ_SCORER_FBPQ) {
    run_fbpq<M, FB_POINT>(a, st);
  } else if (scorer == BPQ_SCORER_FBPQ_TABLES) {
    run_fbpq<M, FB_TABLES>(a, st);
  } else if (scorer == BPQ_SCORER_RECON) {
    run_recon<M, SUB, KP, false>(a, st);
  } else if (scorer == BPQ_SCORER_HBPQ && a.hb_tables) {
    BPQ_CHECK(a.k <= 128 && a.qlist && a.qlist_n, BPQ_EINVAL, "HBPQ table scan: k <= 128 and a fallback list");
    run_fbpq_seg<M, 128, 1, 4, 256, 512, true>(a, st);
    run_recon<M, SUB, KP, true>(a, st);
  } else {
    ScanArgs b = a;
    b.qlist = nullptr;
    b.qlist_n = nullptr;
    run_recon<M, SUB, KP, true>(b, st);
  }
}

template <int M, int SUB>
void dispatch_k(const ScanArgs& a, int scorer, cudaStream_t st) {
  if (a.k <= 32) dispatch_scorer<M, SUB, 32>(a, scorer, st);
  else if (a.k <= 128) dispatch_scorer<M, SUB, 128>(a, scorer, st);
  else dispatch_scorer<M, SUB, 1024>(a, scorer, st);
}

}  // namespace

bool scan_supported(int D, int M) {
  return (D == 128 && (M == 8 || M == 16)) || (D == 32 && M == 8) || (D == 8 && M == 8) || (D == 384 && M == 8);
}

void launch_scan_reduced(const ScanArgs& a, bool f16, cudaStream_t st) {
  if (a.nq <= 0) return;
  BPQ_CHECK(a.k >= 1 && a.k <= MAX_K, BPQ_EINVAL, "shortlist must be in [1, 1024]");
  BPQ_CHECK(a.D == 128 && (a.M == 8 || a.M == 16), BPQ_EINVAL,
            "the reduced-precision scan is built for D = 128, M = 8 or 16");
  BPQ_CHECK(a.sl_out && a.lut_scale && (f16 ? a.lut16 != nullptr : a.lut8 != nullptr), BPQ_EINVAL,
            "shortlist scan: missing table or output");
  // warp buffers of 128, chunks of 256 cells and a block buffer of 1024 entries (shortlists
  // up to 608) or 2048 keep the shared memory near 27 KB: eight CTAs per SM
  if (a.k <= 608) {
    if (a.M == 8 && f16) run_fbpq_seg_t<8, 128, 1, 4, 128, 256, false, false, FB_F16, 1024>(a, st);
    else if (a.M == 8) run_fbpq_seg_t<8, 128, 1, 4, 128, 256, false, false, FB_Q8, 1024>(a, st);
    else if (f16) run_fbpq_seg_t<16, 128, 1, 4, 128, 256, false, false, FB_F16, 1024>(a, st);
    else run_fbpq_seg_t<16, 128, 1, 4, 128, 256, false, false, FB_Q8, 1024>(a, st);
  } else {
    if (a.M == 8 && f16) run_fbpq_seg_t<8, 128, 1, 4, 128, 256, false, false, FB_F16, 2048>(a, st);
    else if (a.M == 8) run_fbpq_seg_t<8, 128, 1, 4, 128, 256, false, false, FB_Q8, 2048>(a, st);
    else if (f16) run_fbpq_seg_t<16, 128, 1, 4, 128, 256, false, false, FB_F16, 2048>(a, st);
    else run_fbpq_seg_t<16, 128, 1, 4, 128, 256, false, false, FB_Q8, 2048>(a, st);
  }
}

size_t position_hint_count(int64_t n_points) { return (size_t)((n_points + 255) / 256) + 2; }

void launch_position_hints(const uint32_t* offsets, int64_t ncells, int64_t n_points, uint32_t* hint,
                           cudaStream_t st) {
  if (n_points <= 0) return;
  const int64_t nb = (n_points + 255) / 256;
  position_hint_kernel<<<(unsigned)((nb + 256) / 256), 256, 0, st>>>(offsets, ncells, n_points, nb, hint);
  check_launch("position hint kernel");
}

void launch_rescore(const RescoreArgs& r, cudaStream_t st) {
  if (r.nq <= 0) return;
  BPQ_CHECK(r.S >= 1 && r.S <= MAX_K && r.k >= 1 && r.k <= r.S, BPQ_EINVAL, "need 1 <= k <= shortlist <= 1024");
  const int grid = (int)std::min<int64_t>(r.nq, 1 << 20);
  if (r.M == 8) rescore_kernel<8><<<grid, 256, 0, st>>>(r);
  else if (r.M == 16) rescore_kernel<16><<<grid, 256, 0, st>>>(r);
  else throw Error(BPQ_EINVAL, "the re-score kernel is built for M = 8 or 16");
  check_launch("re-score kernel");
}

void launch_scan(const ScanArgs& a, int scorer, cudaStream_t st) {
  if (a.nq <= 0) return;
  BPQ_CHECK(a.k >= 1 && a.k <= MAX_K, BPQ_EINVAL, "k must be in [1, 1024]");
  const int D = a.D, M = a.M;
  if (D == 128 && M == 8) dispatch_k<8, 16>(a, scorer, st);
  else if (D == 128 && M == 16) dispatch_k<16, 8>(a, scorer, st);
  else if (D == 32 && M == 8) dispatch_k<8, 4>(a, scorer, st);
  else if (D == 8 && M == 8) dispatch_k<8, 1>(a, scorer, st);
  else if (D == 384 && M == 8) dispatch_k<8, 48>(a, scorer, st);
  else throw Error(BPQ_EINVAL, "unsupported (D, M) for the scan kernels");
}

}  // namespace bpq
