// Cell traversal of the inverted multi-index (§2.3.3).
//
// The paper walks cells in increasing d1[i] + d2[j] with the multi-sequence
// algorithm (a priority queue over the two sorted coarse-distance lists) until
// the visited cells hold l points.  A sequential heap is a poor fit for a GPU,
// so this kernel computes the same visit order in bands:
//
//   1. sort d2 (with its indices) in shared memory: s2, p2; every row i then has
//      keys d1[i] + s2[v] that are non-decreasing in v, and the cells of row i
//      visited so far are the columns v < vlo[i] (rows need no order);
//   2. a band is every cell whose key lies in (tau_lo, tau_hi]; tau_hi is found
//      by bisection on the number of cells with key <= tau (a binary search in
//      the rows whose next cell is <= tau, summed over the block), stopping
//      once the band holds between half the target and the target; the first
//      band targets L / rho cells (rho = mean points per non-empty cell) and
//      every further band twice the previous one, up to a fixed capacity;
//   3. the band's cells are enumerated row by row, their point counts read from
//      the cell offsets, empty cells dropped, and the rest sorted by
//      (key, cell id);
//   4. if the band's points do not reach the budget the whole band is emitted
//      and the next band starts at tau_hi; otherwise the band is cut at the first
//      cell whose running count reaches L.
//
// The emitted sequence is the full sort of all T^2 cells by (key, cell id),
// restricted to non-empty cells, up to the multi-sequence stopping point.  Keys
// are FP32 sums of FP32 table entries; for integer-valued inputs they are exact.
#include <algorithm>

#include "bpq_internal.cuh"

namespace bpq {
namespace {

constexpr int NT = 256;
constexpr int ECAP = 2048;  // band capacity (cells, empty ones included)

struct Red {
  long long v[33];
};

__device__ long long block_sum(long long x, Red& r) {
  x = warp_sum(x);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) r.v[w] = x;
  __syncthreads();
  if (w == 0) {
    long long t = (l < NT / 32) ? r.v[l] : 0;
    t = warp_sum(t);
    if (l == 0) r.v[32] = t;
  }
  __syncthreads();
  return r.v[32];
}

__device__ uint32_t block_min_u32(uint32_t x, Red& r) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = min(x, __shfl_xor_sync(0xffffffffu, x, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) r.v[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t t = (l < NT / 32) ? (uint32_t)r.v[l] : 0xffffffffu;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = min(t, __shfl_xor_sync(0xffffffffu, t, o));
    if (l == 0) r.v[32] = t;
  }
  __syncthreads();
  return (uint32_t)r.v[32];
}

// Inclusive scan of one value per thread; returns this thread's inclusive sum;
// *total receives the block total.
__device__ long long block_incl_scan(long long x, Red& r, long long* total) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (l >= o) x += y;
  }
  __syncthreads();
  if (l == 31) r.v[w] = x;
  __syncthreads();
  if (w == 0) {
    long long t = (l < NT / 32) ? r.v[l] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, t, o);
      if (l >= o) t += y;
    }
    if (l < NT / 32) r.v[l] = t;  // inclusive warp totals
  }
  __syncthreads();
  long long off = (w > 0) ? r.v[w - 1] : 0;
  *total = r.v[NT / 32 - 1];
  return x + off;
}

struct Lists {
  const float* s1;  // d1 in row order (unsorted)
  float* s2;        // d2 sorted ascending
  int* p2;          // column of s2[v]
  int* vlo;         // per row: columns already emitted (keys <= tau_lo)
  int* vhi;
  int* rowpref;     // T + 1
  uint64_t* band;
  int T;
};

// Columns v of row u with key <= h, knowing that the first `from` qualify.
__device__ __forceinline__ int row_count(const Lists& S, int u, int from, uint32_t h) {
  const float a = S.s1[u];
  int lo = from, hi = S.T;  // first v with key > h lies in [lo, hi]
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (f2ord(__fadd_rn(a, S.s2[mid])) <= h)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// Cells with tau_lo < key <= h (all rows).  Rows whose next cell is above h add nothing.
__device__ long long count_band(const Lists& S, uint32_t h, Red& r) {
  long long c = 0;
  for (int u = threadIdx.x; u < S.T; u += NT) {
    const int v = S.vlo[u];
    if (v < S.T && f2ord(__fadd_rn(S.s1[u], S.s2[v])) <= h) c += row_count(S, u, v + 1, h) - v;
  }
  return block_sum(c, r);
}

__global__ void __launch_bounds__(NT) traverse_kernel(TraverseArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Red red;
  __shared__ int nband_s;
  __shared__ long long emit_pts_s;
  const float rho = a.rho;
  const int T = a.T;
  int TP = 1;
  while (TP < T) TP <<= 1;
  // shared layout: [d2 sort keys / band union][s1 s2 p2 vlo vhi][rowpref]
  uint64_t* keys = reinterpret_cast<uint64_t*>(smem);
  const size_t union_bytes = max((size_t)8 * TP, (size_t)8 * ECAP);
  float* s1 = reinterpret_cast<float*>(smem + union_bytes);
  Lists S;
  S.T = T;
  S.band = keys;
  S.s1 = s1;
  S.s2 = s1 + T;
  S.p2 = reinterpret_cast<int*>(S.s2 + T);
  S.vlo = S.p2 + T;
  S.vhi = S.vlo + T;
  S.rowpref = S.vhi + T;

  for (int64_t q = blockIdx.x; q < a.nq; q += gridDim.x) {
    const int64_t L = a.L ? (int64_t)a.L[q] : (int64_t)a.L_scalar;
    const float* d1 = a.d1 + q * T;
    const float* d2 = a.d2 + q * T;
    // 1. rows as they are, columns sorted by (distance, index)
    __syncthreads();
    for (int t = threadIdx.x; t < TP; t += NT) {
      keys[t] = t < T ? ((uint64_t)f2ord(d2[t]) << 32) | (uint32_t)t : ~0ull;
      if (t < T) {
        s1[t] = d1[t];
        S.vlo[t] = 0;
      }
    }
    block_bitonic_sort(keys, TP);
    float s1max = -__int_as_float(0x7f800000);
    for (int t = threadIdx.x; t < T; t += NT) {
      uint64_t k2 = keys[t];
      S.s2[t] = ord2f((uint32_t)(k2 >> 32));
      S.p2[t] = (int)(uint32_t)k2;
      s1max = fmaxf(s1max, s1[t]);
    }
    // largest key: the largest row distance plus the largest column distance
    const uint32_t s1max_ord = 0xffffffffu - block_min_u32(0xffffffffu - f2ord(s1max), red);
    const uint32_t max_ord = f2ord(__fadd_rn(ord2f(s1max_ord), S.s2[T - 1]));
    long long committed = 0;  // points of the emitted cells
    int nout = 0;
    bool overflow = false;
    int target = (int)fminf((float)ECAP, fmaxf(32.f, ceilf((float)L / fmaxf(rho, 1.f))));
    bool done = false;
    while (!done) {
      // 2. the band's upper key: smallest frontier key first, then bisection
      uint32_t fr = 0xffffffffu;
      for (int u = threadIdx.x; u < T; u += NT) {
        int v = S.vlo[u];
        if (v < T) fr = min(fr, f2ord(__fadd_rn(s1[u], S.s2[v])));
      }
      const uint32_t hmin = block_min_u32(fr, red);
      if (hmin == 0xffffffffu) break;  // every cell visited
      uint32_t h;
      long long cmin = count_band(S, hmin, red);
      if (cmin > target) {
        if (cmin > ECAP) {  // one tie group larger than the band
          overflow = true;
          break;
        }
        h = hmin;
      } else if (count_band(S, max_ord, red) <= target) {
        h = max_ord;
      } else {
        uint32_t lo = hmin, hi = max_ord;  // count(lo) <= target < count(hi)
        while (hi - lo > 1) {
          uint32_t mid = lo + ((hi - lo) >> 1);
          const long long c = count_band(S, mid, red);
          if (c <= target) {
            lo = mid;
            if (2 * c >= target) break;  // band large enough
          } else {
            hi = mid;
          }
        }
        h = lo;
      }
      // 3. enumerate the band: rows u, columns [vlo[u], vhi[u])
      for (int u = threadIdx.x; u < T; u += NT) {
        const int vl = S.vlo[u];
        S.vhi[u] = (vl < T && f2ord(__fadd_rn(s1[u], S.s2[vl])) <= h) ? row_count(S, u, vl + 1, h) : vl;
      }
      __syncthreads();
      {  // exclusive prefix of the band lengths over rows
        const int per = (T + NT - 1) / NT;
        const int r0 = threadIdx.x * per;
        long long loc = 0;
        for (int u = r0; u < min(T, r0 + per); ++u) loc += S.vhi[u] - S.vlo[u];
        long long tot;
        long long incl = block_incl_scan(loc, red, &tot);
        long long run = incl - loc;
        for (int u = r0; u < min(T, r0 + per); ++u) {
          S.rowpref[u] = (int)run;
          run += S.vhi[u] - S.vlo[u];
        }
        if (threadIdx.x == 0) {
          S.rowpref[T] = (int)tot;
          nband_s = 0;
        }
      }
      __syncthreads();
      const int E = S.rowpref[T];
      long long pts = 0;
      for (int e = threadIdx.x; e < E; e += NT) {
        int lo = 0, hi = T;  // last row with rowpref <= e
        while (hi - lo > 1) {
          int mid = (lo + hi) >> 1;
          if (S.rowpref[mid] <= e)
            lo = mid;
          else
            hi = mid;
        }
        const int u = lo;
        const int v = S.vlo[u] + (e - S.rowpref[u]);
        const uint32_t cell = (uint32_t)u * (uint32_t)T + (uint32_t)S.p2[v];
        const uint32_t b = a.offsets[cell];
        const uint32_t n = a.offsets[cell + 1] - b;
        if (n > 0) {
          const float key = __fadd_rn(s1[u], S.s2[v]);
          int pos = atomicAdd(&nband_s, 1);
          S.band[pos] = ((uint64_t)f2ord(key) << 32) | cell;
          pts += n;
        }
      }
      const long long band_pts = block_sum(pts, red);
      const int nb = nband_s;
      // sort the band's non-empty cells by (key, cell id)
      int n2 = 2;
      while (n2 < nb) n2 <<= 1;
      for (int t = nb + threadIdx.x; t < n2; t += NT) S.band[t] = ~0ull;
      block_bitonic_sort(S.band, n2);
      // 4. emit the whole band, or cut it at the budget
      const long long need = L - committed;
      int emit = nb;
      long long emit_pts = band_pts;
      if (band_pts >= need) {
        emit = -1;
        long long run = 0;
        for (int c0 = 0; c0 < nb && emit < 0; c0 += NT) {
          const int c = c0 + threadIdx.x;
          long long x = 0;
          if (c < nb) {
            uint32_t cell = (uint32_t)S.band[c];
            x = a.offsets[cell + 1] - a.offsets[cell];
          }
          long long tot;
          long long incl = block_incl_scan(x, red, &tot);
          // first c with run + incl >= need
          uint32_t cand = (c < nb && run + incl >= need) ? (uint32_t)c : 0xffffffffu;
          uint32_t first = block_min_u32(cand, red);
          if (first != 0xffffffffu) {
            emit = (int)first + 1;
            // points up to and including `first`, from the thread that holds it
            if ((uint32_t)c == first) emit_pts_s = run + incl;
            __syncthreads();
            emit_pts = emit_pts_s;
          }
          run += tot;
        }
        done = true;
      } else if (h == max_ord) {
        done = true;
      }
      if (nout + emit > a.cap) {
        overflow = true;
        break;
      }
      bpq_cell* out = a.cells + q * (int64_t)a.cap + nout;
      for (int t = threadIdx.x; t < emit; t += NT) {
        uint64_t e = S.band[t];
        uint32_t cell = (uint32_t)e;
        uint32_t b = a.offsets[cell];
        out[t] = bpq_cell{cell, b, a.offsets[cell + 1] - b, ord2f((uint32_t)(e >> 32))};
      }
      nout += emit;
      committed += emit_pts;
      // next band
      for (int u = threadIdx.x; u < T; u += NT) S.vlo[u] = S.vhi[u];
      target = min(ECAP, 2 * target);
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      a.ncells[q] = overflow ? -1 : nout;
      a.npoints[q] = committed;
      if (overflow) atomicExch(a.status, 1);
    }
  }
}

}  // namespace

int traverse_band_capacity() { return ECAP; }

static size_t traverse_smem(int T) {
  int TP = 1;
  while (TP < T) TP <<= 1;
  return std::max((size_t)8 * TP, (size_t)8 * ECAP) + (size_t)T * 5 * 4 + (size_t)(T + 1) * 4;
}

void launch_traverse(const TraverseArgs& a, cudaStream_t st) {
  if (a.nq <= 0) return;
  BPQ_CHECK(a.T >= 1 && a.T <= MAX_T, BPQ_EINVAL, "T out of range for the traversal");
  const size_t smem = traverse_smem(a.T);
  BPQ_CUDA(cudaFuncSetAttribute(traverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int grid = (int)std::min<int64_t>(a.nq, 1 << 20);
  traverse_kernel<<<grid, NT, smem, st>>>(a);
  check_launch("traverse kernel");
}

}  // namespace bpq
