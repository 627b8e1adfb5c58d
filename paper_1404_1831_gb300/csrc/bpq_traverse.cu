// Cell traversal of the inverted multi-index (§2.3.3).
//
// The paper walks cells in increasing d1[i] + d2[j] with the multi-sequence
// algorithm (a priority queue over the two sorted coarse-distance lists) until
// the visited cells hold l points.  A sequential heap is a poor fit for a GPU,
// so this kernel (one CTA per query) computes the same visited set in bands of
// the (row i, sorted column v) grid, where row i's keys d1[i] + s2[v] rise with v:
//
//   1. only the columns with the smallest d2 are sorted: a sample gives a value
//      theta, the columns with d2 <= theta are compacted and sorted by one warp
//      in registers (s2, p2).  Every cell outside this prefix has a key of at
//      least min(d1) + theta ("the limit"), so bands stay below the limit; a
//      query that needs more columns falls back to a full radix sort;
//   2. a band is every cell with tau_lo < key <= tau_hi.  The rows whose next
//      cell lies under an upper guess are compacted, and warp 0 alone picks
//      tau_hi (interpolation on the square root of the cell count, the region
//      being a staircase) so the band holds a bounded number of cells;
//   3. the band's cells are enumerated over the compacted rows, their point
//      counts read from the cell offsets and empty cells dropped;
//   4. if the band's points do not reach the budget, every cell is emitted and
//      the next band starts at tau_hi; otherwise the band is cut at the first
//      cell, in (key, cell id) order, at which the running count reaches L.  The
//      cut key comes from a weighted radix select, and the cells tied at that
//      key are taken in cell-id order.
//
// With `ordered`, each band is sorted by (key, cell id) before it is emitted,
// which reproduces the multi-sequence visit order exactly; without it (the
// search path) cells are emitted in any order, which the scan does not need.
// Either way the visited set is the prefix of the full sort of all T^2 cells by
// (key, cell id) that first reaches L points, restricted to non-empty cells.
// Keys are FP32 sums of FP32 table entries; for integer-valued inputs they are
// exact.
#include <algorithm>

#include "bpq_internal.cuh"

namespace bpq {
namespace {

constexpr int NT = 256;  // threads per CTA; also the radix of the sorts and selects
constexpr int NW = NT / 32;
constexpr int ECAP = 2048;  // band capacity (cells, empty ones included)
constexpr uint32_t ORD_INF = 0xffffffffu;

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
    long long t = (l < NW) ? r.v[l] : 0;
    t = warp_sum(t);
    if (l == 0) r.v[32] = t;
  }
  __syncthreads();
  return r.v[32];
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = min(x, (unsigned long long)__shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

__device__ unsigned long long block_min_u64(unsigned long long x, Red& r) {
  x = warp_min_u64(x);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) r.v[w] = (long long)x;
  __syncthreads();
  if (w == 0) {
    unsigned long long t = (l < NW) ? (unsigned long long)r.v[l] : ~0ull;
    t = warp_min_u64(t);
    if (l == 0) r.v[32] = (long long)t;
  }
  __syncthreads();
  return (unsigned long long)r.v[32];
}

__device__ uint32_t block_min_u32(uint32_t x, Red& r) { return (uint32_t)block_min_u64(x, r); }

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
    long long t = (l < NW) ? r.v[l] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, t, o);
      if (l >= o) t += y;
    }
    if (l < NW) r.v[l] = t;  // inclusive warp totals
  }
  __syncthreads();
  long long off = (w > 0) ? r.v[w - 1] : 0;
  *total = r.v[NW - 1];
  return x + off;
}

// Bitonic sort (ascending) of 32 * N keys held by one warp, N per lane, element
// lane * N + i in x[i].  Pairs closer than N are in the same lane; farther
// pairs are exchanged with shuffles.  Fully unrolled, so register indices are
// compile-time constants.
template <int N>
__device__ __forceinline__ void warp_sort(uint64_t (&x)[N]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int size = 2; size <= 32 * N; size <<= 1) {
#pragma unroll
    for (int j = size >> 1; j > 0; j >>= 1) {
      if (j < N) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const int p = i ^ j;
          if (p > i) {
            const bool up = (((lane * N + i) & size) == 0);
            const uint64_t a = x[i], b = x[p];
            const bool sw = (a > b) == up;
            x[i] = sw ? b : a;
            x[p] = sw ? a : b;
          }
        }
      } else {
        const int lj = j / N;
        const bool lower = (lane & lj) == 0;
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const uint64_t o = __shfl_xor_sync(0xffffffffu, x[i], lj);
          const bool up = (((lane * N + i) & size) == 0);
          x[i] = (lower == up) ? min(x[i], o) : max(x[i], o);
        }
      }
    }
  }
}

// Warp 0 sorts buf[0..n) (n <= 32 * N, padding with ~0) in place.
template <int N>
__device__ void warp_sort_buf_n(uint64_t* buf, int n) {
  const int lane = threadIdx.x & 31;
  uint64_t x[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const int e = lane * N + i;
    x[i] = e < n ? buf[e] : ~0ull;
  }
  warp_sort<N>(x);
#pragma unroll
  for (int i = 0; i < N; ++i) {
    const int e = lane * N + i;
    if (e < n) buf[e] = x[i];
  }
}

// Warp 0 sorts buf[0..n), n <= 256.
__device__ void warp_sort_buf(uint64_t* buf, int n) {
  if (n <= 32) warp_sort_buf_n<1>(buf, n);
  else if (n <= 64) warp_sort_buf_n<2>(buf, n);
  else if (n <= 128) warp_sort_buf_n<4>(buf, n);
  else warp_sort_buf_n<8>(buf, n);
}

// Stable LSD radix sort (ascending) of n uint32 keys with uint16 payloads, 8-bit
// digits (the full-sort fallback).  Elements are ranked in rounds of NT: inside
// a round equal digits keep thread order (warp match plus per-warp counts) and
// rounds run in order, so every pass is stable.  Four passes leave the result in
// k, v.
__device__ void block_radix_sort(uint32_t* k, uint16_t* v, uint32_t* k2, uint16_t* v2, int n, uint32_t* run,
                                 uint32_t* wc) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int shift = 0; shift < 32; shift += 8) {
    run[threadIdx.x] = 0;
    __syncthreads();
    for (int e0 = 0; e0 < n; e0 += NT) {
      const int e = e0 + threadIdx.x;
      warp_hist_add(run, e < n ? (k[e] >> shift) & 255u : 0u, e < n);
    }
    __syncthreads();
    if (w == 0) {  // exclusive scan of the 256 digit counts
      uint32_t c[8], tot = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        c[i] = run[l * 8 + i];
        tot += c[i];
      }
      uint32_t incl = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (l >= o) incl += y;
      }
      uint32_t ex = incl - tot;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        run[l * 8 + i] = ex;
        ex += c[i];
      }
    }
    __syncthreads();
    for (int r0 = 0; r0 < n; r0 += NT) {
#pragma unroll
      for (int x = 0; x < NW; ++x) wc[x * 256 + threadIdx.x] = 0;
      __syncthreads();
      const int e = r0 + threadIdx.x;
      const bool valid = e < n;
      const uint32_t key = valid ? k[e] : 0u;
      const uint32_t d = valid ? ((key >> shift) & 255u) : 256u;
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      const uint32_t below = __popc(peers & lanemask_lt());
      if (valid && below == 0) wc[w * 256 + d] = __popc(peers);
      __syncthreads();
      if (valid) {
        uint32_t pos = run[d] + below;
        for (int x = 0; x < w; ++x) pos += wc[x * 256 + d];
        k2[pos] = key;
        v2[pos] = v[e];
      }
      __syncthreads();
      uint32_t add = 0;
#pragma unroll
      for (int x = 0; x < NW; ++x) add += wc[x * 256 + threadIdx.x];
      run[threadIdx.x] += add;
      __syncthreads();
    }
    uint32_t* tk = k;
    k = k2;
    k2 = tk;
    uint16_t* tv = v;
    v = v2;
    v2 = tv;
  }
}

// Columns v < P2 of a row with distance a whose key is <= h, knowing that the
// first `from` qualify.
__device__ __forceinline__ int row_count(const float* s2, int P2, float a, int from, uint32_t h) {
  // galloping from `from` (a band moves most rows by a few columns), then bisection
  int lo = from, hi = from, step = 1;
  while (hi < P2 && f2ord(__fadd_rn(a, s2[hi])) <= h) {
    lo = hi + 1;
    hi = lo + step;
    step <<= 1;
  }
  hi = min(hi, P2);  // first v with key > h lies in [lo, hi]
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (f2ord(__fadd_rn(a, s2[mid])) <= h)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// Smallest key v (as ord bits) among the band entries such that the points of
// the entries with key <= v reach `need`; *below receives the points of the
// entries with key < v.  Weighted 8-bit radix select.
__device__ uint32_t weighted_select(const uint64_t* band, const uint32_t* cnt, int n, long long need,
                                    unsigned long long* hist, long long* below) {
  uint32_t prefix = 0, mask = 0;
  long long under = 0;
  const int l = threadIdx.x & 31;
  for (int shift = 24; shift >= 0; shift -= 8) {
    hist[threadIdx.x] = 0;
    __syncthreads();
    for (int e0 = 0; e0 < n; e0 += NT) {
      const int e = e0 + threadIdx.x;
      const uint32_t key = e < n ? (uint32_t)(band[e] >> 32) : 0u;
      warp_hist_add_w(hist, (key >> shift) & 255u, e < n ? cnt[e] : 0u, e < n && (key & mask) == prefix);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      unsigned long long c[8], tot = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        c[i] = hist[l * 8 + i];
        tot += c[i];
      }
      unsigned long long incl = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (l >= o) incl += y;
      }
      unsigned long long run = incl - tot;
      const long long want = need - under;
      if ((long long)run < want && want <= (long long)incl) {
        int d = 0;
        while ((long long)(run + c[d]) < want) run += c[d++];
        hist[256] = (unsigned long long)(l * 8 + d);
        hist[257] = run;
      }
    }
    __syncthreads();
    prefix |= (uint32_t)hist[256] << shift;
    mask |= 255u << shift;
    under += (long long)hist[257];
    __syncthreads();
  }
  *below = under;
  return prefix;
}

// Shared-memory layout of one CTA, for T coarse codewords per half.
struct Layout {
  size_t u_bytes;  // union: radix scratch | sort buffer | band
  size_t total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline Layout smem_layout(int T) {
  int TP = 1;
  while (TP < T) TP <<= 1;
  Layout l;
  const size_t radix = (size_t)TP * 12 + (size_t)(NW + 1) * 256 * 4;
  l.u_bytes = align16(max(radix, (size_t)8 * max(ECAP, TP)));
  // bcnt[ECAP] u32, s1[T] f32, s2[T] f32, afk[T] u32, p2/vlo/arow/vhic[T] u16, rowpref[T+1] u16
  l.total = l.u_bytes + (size_t)ECAP * 4 + (size_t)T * 12 + (size_t)T * 8 + (size_t)(T + 1) * 2 + 16;
  return l;
}

// The general path: one CTA per query.  With only_marked, it takes only the
// queries the warp kernel could not finish (ncells == FALLBACK), from the warp
// kernel's list when it kept one.
constexpr int FALLBACK = -2;

__global__ void __launch_bounds__(NT, 4) traverse_kernel(TraverseArgs a, int only_marked) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Red red;
  __shared__ int nband_s, nout_s, na_s, cnt_s;
  __shared__ long long emit_pts_s;
  __shared__ uint32_t theta_s, ovf_s;
  __shared__ unsigned long long hist[258];
  const float rho = a.rho;
  const int T = a.T;
  int TP = 1;
  while (TP < T) TP <<= 1;
  const Layout lay = smem_layout(T);
  // union region
  uint32_t* sk = reinterpret_cast<uint32_t*>(smem);
  uint32_t* sk2 = sk + TP;
  uint16_t* sv = reinterpret_cast<uint16_t*>(sk2 + TP);
  uint16_t* sv2 = sv + TP;
  uint32_t* srun = reinterpret_cast<uint32_t*>(sv2 + TP);
  uint32_t* swc = srun + 256;
  uint64_t* band = reinterpret_cast<uint64_t*>(smem);  // also the column sort buffer
  // fixed region
  uint32_t* bcnt = reinterpret_cast<uint32_t*>(smem + lay.u_bytes);
  float* s1 = reinterpret_cast<float*>(bcnt + ECAP);
  float* s2 = s1 + T;
  uint32_t* afk = reinterpret_cast<uint32_t*>(s2 + T);
  uint16_t* p2 = reinterpret_cast<uint16_t*>(afk + T);
  uint16_t* vlo = p2 + T;
  uint16_t* arow = vlo + T;
  uint16_t* vhic = arow + T;
  uint16_t* rowpref = vhic + T;  // T + 1
  // d2 ord keys live in a copy outside the union while the prefix is built
  uint32_t* dk = afk;

  const bool listed = only_marked && a.fb_list;
  const int64_t n_units = listed ? (int64_t)*a.fb_n : a.nq;
  for (int64_t u = blockIdx.x; u < n_units; u += gridDim.x) {
    const int64_t q = listed ? (int64_t)a.fb_list[u] : u;
    if (only_marked && !listed && a.ncells[q] != FALLBACK) continue;  // uniform across the CTA
    const int64_t L = a.L ? (int64_t)a.L[q] : (int64_t)a.L_scalar;
    const float* d1 = a.d1 + q * T;
    const float* d2 = a.d2 + q * T;
    __syncthreads();
    float m1 = __int_as_float(0x7f800000);
    for (int t = threadIdx.x; t < T; t += NT) {
      const float x = d1[t];
      s1[t] = x;
      m1 = fminf(m1, x);
      dk[t] = f2ord(d2[t]);
      vlo[t] = 0;
    }
    const float min1 = ord2f(block_min_u32(f2ord(m1), red));
    // 1. sorted prefix of the columns
    int P2;
    uint32_t limit;  // every key >= limit lies outside the sorted prefix
    bool full = false;
    if (T > 1024) {
      full = true;
    } else {
      uint32_t theta = ORD_INF;
      if (T > 256) {
        // sample every (TP/256)-th column; theta = a low quantile of the sample
        const int stride = TP / 256;
        const int srank = (L <= (int64_t)(2048.f * fmaxf(rho, 1.f))) ? 63 : 127;
        if (threadIdx.x < 32) {
          uint64_t x[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int col = (threadIdx.x * 8 + i) * stride;
            x[i] = col < T ? ((uint64_t)dk[col] << 32) : ~0ull;
          }
          warp_sort<8>(x);
          // element srank sits in lane srank / 8, slot srank % 8
          const uint64_t pick = __shfl_sync(0xffffffffu, x[srank % 8], srank / 8);
          if (threadIdx.x == 0) theta_s = (uint32_t)(pick >> 32);
        }
        __syncthreads();
        theta = theta_s;
      }
      // compact the columns with key <= theta, then warp 0 sorts them
      if (threadIdx.x == 0) cnt_s = 0;
      __syncthreads();
      for (int t0 = 0; t0 < T; t0 += NT) {
        const int t = t0 + threadIdx.x;
        const bool take = t < T && dk[t] <= theta;
        const uint32_t m = __ballot_sync(0xffffffffu, take);
        int at = 0;
        if ((threadIdx.x & 31) == 0 && m) at = atomicAdd(&cnt_s, __popc(m));
        at = __shfl_sync(0xffffffffu, at, 0);
        if (take) band[at + __popc(m & lanemask_lt())] = ((uint64_t)dk[t] << 32) | (uint32_t)t;
      }
      __syncthreads();
      P2 = cnt_s;
      if (P2 <= 256) {
        if (threadIdx.x < 32) warp_sort_buf(band, P2);
        __syncthreads();
      } else {  // larger prefixes: block-wide bitonic sort
        int n2 = 2;
        while (n2 < P2) n2 <<= 1;
        for (int t = P2 + threadIdx.x; t < n2; t += NT) band[t] = ~0ull;
        block_bitonic_sort(band, n2);
      }
      for (int t = threadIdx.x; t < P2; t += NT) {
        const uint64_t e = band[t];
        s2[t] = ord2f((uint32_t)(e >> 32));
        p2[t] = (uint16_t)(uint32_t)e;
      }
      limit = (theta == ORD_INF) ? ORD_INF : f2ord(__fadd_rn(min1, ord2f(theta)));
    }
    if (full) {
      for (int t = threadIdx.x; t < T; t += NT) {
        sk[t] = dk[t];
        sv[t] = (uint16_t)t;
      }
      __syncthreads();
      block_radix_sort(sk, sv, sk2, sv2, T, srun, swc);
      for (int t = threadIdx.x; t < T; t += NT) {
        s2[t] = ord2f(sk[t]);
        p2[t] = sv[t];
      }
      P2 = T;
      limit = ORD_INF;
    }
    __syncthreads();

    long long committed = 0;  // points of the emitted cells
    int nout = 0;
    bool overflow = false;
    int target = (int)fminf((float)ECAP, fmaxf(32.f, ceilf((float)L / fmaxf(rho, 1.f))));
    float pspan = 0.f;  // key span and cells of the previous band (the band-edge model)
    long long pcnt = 0;
    bool done = false;
    while (!done) {
      // 2. the smallest frontier key and its row
      unsigned long long fm = ~0ull;
      for (int u = threadIdx.x; u < T; u += NT) {
        const int v = vlo[u];
        if (v < P2) fm = min(fm, ((unsigned long long)f2ord(__fadd_rn(s1[u], s2[v])) << 32) | (uint32_t)u);
      }
      fm = block_min_u64(fm, red);
      const uint32_t hmin = (uint32_t)(fm >> 32);
      if (fm == ~0ull || hmin >= limit) {
        if (P2 < T) {  // the prefix is used up: sort every column and go on
          for (int t = threadIdx.x; t < T; t += NT) {
            sk[t] = f2ord(d2[t]);
            sv[t] = (uint16_t)t;
          }
          __syncthreads();
          block_radix_sort(sk, sv, sk2, sv2, T, srun, swc);
          for (int t = threadIdx.x; t < T; t += NT) {
            s2[t] = ord2f(sk[t]);
            p2[t] = sv[t];
          }
          P2 = T;
          limit = ORD_INF;
          __syncthreads();
          continue;
        }
        break;  // every cell visited
      }
      const int rowh = (int)(uint32_t)fm;
      // upper guess: `target` more columns in the row with the smallest frontier key
      const uint32_t lim1 = limit == ORD_INF ? ORD_INF - 1 : limit - 1;
      const uint32_t g_hi =
          min(lim1, f2ord(__fadd_rn(s1[rowh], s2[min(P2 - 1, (int)vlo[rowh] + target)])));
      const uint32_t g1 = min(
          g_hi, f2ord(__fadd_rn(s1[rowh], s2[min(P2 - 1, (int)vlo[rowh] + (int)ceilf(sqrtf(2.f * target)))])));
      // rows whose next cell is <= g_hi
      if (threadIdx.x == 0) na_s = 0;
      __syncthreads();
      for (int u0 = 0; u0 < T; u0 += NT) {
        const int u = u0 + threadIdx.x;
        uint32_t fk = ORD_INF;
        if (u < T && vlo[u] < P2) fk = f2ord(__fadd_rn(s1[u], s2[vlo[u]]));
        const bool take = fk <= g_hi;
        const uint32_t m = __ballot_sync(0xffffffffu, take);
        int at = 0;
        if ((threadIdx.x & 31) == 0 && m) at = atomicAdd(&na_s, __popc(m));
        at = __shfl_sync(0xffffffffu, at, 0);
        if (take) {
          const int i = at + __popc(m & lanemask_lt());
          arow[i] = (uint16_t)u;
          afk[i] = fk;
        }
      }
      __syncthreads();
      const int na = na_s;
      // the band's upper key h, searched by counts of the cells with key in
      // (vlo, h].  Every thread takes part in the counts (block sums) and follows
      // the same search.  Per compacted row, Lp holds the first column whose key
      // exceeds lo (exact once lo is counted) and Hp the first whose key exceeds
      // hi (P2 while hi is not counted), so a count searches each row only
      // between the two; a thread keeps the same rows throughout, so no barrier
      // guards them.  They live in the union region, free until the band is
      // enumerated.
      uint16_t* Lp = reinterpret_cast<uint16_t*>(smem);
      uint16_t* Hp = Lp + TP;
      uint16_t* Tp = Hp + TP;
      for (int i = threadIdx.x; i < na; i += NT) {
        Lp[i] = vlo[arow[i]];
        Hp[i] = (uint16_t)P2;
      }
      {
        auto count = [&](uint32_t h) -> long long {  // per-row results go to Tp
          long long c = 0;
          for (int i = threadIdx.x; i < na; i += NT) {
            const int u = arow[i], v = vlo[u];
            int r = v;
            if (afk[i] <= h) r = row_count(s2, Hp[i], s1[u], max((int)Lp[i], v + 1), h);
            Tp[i] = (uint16_t)r;
            c += r - v;
          }
          return block_sum(c, red);
        };
        auto take_lo = [&]() {
          uint16_t* t = Lp;
          Lp = Tp;
          Tp = t;
        };
        auto take_hi = [&]() {
          uint16_t* t = Hp;
          Hp = Tp;
          Tp = t;
        };
        const long long cap = ECAP;
        const long long lo_ok = max(1, target / 2), hi_ok = min(cap, 2LL * target);
        // aim a little above the middle of [lo_ok, hi_ok] (larger bands, fewer passes)
        const float aim = 1.2f * sqrtf((float)lo_ok * (float)hi_ok);
        const float fmin = ord2f(hmin);
        // The first band grows from a corner of the grid, so its cell count grows
        // about quadratically with the key; later bands are strips along the
        // frontier, which grow about linearly.  Guesses follow that model: the
        // first from g1, later ones from the previous band's cells per key unit.
        const bool quad = !(pspan > 0.f && pcnt > 0);
        uint32_t lo = hmin, hi = g_hi;  // hi = g_hi is not counted until chi >= 0
        long long clo = -1, chi = -1;   // -1: not counted (the model takes 0 at hmin)
        if (g_hi > hmin) {
          uint32_t mid = quad ? g1 : f2ord(fmin + pspan * (aim / (float)pcnt));
          mid = min(g_hi, max(hmin + 1, mid));
          for (int it = 0; it < 64; ++it) {
            const long long c = count(mid);
            if (c <= hi_ok) {
              lo = mid;
              clo = c;
              take_lo();
              if (c >= lo_ok || (mid == g_hi && chi < 0)) break;  // in the window, or all of g_hi fits
            } else {
              hi = mid;
              chi = c;
              take_hi();
            }
            if (hi <= lo + 1) break;
            const float flo = ord2f(lo), fhi = ord2f(hi), cl = (float)max(clo, 0LL);
            float f;
            if (chi < 0) {  // only the lower side counted: extrapolate from hmin
              const float r = aim / fmaxf(cl, 1.f);
              f = fmin + (flo - fmin) * (quad ? sqrtf(r) : r);
            } else if (it < 6) {  // interpolate inside the bracket
              const float ch = (float)chi;
              const float t = quad ? (sqrtf(aim) - sqrtf(cl)) / fmaxf(sqrtf(ch) - sqrtf(cl), 1e-6f)
                                   : (aim - cl) / fmaxf(ch - cl, 1.f);
              f = flo + (fhi - flo) * fminf(fmaxf(t, 0.05f), 0.95f);
            } else {
              f = -1.f;  // bisection below
            }
            if (f >= 0.f) {
              mid = f2ord(f);
            } else {
              mid = lo + ((hi - lo) >> 1);
            }
            mid = max(lo + 1, mid);
            mid = (chi < 0) ? min(hi, mid) : min(hi - 1, mid);
          }
        }
        // nothing above hmin was counted as fitting: the band is hmin's tie
        // group, unless that alone overflows the band capacity
        bool ovf = false;
        if (clo < 0) {
          clo = count(hmin);
          take_lo();
          ovf = clo > cap;
        }
        if (threadIdx.x == 0) ovf_s = ovf ? 1u : 0u;
        pspan = ord2f(lo) - fmin;
        pcnt = clo;
      }
      __syncthreads();
      if (ovf_s) {
        overflow = true;
        break;
      }
      // 3. enumerate the band over the compacted rows (each row ends at its Lp)
      for (int i = threadIdx.x; i < na; i += NT) vhic[i] = Lp[i];
      __syncthreads();
      {  // exclusive prefix of the band lengths over the compacted rows
        const int per = (na + NT - 1) / NT;
        const int r0 = threadIdx.x * per;
        long long loc = 0;
        for (int i = r0; i < min(na, r0 + per); ++i) loc += vhic[i] - vlo[arow[i]];
        long long tot;
        const long long incl = block_incl_scan(loc, red, &tot);
        long long run = incl - loc;
        for (int i = r0; i < min(na, r0 + per); ++i) {
          rowpref[i] = (uint16_t)run;
          run += vhic[i] - vlo[arow[i]];
        }
        if (threadIdx.x == 0) {
          rowpref[na] = (uint16_t)tot;
          nband_s = 0;
          nout_s = 0;
        }
      }
      __syncthreads();
      const int E = rowpref[na];
      long long pts = 0;
      for (int e = threadIdx.x; e < E; e += NT) {
        int lo = 0, hi = na;  // last compacted row with rowpref <= e
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (rowpref[mid] <= e)
            lo = mid;
          else
            hi = mid;
        }
        const int u = arow[lo];
        const int v = vlo[u] + (e - rowpref[lo]);
        const uint32_t cell = (uint32_t)u * (uint32_t)T + (uint32_t)p2[v];
        const uint32_t b = a.offsets[cell];
        const uint32_t n = a.offsets[cell + 1] - b;
        if (n > 0) {
          const float key = __fadd_rn(s1[u], s2[v]);
          const int pos = atomicAdd(&nband_s, 1);
          band[pos] = ((uint64_t)f2ord(key) << 32) | cell;
          bcnt[pos] = n;
          pts += n;
        }
      }
      const long long band_pts = block_sum(pts, red);
      const int nb = nband_s;
      const long long need = L - committed;
      bpq_cell* out = a.cells + q * (int64_t)a.cap;
      bool last = band_pts >= need;
      if (a.ordered) {
        // 4a. sorted band; cut at the first cell whose running count reaches L
        int n2 = 2;
        while (n2 < nb) n2 <<= 1;
        for (int t = nb + threadIdx.x; t < n2; t += NT) band[t] = ~0ull;
        block_bitonic_sort(band, n2);
        int emit = nb;
        long long emit_pts = band_pts;
        if (band_pts >= need) {
          emit = -1;
          long long run = 0;
          for (int c0 = 0; c0 < nb && emit < 0; c0 += NT) {
            const int c = c0 + threadIdx.x;
            long long x = 0;
            if (c < nb) {
              const uint32_t cell = (uint32_t)band[c];
              x = a.offsets[cell + 1] - a.offsets[cell];
            }
            long long tot;
            const long long incl = block_incl_scan(x, red, &tot);
            const uint32_t cand = (c < nb && run + incl >= need) ? (uint32_t)c : ORD_INF;
            const uint32_t first = block_min_u32(cand, red);
            if (first != ORD_INF) {
              emit = (int)first + 1;
              if ((uint32_t)c == first) emit_pts_s = run + incl;
              __syncthreads();
              emit_pts = emit_pts_s;
            }
            run += tot;
          }
        }
        if (nout + emit > a.cap) {
          overflow = true;
          break;
        }
        for (int t = threadIdx.x; t < emit; t += NT) {
          const uint64_t e = band[t];
          const uint32_t cell = (uint32_t)e;
          const uint32_t b = a.offsets[cell];
          out[nout + t] = bpq_cell{cell, b, a.offsets[cell + 1] - b, ord2f((uint32_t)(e >> 32))};
        }
        nout += emit;
        committed += emit_pts;
      } else if (band_pts < need) {
        // 4b. the whole band, in enumeration order
        if (nout + nb > a.cap) {
          overflow = true;
          break;
        }
        for (int t = threadIdx.x; t < nb; t += NT) {
          const uint64_t e = band[t];
          const uint32_t cell = (uint32_t)e;
          out[nout + t] = bpq_cell{cell, a.offsets[cell], bcnt[t], ord2f((uint32_t)(e >> 32))};
        }
        nout += nb;
        committed += band_pts;
      } else {
        // 4c. cut: every cell below the cut key, then the tied cells in cell-id order
        long long below;
        const uint32_t vcut = weighted_select(band, bcnt, nb, need, hist, &below);
        for (int t = threadIdx.x; t < nb; t += NT) {
          const uint64_t e = band[t];
          if ((uint32_t)(e >> 32) < vcut) {
            const int pos = nout + atomicAdd(&nout_s, 1);
            const uint32_t cell = (uint32_t)e;
            if (pos < a.cap) out[pos] = bpq_cell{cell, a.offsets[cell], bcnt[t], ord2f((uint32_t)(e >> 32))};
          }
        }
        __syncthreads();
        int added = nout_s;
        long long got = below;
        uint32_t lastcell = 0;
        bool first_tie = true;
        while (got < need) {
          uint32_t cand = ORD_INF;
          for (int t = threadIdx.x; t < nb; t += NT) {
            const uint64_t e = band[t];
            const uint32_t cell = (uint32_t)e;
            if ((uint32_t)(e >> 32) == vcut && (first_tie || cell > lastcell)) cand = min(cand, cell);
          }
          const uint32_t c = block_min_u32(cand, red);
          if (c == ORD_INF) break;  // not reached: the tied cells hold the remaining points
          const uint32_t b = a.offsets[c];
          const uint32_t n = a.offsets[c + 1] - b;
          if (threadIdx.x == 0 && nout + added < a.cap) out[nout + added] = bpq_cell{c, b, n, ord2f(vcut)};
          ++added;
          got += n;
          lastcell = c;
          first_tie = false;
        }
        if (nout + added > a.cap) {
          overflow = true;
          break;
        }
        nout += added;
        committed += got;
      }
      if (last) done = true;
      // next band
      for (int i = threadIdx.x; i < na; i += NT) vlo[arow[i]] = vhic[i];
      target = min(ECAP, 2 * target);
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      a.ncells[q] = overflow ? -1 : nout;
      a.npoints[q] = committed;
      if (overflow) atomicOr(a.status, STATUS_OVERFLOW);
    }
  }
}


// ---------------------------------------------------------------------------
// The common path (T <= 1024): one warp per query, no block-wide barriers.
//  * samples of d1 and d2 give thresholds theta1, theta2 for about `want` rows
//    and columns; the columns with d2 <= theta2 (at most PCAP) are compacted and
//    sorted in registers, and the rows with d1 <= theta1 (at most RCAP) are
//    compacted.  Every cell outside this row x column grid has a key of at least
//    the limit min(min(d1) + theta2, theta1 + min(d2)), so bands stay below it;
//    when the budget is not reached below the limit the grid is rebuilt larger
//    (rows keep their progress: the old grid's rows are among the new ones);
//  * each band holds at most BCAP cells: its edge is searched with warp-wide
//    counts and its cells are enumerated.  The band that reaches the budget is
//    sorted by (key, cell id) in registers and cut there; earlier bands are
//    emitted whole, sorted only with `ordered` (the visit order is then exact).
// A query whose grid would exceed the caps, or with a tie group larger than a
// band, is marked FALLBACK and finished by the CTA kernel.
// ---------------------------------------------------------------------------
constexpr int WPB = 4;      // warps (queries) per CTA
constexpr int PCAP = 256;   // sorted column prefix
constexpr int RCAP = 256;   // row prefix
constexpr int BCAP = 256;   // band cells
constexpr int WARP_TMAX = 1024;

struct WarpSmem {
  uint64_t band[BCAP];  // also the column compaction buffer
  float cs2[PCAP];
  float rs1[RCAP];
  uint32_t rfk[RCAP];   // frontier key per row (ord bits), ORD_INF when the row is used up
  uint16_t cp2[PCAP];
  uint16_t rid[RCAP];
  uint16_t rvhi[RCAP];
  uint16_t vlo[RCAP];   // columns already visited, per grid row
};

__device__ __forceinline__ uint32_t warp_min_u32(uint32_t x) { return __reduce_min_sync(0xffffffffu, x); }

template <typename V>
__device__ __forceinline__ V warp_excl_scan(V x, V* total) {
  const int l = threadIdx.x & 31;
  V v = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const V y = __shfl_up_sync(0xffffffffu, v, o);
    if (l >= o) v += y;
  }
  *total = __shfl_sync(0xffffffffu, v, 31);
  return v - x;
}

// Builds the row x column grid for about `want` rows and columns.  Returns false
// if it would exceed the caps.
__device__ __noinline__ bool build_grid(WarpSmem& W, const float* d1, const float* d2, int T, int TP, float want,
                                        float min1, float min2, int Rold, int* P2out, int* Rout, uint32_t* limit) {
  const int lane = threadIdx.x & 31;
  // a rebuild keeps the progress of the previous grid's rows: their (row id,
  // visited columns) go to rfk (rewritten below), sorted by row id.  The new
  // thresholds are not lower, so the old rows are among the new ones and the old
  // sorted columns stay a prefix of the new ones.
  for (int r = lane; r < Rold; r += 32) W.rfk[r] = ((uint32_t)W.rid[r] << 16) | W.vlo[r];
  __syncwarp();
  uint32_t th1 = ORD_INF, th2 = ORD_INF;
  if (T > PCAP) {  // thresholds: a quantile of 64 sampled rows / columns each
    const int stride = TP / 64;
    const int sr = min(63, max(0, (int)(want / (float)stride) - 1));
    uint64_t x[2], y[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int col = (lane * 2 + i) * stride;
      x[i] = col < T ? ((uint64_t)f2ord(d2[col]) << 32) : ~0ull;
      y[i] = col < T ? ((uint64_t)f2ord(d1[col]) << 32) : ~0ull;
    }
    warp_sort<2>(x);
    warp_sort<2>(y);
    th2 = (uint32_t)(__shfl_sync(0xffffffffu, x[sr & 1], sr >> 1) >> 32);
    th1 = (uint32_t)(__shfl_sync(0xffffffffu, y[sr & 1], sr >> 1) >> 32);
  }
  int P2 = 0, R = 0;
  for (int t0 = 0; t0 < T; t0 += 8 * 32) {
    // eight loads in flight per lane before the compaction uses them
    uint32_t kc[8];
    float dr[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int t = t0 + u * 32 + lane;
      kc[u] = t < T ? f2ord(__ldg(d2 + t)) : ORD_INF;
      dr[u] = t < T ? __ldg(d1 + t) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int t = t0 + u * 32 + lane;
      const bool tc = t < T && kc[u] <= th2;
      const bool tr = t < T && f2ord(dr[u]) <= th1;
      const uint32_t mc = __ballot_sync(0xffffffffu, tc);
      const uint32_t mr = __ballot_sync(0xffffffffu, tr);
      const int pc = P2 + __popc(mc & lanemask_lt());
      const int pr = R + __popc(mr & lanemask_lt());
      if (tc && pc < PCAP) W.band[pc] = ((uint64_t)kc[u] << 32) | (uint32_t)t;
      if (tr && pr < RCAP) {
        W.rs1[pr] = dr[u];
        W.rid[pr] = (uint16_t)t;
      }
      P2 += __popc(mc);
      R += __popc(mr);
    }
  }
  if (P2 > PCAP || R > RCAP) return false;
  __syncwarp();
  {  // bitonic sort in shared memory (a loop: small code) over the next power of two
    int n2 = 64;
    while (n2 < P2) n2 <<= 1;
    for (int v = P2 + lane; v < n2; v += 32) W.band[v] = ~0ull;
    warp_bitonic_sort(W.band, n2);
  }
  __syncwarp();
  for (int v = lane; v < P2; v += 32) {
    const uint64_t e = W.band[v];
    W.cs2[v] = ord2f((uint32_t)(e >> 32));
    W.cp2[v] = (uint16_t)(uint32_t)e;
  }
  __syncwarp();
  for (int r = lane; r < R; r += 32) {  // each new row's progress: a search of the old rows
    const uint32_t id = W.rid[r];
    int lo = 0, hi = Rold;  // first old row with id >= this one
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if ((W.rfk[mid] >> 16) < id) lo = mid + 1; else hi = mid;
    }
    W.vlo[r] = (lo < Rold && (W.rfk[lo] >> 16) == id) ? (uint16_t)(W.rfk[lo] & 0xffffu) : (uint16_t)0;
  }
  __syncwarp();
  for (int r = lane; r < R; r += 32) {
    const int v = W.vlo[r];
    W.rfk[r] = v < P2 ? f2ord(__fadd_rn(W.rs1[r], W.cs2[v])) : ORD_INF;
  }
  __syncwarp();
  *P2out = P2;
  *Rout = R;
  *limit = (th2 == ORD_INF) ? ORD_INF
                            : min(f2ord(__fadd_rn(min1, ord2f(th2))), f2ord(__fadd_rn(ord2f(th1), min2)));
  return true;
}

// A query the warp kernel cannot finish: marked for the CTA kernel (and listed).
__device__ __forceinline__ void hand_over(const TraverseArgs& a, int64_t q) {
  a.ncells[q] = FALLBACK;
  if (a.fb_list) {
    a.handed[q] = 1;
    a.fb_list[atomicAdd(a.fb_n, 1)] = (int32_t)q;
  }
}

__global__ void __launch_bounds__(WPB * 32, 7) traverse_warp_kernel(TraverseArgs a) {
  __shared__ WarpSmem smw[WPB];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WarpSmem& W = smw[warp];
  const int T = a.T;
  int TP = 1;
  while (TP < T) TP <<= 1;
  const float rho = fmaxf(a.rho, 1.f);
  for (int64_t q = (int64_t)blockIdx.x * WPB + warp; q < a.nq; q += (int64_t)gridDim.x * WPB) {
    const int64_t L = a.L ? (int64_t)a.L[q] : (int64_t)a.L_scalar;
    const float* d1 = a.d1 + q * T;
    const float* d2 = a.d2 + q * T;
    // rows and columns for about 5 sqrt(L / rho) + 32 visited cells; a query
    // that would need more than the caps goes straight to the CTA kernel
    float want = 5.f * sqrtf((float)L / rho) + 32.f;
    float pspan = 0.f;  // key span and cells of the previous band (the band-edge model)
    long long pcnt = 0;
    const float want_max = 0.9f * (float)PCAP;
    if (want > want_max && T > PCAP) {
      if (lane == 0) hand_over(a, q);
      continue;
    }
    __syncwarp();
    uint32_t m1 = ORD_INF, m2 = ORD_INF;
#pragma unroll 8
    for (int t = lane; t < T; t += 32) {
      m1 = min(m1, f2ord(__ldg(d1 + t)));
      m2 = min(m2, f2ord(__ldg(d2 + t)));
    }
    const float min1 = ord2f(warp_min_u32(m1)), min2 = ord2f(warp_min_u32(m2));
    int P2 = 0, R = 0;
    uint32_t limit = ORD_INF;
    bool fb = !build_grid(W, d1, d2, T, TP, want, min1, min2, 0, &P2, &R, &limit);
    long long committed = 0;
    int nout = 0;
    bool overflow = false;
    bpq_cell* out = a.cells + q * (int64_t)a.cap;
    while (!fb) {
      // smallest frontier key
      unsigned long long fm = ~0ull;
      for (int r = lane; r < R; r += 32) {
        const uint32_t f = W.rfk[r];
        if (f != ORD_INF) fm = min(fm, ((unsigned long long)f << 32) | (uint32_t)r);
      }
      fm = warp_min_u64(fm);
      const uint32_t hmin = (uint32_t)(fm >> 32);
      if (fm == ~0ull || hmin >= limit) {
        if (limit == ORD_INF) break;  // every cell visited
        // the grid is used up before the budget: a larger one, or the CTA kernel
        if (want >= want_max) {
          fb = true;
          break;
        }
        want = fminf(want_max, 2.f * want);
        fb = !build_grid(W, d1, d2, T, TP, want, min1, min2, R, &P2, &R, &limit);
        continue;
      }
      const int rh = (int)(uint32_t)fm;
      // The band's upper key, searched by counts of the cells with key in
      // (vlo, h] as in the CTA kernel: guesses from the band growth model, and
      // per row the first column above lo (Lp, exact once lo is counted) and
      // above hi (Hp; P2 while hi is not counted), kept between counts in the
      // band buffer (free until the band is enumerated).  Lane l keeps rows
      // l, l + 32, ... throughout, so no barrier guards them.
      uint16_t* Lp = reinterpret_cast<uint16_t*>(W.band);
      uint16_t* Hp = Lp + RCAP;
      uint16_t* Tp = Hp + RCAP;
      for (int r = lane; r < R; r += 32) {
        Lp[r] = W.vlo[r];
        Hp[r] = (uint16_t)P2;
      }
      auto count = [&](uint32_t h) -> long long {  // per-row results go to Tp
        int c = 0;  // at most RCAP x PCAP cells
        for (int r = lane; r < R; r += 32) {
          const int v = W.vlo[r];
          int e = v;
          if (W.rfk[r] <= h) e = row_count(W.cs2, Hp[r], W.rs1[r], max((int)Lp[r], v + 1), h);
          Tp[r] = (uint16_t)e;
          c += e - v;
        }
        return (long long)warp_sum(c);
      };
      auto take_lo = [&]() {
        uint16_t* t = Lp;
        Lp = Tp;
        Tp = t;
      };
      auto take_hi = [&]() {
        uint16_t* t = Hp;
        Hp = Tp;
        Tp = t;
      };
      const uint32_t lim1 = limit == ORD_INF ? ORD_INF - 1 : limit - 1;
      const int vh = W.vlo[rh];
      const float sh = W.rs1[rh];
      const uint32_t g_hi = min(lim1, f2ord(__fadd_rn(sh, W.cs2[min(P2 - 1, vh + BCAP)])));
      const uint32_t g1 = min(g_hi, f2ord(__fadd_rn(sh, W.cs2[min(P2 - 1, vh + 16)])));
      const long long lo_ok = BCAP / 2, hi_ok = BCAP;
      const float aim = 1.2f * sqrtf((float)lo_ok * (float)hi_ok);
      const float fmin = ord2f(hmin);
      const bool quad = !(pspan > 0.f && pcnt > 0);
      uint32_t lo = hmin, hi = g_hi;  // hi = g_hi is not counted until chi >= 0
      long long clo = -1, chi = -1;
      if (g_hi > hmin) {
        uint32_t mid = quad ? g1 : f2ord(fmin + pspan * (aim / (float)pcnt));
        mid = min(g_hi, max(hmin + 1, mid));
        for (int it = 0; it < 64; ++it) {
          const long long c = count(mid);
          if (c <= hi_ok) {
            lo = mid;
            clo = c;
            take_lo();
            if (c >= lo_ok || (mid == g_hi && chi < 0)) break;  // in the window, or all of g_hi fits
          } else {
            hi = mid;
            chi = c;
            take_hi();
          }
          if (hi <= lo + 1) break;
          const float flo = ord2f(lo), fhi = ord2f(hi), cl = (float)max(clo, 0LL);
          float f;
          if (chi < 0) {  // only the lower side counted: extrapolate from hmin
            const float r = aim / fmaxf(cl, 1.f);
            f = fmin + (flo - fmin) * (quad ? sqrtf(r) : r);
          } else if (it < 6) {  // interpolate inside the bracket
            const float ch = (float)chi;
            const float t = quad ? (sqrtf(aim) - sqrtf(cl)) / fmaxf(sqrtf(ch) - sqrtf(cl), 1e-6f)
                                 : (aim - cl) / fmaxf(ch - cl, 1.f);
            f = flo + (fhi - flo) * fminf(fmaxf(t, 0.05f), 0.95f);
          } else {
            f = -1.f;
          }
          mid = (f >= 0.f) ? f2ord(f) : lo + ((hi - lo) >> 1);
          mid = max(lo + 1, mid);
          mid = (chi < 0) ? min(hi, mid) : min(hi - 1, mid);
        }
      }
      if (clo < 0) {  // nothing above hmin fits: hmin's tie group, unless it overflows a band
        clo = count(hmin);
        take_lo();
        if (clo > BCAP) {
          fb = true;
          break;
        }
      }
      pspan = ord2f(lo) - fmin;
      pcnt = clo;
      // the band's cells: columns [vlo, Lp) of every row
      int loc = 0;
      for (int r = lane; r < R; r += 32) {
        const int v = W.vlo[r];
        const int vhi = Lp[r];
        W.rvhi[r] = (uint16_t)vhi;
        loc += vhi - v;
      }
      __syncwarp();  // the band buffer is overwritten below
      int E;
      int pos = warp_excl_scan(loc, &E);
      for (int r = lane; r < R; r += 32) {
        const int v0 = W.vlo[r], v1 = W.rvhi[r];
        const uint32_t rowbase = (uint32_t)W.rid[r] * (uint32_t)T;
        const float s1r = W.rs1[r];
        for (int v = v0; v < v1; ++v)
          W.band[pos++] = ((uint64_t)f2ord(__fadd_rn(s1r, W.cs2[v])) << 32) | (rowbase + W.cp2[v]);
      }
      __syncwarp();
      // lane l holds entries 8l .. 8l + 7
      uint64_t x[8];
      uint32_t cnt[8], beg[8];
      long long mysum = 0;
      auto load_counts = [&]() {
        mysum = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          cnt[i] = 0;
          beg[i] = 0;
          if (lane * 8 + i < E) {
            const uint32_t cell = (uint32_t)x[i];
            beg[i] = __ldg(a.offsets + cell);
            cnt[i] = __ldg(a.offsets + cell + 1) - beg[i];
          }
          mysum += cnt[i];
        }
      };
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int e = lane * 8 + i;
        x[i] = e < E ? W.band[e] : ~0ull;
      }
      const long long need = L - committed;
      load_counts();
      long long band_pts = warp_sum(mysum);
      if (a.ordered || band_pts >= need) {
        // the visit order, or the last band (its cut needs the (key, cell id) order):
        // bitonic sort of the band in shared memory (a loop: small code)
        int n2 = 64;
        while (n2 < E) n2 <<= 1;
        for (int v = E + lane; v < n2; v += 32) W.band[v] = ~0ull;
        warp_bitonic_sort(W.band, n2);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int e = lane * 8 + i;
          x[i] = e < E ? W.band[e] : ~0ull;
        }
        load_counts();
      }
      long long dummy;
      const long long before = warp_excl_scan(mysum, &dummy);
      // the cut: first entry whose running count reaches need
      int cut = E;  // entries [0, cut) are emitted
      {
        int mine = 1 << 30;
        long long run = before;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          run += cnt[i];
          if (mine == (1 << 30) && cnt[i] > 0 && run >= need) mine = lane * 8 + i;
        }
        const int first = (int)warp_min_u32((uint32_t)mine);
        if (first != (1 << 30)) cut = first + 1;
      }
      // emit the non-empty entries before the cut, in order
      int nz_total;
      int nzb;
      {
        int mine = 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) mine += (lane * 8 + i < cut && cnt[i] > 0);
        nzb = warp_excl_scan(mine, &nz_total);
      }
      if (nout + nz_total > a.cap) {
        overflow = true;
        break;
      }
      long long emitted_pts = 0;
      {
        int at = nout + nzb;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          if (lane * 8 + i < cut && cnt[i] > 0) {
            out[at++] = bpq_cell{(uint32_t)x[i], beg[i], cnt[i], ord2f((uint32_t)(x[i] >> 32))};
            emitted_pts += cnt[i];
          }
        }
      }
      emitted_pts = warp_sum(emitted_pts);
      nout += nz_total;
      committed += emitted_pts;
      if (band_pts >= need) break;
      // next band: advance every row to its band end
      __syncwarp();
      for (int r = lane; r < R; r += 32) {
        const int v = W.rvhi[r];
        W.vlo[r] = (uint16_t)v;
        W.rfk[r] = v < P2 ? f2ord(__fadd_rn(W.rs1[r], W.cs2[v])) : ORD_INF;
      }
      __syncwarp();
    }
    if (lane == 0) {
      if (fb) {
        hand_over(a, q);
      } else {
        if (a.handed) a.handed[q] = 0;
        a.ncells[q] = overflow ? -1 : nout;
        a.npoints[q] = committed;
        if (overflow) atomicOr(a.status, STATUS_OVERFLOW);
      }
    }
  }
}

}  // namespace

int traverse_band_capacity() { return ECAP; }

bool launch_traverse_warp(const TraverseArgs& a, cudaStream_t st) {
  if (a.nq <= 0) return false;
  BPQ_CHECK(a.T >= 1 && a.T <= MAX_T, BPQ_EINVAL, "T out of range for the traversal");
  const size_t smem = smem_layout(a.T).total;
  BPQ_CHECK(smem <= 227 * 1024, BPQ_EINVAL, "T too large for the traversal's shared memory");
  BPQ_CUDA(cudaFuncSetAttribute(traverse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (a.T > WARP_TMAX) {  // the general path for every query
    const int grid = (int)std::min<int64_t>(a.nq, 1 << 20);
    traverse_kernel<<<grid, NT, smem, st>>>(a, 0);
    check_launch("traverse kernel");
    return false;
  }
  // common path: one warp per query
  const int wgrid = (int)std::min<int64_t>((a.nq + WPB - 1) / WPB, 1 << 20);
  traverse_warp_kernel<<<wgrid, WPB * 32, 0, st>>>(a);
  check_launch("traverse warp kernel");
  return true;
}

// The queries the warp kernel marked, one CTA each (from its list when it kept
// one: the CTAs past the list's end exit at once).
void launch_traverse_marked(const TraverseArgs& a, cudaStream_t st) {
  const size_t smem = smem_layout(a.T).total;
  const int grid = (int)std::min<int64_t>(a.nq, 4096);
  traverse_kernel<<<grid, NT, smem, st>>>(a, 1);
  check_launch("traverse kernel");
}

void launch_traverse(const TraverseArgs& a, cudaStream_t st) {
  if (launch_traverse_warp(a, st)) launch_traverse_marked(a, st);
}

namespace {

// One warp per query: in-place, order-keeping compaction of the visited cells
// with the shard's begin and count (a step's 32 records are read before any of
// them is overwritten; writes go at or below the read positions).
__global__ void __launch_bounds__(256) localize_cells_kernel(TraverseArgs a, const uint32_t* __restrict__ loff) {
  const int lane = threadIdx.x & 31;
  const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (q >= a.nq) return;
  const int n = a.ncells[q];
  if (n <= 0) return;  // empty, or an overflow (-1) that the status word reports
  bpq_cell* cl = a.cells + q * (int64_t)a.cap;
  int kept = 0;
  for (int e0 = 0; e0 < n; e0 += 32) {
    const int e = e0 + lane;
    bpq_cell c{};
    bool keep = false;
    if (e < n) {
      c = cl[e];
      c.begin = __ldg(loff + c.cell);
      c.count = __ldg(loff + c.cell + 1) - c.begin;
      keep = c.count > 0;
    }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    __syncwarp();
    if (keep) cl[kept + __popc(m & lanemask_lt())] = c;
    kept += __popc(m);
  }
  if (lane == 0) a.ncells[q] = kept;
}

}  // namespace

void launch_localize_cells(const TraverseArgs& a, const uint32_t* loff, cudaStream_t st) {
  if (a.nq <= 0) return;
  localize_cells_kernel<<<(unsigned)((a.nq + 7) / 8), 256, 0, st>>>(a, loff);
  check_launch("cell localization kernel");
}

}  // namespace bpq
