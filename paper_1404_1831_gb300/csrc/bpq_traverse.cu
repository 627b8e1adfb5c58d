// Cell traversal of the inverted multi-index (§2.3.3).
//
// The paper walks cells in increasing d1[i] + d2[j] with the multi-sequence
// algorithm (a priority queue over the two sorted coarse-distance lists) until
// the visited cells hold l points.  A sequential heap is a poor fit for a GPU,
// so this kernel (one CTA per query) computes the same visited set in bands:
//
//   1. sort d2 with its indices (stable radix sort): s2, p2.  Every row i then
//      has keys d1[i] + s2[v] that are non-decreasing in v, and the cells of row
//      i visited so far are the columns v < vlo[i] (rows need no order);
//   2. a band is every cell with tau_lo < key <= tau_hi.  tau_hi is chosen so the
//      band holds between half the target and the target number of cells: the
//      cell count of a candidate tau is a binary search in each row whose next
//      cell is <= tau, summed over the block, and tau is searched by
//      interpolation on the square root of the count (the region is a
//      two-dimensional staircase) inside a bracket.  The first band targets
//      L / rho cells (rho = mean points per non-empty cell), later ones twice
//      the previous target, up to a fixed capacity;
//   3. the band's cells are enumerated row by row, their point counts read from
//      the cell offsets and empty cells dropped;
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

__device__ uint32_t block_min_u32(uint32_t x, Red& r) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = min(x, __shfl_xor_sync(0xffffffffu, x, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) r.v[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t t = (l < NW) ? (uint32_t)r.v[l] : 0xffffffffu;
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

// Stable LSD radix sort (ascending) of n uint32 keys with uint16 payloads, 8-bit
// digits.  Elements are ranked in rounds of NT (element r*NT + t by thread t):
// inside a round equal digits keep thread order (warp match plus per-warp
// counts) and rounds run in order, so every pass is stable.  A pass whose digit
// every key shares (kmin and kmax agree on all bits from it up) is skipped.  The
// result ends in k, v.
__device__ void block_radix_sort(uint32_t* k, uint16_t* v, uint32_t* k2, uint16_t* v2, int n, uint32_t kmin,
                                 uint32_t kmax, uint32_t* run, uint32_t* wc) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  uint32_t* const k0 = k;
  uint16_t* const v0 = v;
  for (int shift = 0; shift < 32; shift += 8) {
    if (((kmin ^ kmax) >> shift) == 0) break;  // this digit and all above are common
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
  if (k != k0) {  // odd number of passes: copy back
    for (int e = threadIdx.x; e < n; e += NT) {
      k0[e] = k[e];
      v0[e] = v[e];
    }
  }
  __syncthreads();
}

struct Lists {
  const float* s1;     // d1 in row order (unsorted)
  const float* s2;     // d2 sorted ascending
  const uint16_t* p2;  // column of s2[v]
  uint16_t* vlo;       // per row: columns already emitted (keys <= tau_lo)
  uint16_t* vhi;
  uint16_t* rowpref;   // T + 1
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

constexpr int NTH = 8;  // thresholds evaluated per block reduction

// Band cell counts for NTH ascending thresholds h[0..NTH) at once; the results
// land in out[0..NTH) on every thread.
__device__ void count_band_multi(const Lists& S, const uint32_t* h, long long* out, long long (*red8)[NTH]) {
  long long c[NTH];
#pragma unroll
  for (int j = 0; j < NTH; ++j) c[j] = 0;
  for (int u = threadIdx.x; u < S.T; u += NT) {
    const int v = S.vlo[u];
    if (v >= S.T) continue;
    const uint32_t kf = f2ord(__fadd_rn(S.s1[u], S.s2[v]));
    if (kf > h[NTH - 1]) continue;
#pragma unroll
    for (int j = 0; j < NTH; ++j)
      if (kf <= h[j]) c[j] += row_count(S, u, v + 1, h[j]) - v;
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < NTH; ++j) c[j] = warp_sum(c[j]);
  __syncthreads();
  if (l == 0)
#pragma unroll
    for (int j = 0; j < NTH; ++j) red8[w][j] = c[j];
  __syncthreads();
  if (threadIdx.x < NTH) {
    long long t = 0;
    for (int x = 0; x < NW; ++x) t += red8[x][threadIdx.x];
    red8[NW][threadIdx.x] = t;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < NTH; ++j) out[j] = red8[NW][j];
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

__global__ void __launch_bounds__(NT) traverse_kernel(TraverseArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Red red;
  __shared__ int nband_s;
  __shared__ int nout_s;
  __shared__ long long emit_pts_s;
  __shared__ unsigned long long hist[258];
  __shared__ long long red8[NW + 1][NTH];
  const float rho = a.rho;
  const int T = a.T;
  int TP = 1;
  while (TP < T) TP <<= 1;
  // shared layout: [sort scratch | band (union)][bcnt][s1 s2][p2 vlo vhi rowpref]
  const size_t sort_bytes = (size_t)TP * 12 + (size_t)(NW + 1) * 256 * 4;
  const size_t union_bytes = (max(sort_bytes, (size_t)8 * ECAP) + 15) & ~(size_t)15;
  uint32_t* sk = reinterpret_cast<uint32_t*>(smem);
  uint32_t* sk2 = sk + TP;
  uint16_t* sv = reinterpret_cast<uint16_t*>(sk2 + TP);
  uint16_t* sv2 = sv + TP;
  uint32_t* srun = reinterpret_cast<uint32_t*>(sv2 + TP);
  uint32_t* swc = srun + 256;
  uint64_t* band = reinterpret_cast<uint64_t*>(smem);
  uint32_t* bcnt = reinterpret_cast<uint32_t*>(smem + union_bytes);
  float* s1 = reinterpret_cast<float*>(bcnt + ECAP);
  float* s2 = s1 + T;
  uint16_t* p2 = reinterpret_cast<uint16_t*>(s2 + T);
  Lists S;
  S.T = T;
  S.s1 = s1;
  S.s2 = s2;
  S.p2 = p2;
  S.vlo = p2 + T;
  S.vhi = S.vlo + T;
  S.rowpref = S.vhi + T;

  for (int64_t q = blockIdx.x; q < a.nq; q += gridDim.x) {
    const int64_t L = a.L ? (int64_t)a.L[q] : (int64_t)a.L_scalar;
    const float* d1 = a.d1 + q * T;
    const float* d2 = a.d2 + q * T;
    // 1. rows as they are; columns sorted by (distance, index)
    __syncthreads();
    float s1min = __int_as_float(0x7f800000), s1max = -__int_as_float(0x7f800000);
    int argmin = 0;
    uint32_t kmin = 0xffffffffu, kmax = 0u;
    for (int t = threadIdx.x; t < T; t += NT) {
      const uint32_t kk = f2ord(d2[t]);
      sk[t] = kk;
      kmin = min(kmin, kk);
      kmax = max(kmax, kk);
      sv[t] = (uint16_t)t;
      const float x = d1[t];
      s1[t] = x;
      S.vlo[t] = 0;
      if (x < s1min) {
        s1min = x;
        argmin = t;
      }
      s1max = fmaxf(s1max, x);
    }
    kmin = block_min_u32(kmin, red);
    kmax = 0xffffffffu - block_min_u32(0xffffffffu - kmax, red);
    block_radix_sort(sk, sv, sk2, sv2, T, kmin, kmax, srun, swc);
    for (int t = threadIdx.x; t < T; t += NT) {
      s2[t] = ord2f(sk[t]);
      p2[t] = sv[t];
    }
    // the row with the smallest d1 (lowest index among ties) and the largest key
    const uint32_t mn = block_min_u32(f2ord(s1min), red);
    const uint32_t rmin = block_min_u32(f2ord(s1min) == mn ? (uint32_t)argmin : 0xffffffffu, red);
    const uint32_t s1max_ord = 0xffffffffu - block_min_u32(0xffffffffu - f2ord(s1max), red);
    const uint32_t max_ord = f2ord(__fadd_rn(ord2f(s1max_ord), s2[T - 1]));
    long long committed = 0;  // points of the emitted cells
    int nout = 0;
    bool overflow = false;
    int target = (int)fminf((float)ECAP, fmaxf(32.f, ceilf((float)L / fmaxf(rho, 1.f))));
    bool done = false;
    while (!done) {
      // 2. the band's upper key
      uint32_t fr = 0xffffffffu;
      for (int u = threadIdx.x; u < T; u += NT) {
        const int v = S.vlo[u];
        if (v < T) fr = min(fr, f2ord(__fadd_rn(s1[u], s2[v])));
      }
      const uint32_t hmin = block_min_u32(fr, red);
      if (hmin == 0xffffffffu) break;  // every cell visited
      uint32_t h;
      const long long cmin = count_band(S, hmin, red);
      if (cmin > target) {
        if (cmin > ECAP) {  // one tie group larger than the band
          overflow = true;
          break;
        }
        h = hmin;
      } else {
        // bracket [lo, hi] with count(lo) <= target < count(hi)
        uint32_t lo = hmin, hi = max_ord;
        long long clo = cmin, chi = -1;
        {  // first guess: `target` more cells in the row with the smallest d1
          const int vr = min(T - 1, (int)S.vlo[rmin] + target);
          const uint32_t g = f2ord(__fadd_rn(s1[rmin], s2[vr]));
          if (g > lo && g < hi) {
            const long long cg = count_band(S, g, red);
            if (cg <= target) {
              lo = g;
              clo = cg;
            } else {
              hi = g;
              chi = cg;
            }
          }
        }
        if (chi < 0) {
          chi = count_band(S, hi, red);
          if (chi <= target) {
            lo = hi;
            clo = chi;
          }
        }
        // each round evaluates NTH thresholds spread around the interpolated one
        // (counts grow like the square of the key inside a staircase)
        while (hi - lo > 1 && 2 * clo < target) {
          const float flo = ord2f(lo), fhi = ord2f(hi);
          const float sl = sqrtf((float)clo), sh = sqrtf((float)chi), sa = sqrtf(0.75f * (float)target);
          const float est = fminf(fmaxf((sa - sl) / fmaxf(sh - sl, 1e-6f), 0.02f), 0.98f);
          const float spread[NTH] = {0.35f, 0.55f, 0.75f, 0.9f, 1.0f, 1.12f, 1.3f, 1.6f};
          uint32_t th[NTH];
          uint32_t prev = lo;
#pragma unroll
          for (int j = 0; j < NTH; ++j) {
            uint32_t t = f2ord(flo + fminf(est * spread[j], 0.999f) * (fhi - flo));
            if (t <= prev) t = prev + 1;
            if (t >= hi) t = hi - 1;
            th[j] = max(t, prev);
            prev = th[j];
          }
          if (hi - lo <= (uint32_t)NTH + 1) {  // narrow bracket: every key in it
#pragma unroll
            for (int j = 0; j < NTH; ++j) th[j] = min(hi - 1, lo + 1 + j);
          }
          long long cnt[NTH];
          count_band_multi(S, th, cnt, red8);
          int best = -1;
#pragma unroll
          for (int j = 0; j < NTH; ++j)
            if (cnt[j] <= target) best = j;
          if (best >= 0) {
            lo = th[best];
            clo = cnt[best];
          }
          for (int j = NTH - 1; j > best; --j) {
            if (th[j] > lo) {
              hi = th[j];
              chi = cnt[j];
            }
          }
        }
        h = lo;
      }
      // 3. enumerate the band: rows u, columns [vlo[u], vhi[u])
      for (int u = threadIdx.x; u < T; u += NT) {
        const int vl = S.vlo[u];
        S.vhi[u] = (uint16_t)((vl < T && f2ord(__fadd_rn(s1[u], s2[vl])) <= h) ? row_count(S, u, vl + 1, h) : vl);
      }
      __syncthreads();
      {  // exclusive prefix of the band lengths over rows
        const int per = (T + NT - 1) / NT;
        const int r0 = threadIdx.x * per;
        long long loc = 0;
        for (int u = r0; u < min(T, r0 + per); ++u) loc += S.vhi[u] - S.vlo[u];
        long long tot;
        const long long incl = block_incl_scan(loc, red, &tot);
        long long run = incl - loc;
        for (int u = r0; u < min(T, r0 + per); ++u) {
          S.rowpref[u] = (uint16_t)run;
          run += S.vhi[u] - S.vlo[u];
        }
        if (threadIdx.x == 0) {
          S.rowpref[T] = (uint16_t)tot;
          nband_s = 0;
          nout_s = 0;
        }
      }
      __syncthreads();
      const int E = S.rowpref[T];
      long long pts = 0;
      for (int e = threadIdx.x; e < E; e += NT) {
        int lo = 0, hi = T;  // last row with rowpref <= e
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (S.rowpref[mid] <= e)
            lo = mid;
          else
            hi = mid;
        }
        const int u = lo;
        const int v = S.vlo[u] + (e - S.rowpref[u]);
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
      const bool last = band_pts >= need || h == max_ord;
      bpq_cell* out = a.cells + q * (int64_t)a.cap;
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
            const uint32_t cand = (c < nb && run + incl >= need) ? (uint32_t)c : 0xffffffffu;
            const uint32_t first = block_min_u32(cand, red);
            if (first != 0xffffffffu) {
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
          uint32_t cand = 0xffffffffu;
          for (int t = threadIdx.x; t < nb; t += NT) {
            const uint64_t e = band[t];
            const uint32_t cell = (uint32_t)e;
            if ((uint32_t)(e >> 32) == vcut && (first_tie || cell > lastcell)) cand = min(cand, cell);
          }
          const uint32_t c = block_min_u32(cand, red);
          if (c == 0xffffffffu) break;  // not reached: the tied cells hold the remaining points
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

size_t traverse_smem(int T) {
  int TP = 1;
  while (TP < T) TP <<= 1;
  const size_t sort_bytes = (size_t)TP * 12 + (size_t)(NW + 1) * 256 * 4;
  const size_t union_bytes = (std::max(sort_bytes, (size_t)8 * ECAP) + 15) & ~(size_t)15;
  return union_bytes + (size_t)ECAP * 4 + (size_t)T * 8 + (size_t)(4 * T + 1) * 2;
}

}  // namespace

int traverse_band_capacity() { return ECAP; }

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
