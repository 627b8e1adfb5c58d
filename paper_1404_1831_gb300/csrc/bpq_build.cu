// Index build: codebook learning (§2.3.1, §3.2), encoding (§2.3.2, Eqs. 6-7, 12)
// and the cell-contiguous inverted multi-index lists (§2.3.2).
//
// K-means works on the integer grid: training points must be integer-valued,
// cluster sums are accumulated in int64 (exact, so the result does not depend on
// the order of the atomic additions) and each centroid moves to its mean rounded
// half up, floor((2*sum + n) / (2*n)).  Assignment ties go to the lowest index,
// an empty cluster keeps its centroid, and K-means starts from the first K
// training vectors (local HBPQ codebooks start from the global ones).
//
// The lists are ordered by (cell, id) with a stable LSD radix sort on the 64-bit
// key cell << 32 | id, so ids ascend inside every cell.
#include <algorithm>
#include <vector>

#include "bpq_internal.cuh"

namespace bpq {
namespace {

constexpr int NTB = 256;

inline int blocks_for(int64_t n, int per = NTB) { return (int)std::max<int64_t>(1, (n + per - 1) / per); }

// ---------------------------------------------------------------------------
// Nearest codeword (ties to the lowest index) of a DIM-dimensional vector.
// ---------------------------------------------------------------------------
template <int DIM>
__device__ __forceinline__ int argmin_codeword(const float (&x)[DIM], const float* __restrict__ cb, int K) {
  float best = __int_as_float(0x7f800000);
  int bi = 0;
  for (int c = 0; c < K; ++c) {
    const float* w = cb + (int64_t)c * DIM;
    float d = 0.f;
#pragma unroll
    for (int t = 0; t < DIM; ++t) {
      const float e = x[t] - __ldg(w + t);
      d = fmaf(e, e, d);
    }
    if (d < best) {
      best = d;
      bi = c;
    }
  }
  return bi;
}

// One Lloyd assignment step with exact int64 accumulation of the cluster sums.
// Point p is X[p * ldx + col .. + DIM); its codebook is C + group[p] * gstride
// (group == nullptr: a single codebook).
template <int DIM>
__global__ void assign_accum_kernel(const float* __restrict__ X, int64_t ldx, int col, int64_t n,
                                    const float* __restrict__ C, int K, const int32_t* __restrict__ group,
                                    int64_t gstride, int32_t* __restrict__ assign,
                                    unsigned long long* __restrict__ sums, int* __restrict__ counts) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  float x[DIM];
#pragma unroll
  for (int t = 0; t < DIM; ++t) x[t] = X[p * ldx + col + t];
  const int g = group ? group[p] : 0;
  const int c = argmin_codeword<DIM>(x, C + (int64_t)g * gstride, K);
  if (assign) assign[p] = c;
  if (sums) {
    const int64_t slot = (int64_t)g * K + c;
#pragma unroll
    for (int t = 0; t < DIM; ++t)
      atomicAdd(sums + slot * DIM + t, (unsigned long long)(long long)__float2ll_rn(x[t]));
    atomicAdd(counts + slot, 1);
  }
}

__device__ __forceinline__ long long floordiv(long long a, long long b) {  // b > 0
  long long q = a / b;
  if ((a % b != 0) && (a < 0)) --q;
  return q;
}

// Centroid = mean rounded half up; empty clusters keep their centroid.
__global__ void update_kernel(float* __restrict__ C, const unsigned long long* __restrict__ sums,
                              const int* __restrict__ counts, int64_t nslots, int dim) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nslots * dim) return;
  const int n = counts[e / dim];
  if (n > 0) C[e] = (float)floordiv(2 * (long long)sums[e] + n, 2 * (long long)n);
}

__global__ void check_integer_kernel(const float* __restrict__ X, int64_t n, int* __restrict__ bad) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const float v = X[e];
    if (!(v == rintf(v)) || fabsf(v) > 1048576.f) atomicOr(bad, 1);
  }
}

// disp[p] = x[p] - [c^1_i; c^2_j] (the displacement of Eq. 6); also writes i, j.
template <int H>
__global__ void displacement_kernel(const float* __restrict__ X, int64_t n, const float* __restrict__ C1,
                                    const float* __restrict__ C2, int T, float* __restrict__ disp,
                                    int32_t* __restrict__ gi, int32_t* __restrict__ gj) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  float x[H];
  const float* xp = X + p * 2 * H;
#pragma unroll
  for (int t = 0; t < H; ++t) x[t] = xp[t];
  const int i = argmin_codeword<H>(x, C1, T);
#pragma unroll
  for (int t = 0; t < H; ++t) disp[p * 2 * H + t] = x[t] - C1[(int64_t)i * H + t];
#pragma unroll
  for (int t = 0; t < H; ++t) x[t] = xp[H + t];
  const int j = argmin_codeword<H>(x, C2, T);
#pragma unroll
  for (int t = 0; t < H; ++t) disp[p * 2 * H + H + t] = x[t] - C2[(int64_t)j * H + t];
  gi[p] = i;
  gj[p] = j;
}

// Encoding of Eqs. 6-7 (global codebooks) or Eq. 12 (local codebooks).
// With OPQ, X holds rot0 x (cells) and XR the residual-space vectors B rot0 x, with
// C1r, C2r the rotated centroids B c (the code is of XR - C1r/C2r); otherwise
// XR = X and C1r, C2r = C1, C2.
template <int H, int SUB>
__global__ void encode_kernel(const float* __restrict__ X, int64_t n, const float* __restrict__ C1,
                              const float* __restrict__ C2, int T, const float* __restrict__ R,
                              const float* __restrict__ Q, const float* __restrict__ S, int M,
                              int32_t* __restrict__ cell_out, uint8_t* __restrict__ codes_out,
                              const float* __restrict__ XR, const float* __restrict__ C1r,
                              const float* __restrict__ C2r) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const float* xp = X + p * 2 * H;
  const float* xrp = XR + p * 2 * H;
  float x[H];
#pragma unroll
  for (int t = 0; t < H; ++t) x[t] = xp[t];
  const int i = argmin_codeword<H>(x, C1, T);
#pragma unroll
  for (int t = 0; t < H; ++t) x[t] = xp[H + t];
  const int j = argmin_codeword<H>(x, C2, T);
  cell_out[p] = i * T + j;
  const int m2 = M / 2;
  for (int k = 0; k < M; ++k) {
    const bool second = k >= m2;
    const int kk = second ? k - m2 : k;
    const float* cen = second ? C2r + (int64_t)j * H + kk * SUB : C1r + (int64_t)i * H + kk * SUB;
    float r[SUB];
#pragma unroll
    for (int t = 0; t < SUB; ++t) r[t] = xrp[k * SUB + t] - cen[t];
    const float* cb;
    if (Q)
      cb = second ? S + ((int64_t)j * m2 + kk) * KSUB * SUB : Q + ((int64_t)i * m2 + kk) * KSUB * SUB;
    else
      cb = R + (int64_t)k * KSUB * SUB;
    codes_out[p * M + k] = (uint8_t)argmin_codeword<SUB>(r, cb, KSUB);
  }
}

// Squared encoding error ||x - xhat||^2 of n points from their cell and code
// (§4.2, Fig. errors): xhat = [c^1_i; c^2_j] + the codewords of the code, from the
// global codebooks R_k (Eq. 7) or the local codebooks Q^i_k, S^j_k (§3.2).  One
// warp per point, lanes over the dimensions (coalesced rows of x).
__global__ void recon_error_kernel(const float* __restrict__ X, int64_t n, const int32_t* __restrict__ cells,
                                   const uint8_t* __restrict__ codes, const float* __restrict__ C1,
                                   const float* __restrict__ C2, int T, int D, int M, const float* __restrict__ R,
                                   const float* __restrict__ Q, const float* __restrict__ S, float* __restrict__ err) {
  const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (p >= n) return;  // uniform over the warp
  const int H = D / 2, s = D / M, m2 = M / 2;
  const int cell = cells[p];
  const int i = cell / T, j = cell - i * T;
  float acc = 0.f;
  for (int d = lane; d < D; d += 32) {
    const int k = d / s, t = d - k * s;
    const int c = codes[p * M + k];
    const bool second = d >= H;
    const float cen = second ? C2[(int64_t)j * H + d - H] : C1[(int64_t)i * H + d];
    float r;
    if (Q)
      r = second ? S[(((int64_t)j * m2 + k - m2) * KSUB + c) * s + t] : Q[(((int64_t)i * m2 + k) * KSUB + c) * s + t];
    else
      r = R[((int64_t)k * KSUB + c) * s + t];
    const float e = X[p * D + d] - (cen + r);
    acc = fmaf(e, e, acc);
  }
  acc = warp_sum(acc);
  if (lane == 0) err[p] = acc;
}

__global__ void seq_ids_kernel(int32_t* ids, int64_t n, int64_t start) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n) ids[p] = (int32_t)(start + p);
}

__global__ void check_ids_kernel(const int32_t* ids, int64_t n, int* bad) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < n && ids[p] < 0) atomicOr(bad, 1);
}

// ---------------------------------------------------------------------------
// Exclusive scan of uint32 (in place), multi-level.
// ---------------------------------------------------------------------------
constexpr int SCAN_PER = 1024;  // elements per block (256 threads x 4)

__global__ void scan_block_kernel(uint32_t* data, int64_t n, uint32_t* block_sums) {
  __shared__ uint32_t tmp[NTB / 32 + 1];
  const int64_t base = (int64_t)blockIdx.x * SCAN_PER + threadIdx.x * 4;
  uint32_t v[4], s = 0;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    v[t] = (base + t < n) ? data[base + t] : 0u;
    s += v[t];
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  uint32_t incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (l >= o) incl += y;
  }
  if (l == 31) tmp[w] = incl;
  __syncthreads();
  if (w == 0) {
    uint32_t t = (l < NTB / 32) ? tmp[l] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (l >= o) t += y;
    }
    if (l < NTB / 32) tmp[l] = t;
  }
  __syncthreads();
  uint32_t run = incl - s + (w > 0 ? tmp[w - 1] : 0u);
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    if (base + t < n) data[base + t] = run;
    run += v[t];
  }
  if (threadIdx.x == NTB - 1 && block_sums) block_sums[blockIdx.x] = run;
}

__global__ void scan_add_kernel(uint32_t* data, int64_t n, const uint32_t* block_offsets) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) data[e] += block_offsets[e / SCAN_PER];
}

void exclusive_scan_u32(uint32_t* data, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  const int64_t nb = (n + SCAN_PER - 1) / SCAN_PER;
  if (nb == 1) {
    scan_block_kernel<<<1, NTB, 0, st>>>(data, n, nullptr);
    check_launch("scan");
    return;
  }
  DevBuf sums;
  sums.alloc(nb * sizeof(uint32_t));
  scan_block_kernel<<<(unsigned)nb, NTB, 0, st>>>(data, n, sums.as<uint32_t>());
  check_launch("scan");
  exclusive_scan_u32(sums.as<uint32_t>(), nb, st);
  scan_add_kernel<<<blocks_for(n), NTB, 0, st>>>(data, n, sums.as<uint32_t>());
  check_launch("scan add");
  BPQ_CUDA(cudaStreamSynchronize(st));  // `sums` is freed on return
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (uint64 key, uint32 value) pairs, 8-bit digits.
// ---------------------------------------------------------------------------
constexpr int RTILE = NTB * 16;

__global__ void radix_hist_kernel(const uint64_t* keys, int64_t n, int shift, uint32_t* ghist, int64_t ntiles) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t t0 = (int64_t)blockIdx.x * RTILE;
  for (int r = 0; r < 16; ++r) {
    const int64_t e = t0 + r * NTB + threadIdx.x;
    if (e < n) atomicAdd(&h[(keys[e] >> shift) & 255u], 1u);
  }
  __syncthreads();
  ghist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Rounds are processed in order and, inside a round, elements in thread order, so
// equal digits keep their input order (stable).
__global__ void radix_scatter_kernel(const uint64_t* kin, const uint32_t* vin, uint64_t* kout, uint32_t* vout,
                                     int64_t n, int shift, const uint32_t* goff, int64_t ntiles) {
  constexpr int NW = NTB / 32;
  __shared__ uint32_t run[256];
  __shared__ uint32_t wc[NW][256];
  const int w = threadIdx.x >> 5;
  run[threadIdx.x] = goff[(int64_t)threadIdx.x * ntiles + blockIdx.x];
  const int64_t t0 = (int64_t)blockIdx.x * RTILE;
  for (int r = 0; r < 16; ++r) {
    for (int x = 0; x < NW; ++x) wc[x][threadIdx.x] = 0;
    __syncthreads();
    const int64_t e = t0 + r * NTB + threadIdx.x;
    const bool valid = e < n;
    uint64_t key = valid ? kin[e] : 0;
    const uint32_t d = valid ? (uint32_t)((key >> shift) & 255u) : 256u;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t below = __popc(peers & lanemask_lt());
    if (valid && below == 0) wc[w][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      uint32_t pre = run[d];
      for (int x = 0; x < w; ++x) pre += wc[x][d];
      const uint32_t pos = pre + below;
      kout[pos] = key;
      vout[pos] = vin[e];
    }
    __syncthreads();
    uint32_t add = 0;
    for (int x = 0; x < NW; ++x) add += wc[x][threadIdx.x];
    run[threadIdx.x] += add;
    __syncthreads();
  }
}

// Sorts keys/vals in place (uses equally sized scratch); passes cover bits [0, nbits).
void radix_sort_pairs(DevBuf& keys, DevBuf& vals, int64_t n, int nbits, cudaStream_t st) {
  if (n <= 1) return;
  BPQ_CHECK(n < (int64_t)1 << 32, BPQ_EINVAL, "radix sort: too many elements");
  const int64_t ntiles = (n + RTILE - 1) / RTILE;
  DevBuf k2, v2, hist;
  k2.alloc(n * 8);
  v2.alloc(n * 4);
  hist.alloc(256 * ntiles * 4);
  uint64_t* ka = keys.as<uint64_t>();
  uint32_t* va = vals.as<uint32_t>();
  uint64_t* kb = k2.as<uint64_t>();
  uint32_t* vb = v2.as<uint32_t>();
  int passes = 0;
  for (int shift = 0; shift < nbits; shift += 8, ++passes) {
    radix_hist_kernel<<<(unsigned)ntiles, NTB, 0, st>>>(ka, n, shift, hist.as<uint32_t>(), ntiles);
    check_launch("radix hist");
    exclusive_scan_u32(hist.as<uint32_t>(), 256 * ntiles, st);
    radix_scatter_kernel<<<(unsigned)ntiles, NTB, 0, st>>>(ka, va, kb, vb, n, shift, hist.as<uint32_t>(), ntiles);
    check_launch("radix scatter");
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (passes & 1) {
    BPQ_CUDA(cudaMemcpyAsync(keys.p, ka, n * 8, cudaMemcpyDeviceToDevice, st));
    BPQ_CUDA(cudaMemcpyAsync(vals.p, va, n * 4, cudaMemcpyDeviceToDevice, st));
  }
  BPQ_CUDA(cudaStreamSynchronize(st));
}

// keys of the points already in the lists: cell (from the offsets) << 32 | id
__global__ void list_keys_kernel(const uint32_t* offsets, int64_t ncells, const int32_t* ids, int64_t n,
                                 uint64_t* keys, uint32_t* vals) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  int64_t lo = 0, hi = ncells;  // last cell with offsets[c] <= p
  while (hi - lo > 1) {
    int64_t mid = (lo + hi) >> 1;
    if ((int64_t)offsets[mid] <= p) lo = mid; else hi = mid;
  }
  keys[p] = ((uint64_t)lo << 32) | (uint32_t)ids[p];
  vals[p] = (uint32_t)p;
}

__global__ void pending_keys_kernel(const int32_t* cells, const int32_t* ids, int64_t n, int64_t base,
                                    uint64_t* keys, uint32_t* vals) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  keys[base + p] = ((uint64_t)(uint32_t)cells[p] << 32) | (uint32_t)ids[p];
  vals[base + p] = (uint32_t)(base + p);
}

__global__ void gather_lists_kernel(const uint64_t* keys, const uint32_t* vals, int64_t n, int64_t n_old,
                                    const uint8_t* old_codes, const uint8_t* new_codes, int M,
                                    uint8_t* codes, int32_t* ids, uint32_t* counts) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const uint64_t k = keys[p];
  const uint32_t src = vals[p];
  const uint8_t* from = (src < n_old) ? old_codes + (int64_t)src * M : new_codes + ((int64_t)src - n_old) * M;
  for (int t = 0; t < M; ++t) codes[p * M + t] = from[t];
  ids[p] = (int32_t)(uint32_t)k;
  atomicAdd(counts + (k >> 32), 1u);
}

// Per-point cross term of Eq. 9: sum_{k<M/2} X1[i][k][r_k] + sum_{k>=M/2} X2[j][k-M/2][r_k]
// = 2<[c^1_i; c^2_j], r>, for the point at list position p (its cell from the offsets).
__global__ void point_cross_kernel(const uint32_t* offsets, int64_t ncells, const uint8_t* codes, int M, int T,
                                   const float* X1, const float* X2, int64_t n, float* out) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  int64_t lo = 0, hi = ncells;  // last cell with offsets[c] <= p
  while (hi - lo > 1) {
    int64_t mid = (lo + hi) >> 1;
    if ((int64_t)offsets[mid] <= p) lo = mid; else hi = mid;
  }
  const int64_t i = lo / T, j = lo % T;
  const int m2 = M / 2;
  float acc = 0.f;
  for (int k = 0; k < M; ++k) {
    const int b = codes[p * M + k];
    acc += (k < m2) ? X1[(i * m2 + k) * KSUB + b] : X2[(j * m2 + k - m2) * KSUB + b];
  }
  out[p] = acc;
}

__global__ void cell_stats_kernel(const uint32_t* counts, int64_t ncells, unsigned long long* nonempty,
                                  unsigned int* maxc) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  const uint32_t v = counts[c];
  if (v) {
    atomicAdd(nonempty, 1ull);
    atomicMax(maxc, v);
  }
}

template <int DIM>
void assign_accum(const float* X, int64_t ldx, int col, int64_t n, const float* C, int K, const int32_t* group,
                  int64_t gstride, int32_t* assign, unsigned long long* sums, int* counts, cudaStream_t st) {
  assign_accum_kernel<DIM><<<blocks_for(n, 128), 128, 0, st>>>(X, ldx, col, n, C, K, group, gstride, assign,
                                                                sums, counts);
  check_launch("kmeans assign");
}

void assign_dispatch(int dim, const float* X, int64_t ldx, int col, int64_t n, const float* C, int K,
                     const int32_t* group, int64_t gstride, int32_t* assign, unsigned long long* sums,
                     int* counts, cudaStream_t st) {
  switch (dim) {
    case 1: assign_accum<1>(X, ldx, col, n, C, K, group, gstride, assign, sums, counts, st); break;
    case 4: assign_accum<4>(X, ldx, col, n, C, K, group, gstride, assign, sums, counts, st); break;
    case 8: assign_accum<8>(X, ldx, col, n, C, K, group, gstride, assign, sums, counts, st); break;
    case 16: assign_accum<16>(X, ldx, col, n, C, K, group, gstride, assign, sums, counts, st); break;
    case 48: assign_accum<48>(X, ldx, col, n, C, K, group, gstride, assign, sums, counts, st); break;
    case 64: assign_accum<64>(X, ldx, col, n, C, K, group, gstride, assign, sums, counts, st); break;
    case 192: assign_accum<192>(X, ldx, col, n, C, K, group, gstride, assign, sums, counts, st); break;
    default: throw Error(BPQ_EINVAL, "unsupported codeword dimension for K-means");
  }
}

// Lloyd iterations on codebooks C (G groups x K codewords x dim), in place.
void lloyd(const float* X, int64_t ldx, int col, int64_t n, float* C, int G, int K, int dim,
           const int32_t* group, int iters, cudaStream_t st) {
  const int64_t nslots = (int64_t)G * K;
  DevBuf sums, counts;
  sums.alloc(nslots * dim * 8);
  counts.alloc(nslots * 4);
  for (int it = 0; it < iters; ++it) {
    BPQ_CUDA(cudaMemsetAsync(sums.p, 0, sums.bytes, st));
    BPQ_CUDA(cudaMemsetAsync(counts.p, 0, counts.bytes, st));
    assign_dispatch(dim, X, ldx, col, n, C, K, group, (int64_t)K * dim, nullptr,
                    sums.as<unsigned long long>(), counts.as<int>(), st);
    update_kernel<<<blocks_for(nslots * dim), NTB, 0, st>>>(C, sums.as<unsigned long long>(), counts.as<int>(),
                                                            nslots, dim);
    check_launch("kmeans update");
  }
  BPQ_CUDA(cudaStreamSynchronize(st));
}

template <int H>
void displacement(const float* X, int64_t n, const bpq_index& ix, float* disp, int32_t* gi, int32_t* gj,
                  cudaStream_t st) {
  displacement_kernel<H><<<blocks_for(n, 128), 128, 0, st>>>(X, n, ix.C1.as<float>(), ix.C2.as<float>(), ix.p.T,
                                                             disp, gi, gj);
  check_launch("displacement");
}

template <int H, int SUB>
void encode_t(const bpq_index& ix, const float* x, int64_t n, int32_t* cell, uint8_t* codes, cudaStream_t st) {
  const bool local = ix.p.variant == BPQ_VARIANT_LOCAL;
  const float* xc = x;
  const float* xr = x;
  DevBuf bc, br;
  if (ix.opq) {  // rot0 x for the cell, B rot0 x for the code
    bc.alloc((size_t)n * ix.p.D * 4);
    br.alloc((size_t)n * ix.p.D * 4);
    rotate_for_index(ix, x, n, bc.as<float>(), br.as<float>(), st);
    xc = bc.as<float>();
    xr = br.as<float>();
  }
  const float* c1r = ix.opq ? ix.C1r.as<float>() : ix.C1.as<float>();
  const float* c2r = ix.opq ? ix.C2r.as<float>() : ix.C2.as<float>();
  encode_kernel<H, SUB><<<blocks_for(n, 128), 128, 0, st>>>(
      xc, n, ix.C1.as<float>(), ix.C2.as<float>(), ix.p.T, ix.R.as<float>(), local ? ix.Q.as<float>() : nullptr,
      local ? ix.S.as<float>() : nullptr, ix.p.M, cell, codes, xr, c1r, c2r);
  check_launch("encode");
  if (ix.opq) BPQ_CUDA(cudaStreamSynchronize(st));  // the rotated copies are released here
}

}  // namespace

void launch_encode(const bpq_index& ix, const float* x, int64_t n, int32_t* cell, uint8_t* codes, cudaStream_t st) {
  if (n <= 0) return;
  const int D = ix.p.D, M = ix.p.M;
  if (D == 128 && M == 8) encode_t<64, 16>(ix, x, n, cell, codes, st);
  else if (D == 128 && M == 16) encode_t<64, 8>(ix, x, n, cell, codes, st);
  else if (D == 32 && M == 8) encode_t<16, 4>(ix, x, n, cell, codes, st);
  else if (D == 8 && M == 8) encode_t<4, 1>(ix, x, n, cell, codes, st);
  else if (D == 384 && M == 8) encode_t<192, 48>(ix, x, n, cell, codes, st);
  else throw Error(BPQ_EINVAL, "unsupported (D, M) for encoding");
}

void launch_reconstruction_error(const bpq_index& ix, const float* x, int64_t n, const int32_t* cells,
                                 const uint8_t* codes, float* err, cudaStream_t st) {
  if (n <= 0) return;
  const bool local = ix.p.variant == BPQ_VARIANT_LOCAL;
  const int64_t threads = n * 32;
  DevBuf xr;
  if (ix.opq) {  // ||x - xhat|| = ||B rot0 x - (B c + r)|| (orthogonal rotations)
    xr.alloc((size_t)n * ix.p.D * 4);
    rotate_for_index(ix, x, n, nullptr, xr.as<float>(), st);
    x = xr.as<float>();
  }
  recon_error_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
      x, n, cells, codes, ix.opq ? ix.C1r.as<float>() : ix.C1.as<float>(),
      ix.opq ? ix.C2r.as<float>() : ix.C2.as<float>(), ix.p.T, ix.p.D, ix.p.M, ix.R.as<float>(),
      local ? ix.Q.as<float>() : nullptr, local ? ix.S.as<float>() : nullptr, err);
  check_launch("reconstruction error kernel");
  if (ix.opq) BPQ_CUDA(cudaStreamSynchronize(st));
}

void fill_sequential_ids(int32_t* ids, int64_t n, int64_t start, cudaStream_t st) {
  if (n <= 0) return;
  seq_ids_kernel<<<blocks_for(n), NTB, 0, st>>>(ids, n, start);
  check_launch("sequential ids");
}

bool ids_nonnegative(const int32_t* ids, int64_t n, cudaStream_t st) {
  if (n <= 0) return true;
  DevBuf flag;
  flag.alloc(4);
  BPQ_CUDA(cudaMemsetAsync(flag.p, 0, 4, st));
  check_ids_kernel<<<blocks_for(n), NTB, 0, st>>>(ids, n, flag.as<int>());
  check_launch("id check");
  int bad = 0;
  BPQ_CUDA(cudaMemcpyAsync(&bad, flag.p, 4, cudaMemcpyDeviceToHost, st));
  BPQ_CUDA(cudaStreamSynchronize(st));
  return bad == 0;
}

void build_point_cross(bpq_index& ix, cudaStream_t st) {
  const int64_t n = ix.n_points;
  if (ix.p.variant != BPQ_VARIANT_GLOBAL || n == 0) {
    ix.cross.release();
    return;
  }
  ix.cross.alloc(n * 4);
  point_cross_kernel<<<blocks_for(n), NTB, 0, st>>>(ix.offsets.as<uint32_t>(), (int64_t)ix.p.T * ix.p.T,
                                                    ix.codes.as<uint8_t>(), ix.p.M, ix.p.T, ix.X1.as<float>(),
                                                    ix.X2.as<float>(), n, ix.cross.as<float>());
  check_launch("point cross terms");
  BPQ_CUDA(cudaStreamSynchronize(st));
}

void finalize_lists(bpq_index& ix, cudaStream_t st) {
  const int64_t n_old = ix.n_points, n_new = ix.n_pending, n = n_old + n_new;
  const int T = ix.p.T, M = ix.p.M;
  const int64_t ncells = (int64_t)T * T;
  BPQ_CHECK(n < ((int64_t)1 << 32) - 1, BPQ_EINVAL, "at most 2^32 - 2 points per index");
  DevBuf keys, vals, codes, ids, offsets;
  keys.alloc(std::max<int64_t>(n, 1) * 8);
  vals.alloc(std::max<int64_t>(n, 1) * 4);
  if (n_old > 0) {
    list_keys_kernel<<<blocks_for(n_old), NTB, 0, st>>>(ix.offsets.as<uint32_t>(), ncells, ix.ids.as<int32_t>(), n_old,
                                                        keys.as<uint64_t>(), vals.as<uint32_t>());
    check_launch("list keys");
  }
  if (n_new > 0) {
    pending_keys_kernel<<<blocks_for(n_new), NTB, 0, st>>>(ix.pend_cells.as<int32_t>(), ix.pend_ids.as<int32_t>(),
                                                           n_new, n_old, keys.as<uint64_t>(), vals.as<uint32_t>());
    check_launch("pending keys");
  }
  int cell_bits = 1;
  while (((int64_t)1 << cell_bits) < ncells) ++cell_bits;
  radix_sort_pairs(keys, vals, n, 32 + cell_bits, st);
  codes.alloc(std::max<int64_t>(n, 1) * M);
  ids.alloc(std::max<int64_t>(n, 1) * 4);
  offsets.alloc((ncells + 1) * 4);
  BPQ_CUDA(cudaMemsetAsync(offsets.p, 0, (ncells + 1) * 4, st));
  if (n > 0) {
    gather_lists_kernel<<<blocks_for(n), NTB, 0, st>>>(keys.as<uint64_t>(), vals.as<uint32_t>(), n, n_old,
                                                       ix.codes.as<uint8_t>(), ix.pend_codes.as<uint8_t>(), M,
                                                       codes.as<uint8_t>(), ids.as<int32_t>(),
                                                       offsets.as<uint32_t>());
    check_launch("gather lists");
  }
  // counts -> stats -> exclusive offsets (entry ncells becomes n)
  DevBuf stats;
  stats.alloc(16);
  BPQ_CUDA(cudaMemsetAsync(stats.p, 0, 16, st));
  cell_stats_kernel<<<blocks_for(ncells), NTB, 0, st>>>(offsets.as<uint32_t>(), ncells,
                                                        stats.as<unsigned long long>(),
                                                        reinterpret_cast<unsigned int*>(stats.as<char>() + 8));
  check_launch("cell stats");
  exclusive_scan_u32(offsets.as<uint32_t>(), ncells + 1, st);
  unsigned long long st_host[2] = {0, 0};
  BPQ_CUDA(cudaMemcpyAsync(st_host, stats.p, 16, cudaMemcpyDeviceToHost, st));
  BPQ_CUDA(cudaStreamSynchronize(st));
  ix.n_nonempty = (int64_t)st_host[0];
  ix.max_cell = (int64_t)(uint32_t)st_host[1];
  std::swap(ix.codes.p, codes.p);
  std::swap(ix.codes.bytes, codes.bytes);
  std::swap(ix.ids.p, ids.p);
  std::swap(ix.ids.bytes, ids.bytes);
  std::swap(ix.offsets.p, offsets.p);
  std::swap(ix.offsets.bytes, offsets.bytes);
  ix.n_points = n;
  ix.n_pending = 0;
  ix.pend_cap = 0;
  ix.pend_cells.release();
  ix.pend_codes.release();
  ix.pend_ids.release();
  build_point_cross(ix, st);
}

void train_codebooks(bpq_index& ix, const float* learn, int64_t n, cudaStream_t st) {
  const int D = ix.p.D, T = ix.p.T, M = ix.p.M, h = ix.h, s = ix.s, m2 = ix.m2;
  const int iters = ix.p.kmeans_iters;
  BPQ_CHECK(n >= std::max(T, KSUB), BPQ_EINVAL, "need at least max(T, 256) learn vectors");
  {
    DevBuf flag;
    flag.alloc(4);
    BPQ_CUDA(cudaMemsetAsync(flag.p, 0, 4, st));
    check_integer_kernel<<<1024, NTB, 0, st>>>(learn, n * D, flag.as<int>());
    check_launch("integer check");
    int bad = 0;
    BPQ_CUDA(cudaMemcpyAsync(&bad, flag.p, 4, cudaMemcpyDeviceToHost, st));
    BPQ_CUDA(cudaStreamSynchronize(st));
    BPQ_CHECK(!bad, BPQ_EINVAL, "learn vectors must be integer-valued with |x| <= 2^20");
  }
  DevBuf learn_rot;
  std::vector<double> R0;
  if (ix.p.opq) {  // rot0 of the learn set (two subspaces), applied and rounded to the integer grid
    R0 = opq_learn_rotation(learn, n, D, 0, D, 2, st);
    DevBuf r0t;
    {
      std::vector<double> t((size_t)D * D);
      for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) t[(size_t)j * D + i] = R0[(size_t)i * D + j];
      r0t.alloc(t.size() * 8);
      BPQ_CUDA(cudaMemcpy(r0t.p, t.data(), t.size() * 8, cudaMemcpyHostToDevice));
    }
    learn_rot.alloc((size_t)n * D * 4);
    rotate_rows(learn, n, D, r0t.as<double>(), 1, true, learn_rot.as<float>(), st);
    BPQ_CUDA(cudaStreamSynchronize(st));
    learn = learn_rot.as<float>();
  }
  // coarse codebooks C^1, C^2: K-means on the halves, starting from the first T vectors
  ix.C1.alloc((size_t)T * h * 4);
  ix.C2.alloc((size_t)T * h * 4);
  BPQ_CUDA(cudaMemcpy2DAsync(ix.C1.p, h * 4, learn, (size_t)D * 4, h * 4, T, cudaMemcpyDeviceToDevice, st));
  BPQ_CUDA(cudaMemcpy2DAsync(ix.C2.p, h * 4, learn + h, (size_t)D * 4, h * 4, T, cudaMemcpyDeviceToDevice, st));
  lloyd(learn, D, 0, n, ix.C1.as<float>(), 1, T, h, nullptr, iters, st);
  lloyd(learn, D, h, n, ix.C2.as<float>(), 1, T, h, nullptr, iters, st);
  // displacements from the cell centroids, then R_1..R_M
  DevBuf disp, gi, gj;
  disp.alloc((size_t)n * D * 4);
  gi.alloc((size_t)n * 4);
  gj.alloc((size_t)n * 4);
  if (h == 64) displacement<64>(learn, n, ix, disp.as<float>(), gi.as<int32_t>(), gj.as<int32_t>(), st);
  else if (h == 192) displacement<192>(learn, n, ix, disp.as<float>(), gi.as<int32_t>(), gj.as<int32_t>(), st);
  else if (h == 16) displacement<16>(learn, n, ix, disp.as<float>(), gi.as<int32_t>(), gj.as<int32_t>(), st);
  else if (h == 4) displacement<4>(learn, n, ix, disp.as<float>(), gi.as<int32_t>(), gj.as<int32_t>(), st);
  else throw Error(BPQ_EINVAL, "unsupported D for training");
  std::vector<double> R1, R2;
  if (ix.p.opq) {  // rot1, rot2 of the displacement halves (M/2 subspaces each), applied and rounded
    R1 = opq_learn_rotation(disp.as<float>(), n, D, 0, h, m2, st);
    R2 = opq_learn_rotation(disp.as<float>(), n, D, h, h, m2, st);
    DevBuf bt;
    {
      std::vector<double> t((size_t)2 * h * h);
      for (int b = 0; b < 2; ++b)
        for (int i = 0; i < h; ++i)
          for (int j = 0; j < h; ++j) t[(size_t)b * h * h + (size_t)j * h + i] = (b ? R2 : R1)[(size_t)i * h + j];
      bt.alloc(t.size() * 8);
      BPQ_CUDA(cudaMemcpy(bt.p, t.data(), t.size() * 8, cudaMemcpyHostToDevice));
    }
    DevBuf dr;
    dr.alloc((size_t)n * D * 4);
    rotate_rows(disp.as<float>(), n, D, bt.as<double>(), 2, true, dr.as<float>(), st);
    BPQ_CUDA(cudaMemcpyAsync(disp.p, dr.p, (size_t)n * D * 4, cudaMemcpyDeviceToDevice, st));
    BPQ_CUDA(cudaStreamSynchronize(st));
  }
  ix.R.alloc((size_t)M * KSUB * s * 4);
  for (int k = 0; k < M; ++k) {
    float* Rk = ix.R.as<float>() + (size_t)k * KSUB * s;
    BPQ_CUDA(cudaMemcpy2DAsync(Rk, s * 4, disp.as<float>() + k * s, (size_t)D * 4, s * 4, KSUB,
                               cudaMemcpyDeviceToDevice, st));
    lloyd(disp.as<float>(), D, k * s, n, Rk, 1, KSUB, s, nullptr, iters, st);
  }
  if (ix.p.variant == BPQ_VARIANT_LOCAL) {
    // local codebooks of every half-cell, starting from the global ones (Eqs. 10-11)
    const size_t per = (size_t)KSUB * s;
    ix.Q.alloc((size_t)T * m2 * per * 4);
    ix.S.alloc((size_t)T * m2 * per * 4);
    DevBuf tmp;
    tmp.alloc((size_t)T * per * 4);
    for (int half = 0; half < 2; ++half) {
      DevBuf& dst = half ? ix.S : ix.Q;
      const int32_t* grp = half ? gj.as<int32_t>() : gi.as<int32_t>();
      for (int kk = 0; kk < m2; ++kk) {
        const int k = half * m2 + kk;
        const float* Rk = ix.R.as<float>() + (size_t)k * per;
        for (int g = 0; g < T; ++g)
          BPQ_CUDA(cudaMemcpyAsync(tmp.as<float>() + (size_t)g * per, Rk, per * 4, cudaMemcpyDeviceToDevice, st));
        lloyd(disp.as<float>(), D, k * s, n, tmp.as<float>(), T, KSUB, s, grp, iters, st);
        // scatter group-major (g, k) layout: dst[g][kk] = tmp[g]
        BPQ_CUDA(cudaMemcpy2DAsync(dst.as<float>() + (size_t)kk * per, (size_t)m2 * per * 4, tmp.p, per * 4,
                                   per * 4, T, cudaMemcpyDeviceToDevice, st));
      }
    }
  }
  if (ix.p.opq) set_opq_rotations(ix, R0.data(), R1.data(), R2.data(), st);
  BPQ_CUDA(cudaStreamSynchronize(st));
}

}  // namespace bpq
