// Per-query lookup tables and the query-independent FBPQ tables.
//
//  * Coarse tables (Eqs. 2-3, §2.3.3): d1[q][i] = ||q^1 - c^1_i||^2 and
//    d2[q][j] = ||q^2 - c^2_j||^2, the keys of the cell traversal.
//  * PQ table (§3.1, the query terms of Eq. 8 plus the codeword norms of Eq. 9):
//    lut[q][k][t] = ||R_k[t]||^2 - 2<q_k, R_k[t]> = sum_d R_k[t][d] (R_k[t][d] - 2 q_k[d]).
//  * FBPQ cross tables (Eq. 9, §3.3): X1[i][k][t] = 2<c^1_i restricted to block k,
//    R_k[t]> for k < M/2 and X2[j][k][t] likewise with c^2_j and R_{M/2+k}.
//
// With the FBPQ split used by the scan,
//   ||q - c_ij - r||^2 = d1[i] + d2[j] + sum_k lut[k][r_k] + sum_{k<M/2} X1[i][k][r_k]
//                                                       + sum_{k>=M/2} X2[j][k-M/2][r_k].
// For integer-valued inputs (queries in [0, 255], integer codebooks) every
// product and partial sum here is an integer below 2^24, so FP32 is exact.
#include <algorithm>

#include "bpq_internal.cuh"

namespace bpq {
namespace {

constexpr int BM = 64;   // table rows (queries) per CTA
constexpr int BN = 64;   // table columns (codewords) per CTA
constexpr int BK = 16;   // dimensions per shared-memory step
constexpr int MAXP = 18; // problems per launch (2 halves, or up to 16 sub-quantizers)

enum { MODE_SQ = 0, MODE_LUT = 1 };

struct PairProblem {
  const float* B;  // nb x dim codewords, dense
  float* out;      // out[a * ldo + o_off + b]
  int a_off;       // first query column of this problem
  int nb;
  int dim;
  int ldo;
  int o_off;
};
struct PairProblems {
  PairProblem p[MAXP];
};

// out[a][b] = sum_d f(A[a][a_off + d], B[b][d]) with f = (a-b)^2 or b(b - 2a).
template <int MODE>
__global__ void __launch_bounds__(256) pair_table_kernel(const float* __restrict__ A, int lda, int na,
                                                         PairProblems probs) {
  const PairProblem pr = probs.p[blockIdx.z];
  const int b0 = blockIdx.x * BN;
  if (b0 >= pr.nb) return;
  const int a0 = blockIdx.y * BM;
  __shared__ float As[BK][BM + 1];
  __shared__ float Bs[BK][BN + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4] = {};
  for (int d0 = 0; d0 < pr.dim; d0 += BK) {
    for (int e = threadIdx.x; e < BM * BK; e += 256) {
      int r = e / BK, d = e % BK;
      int a = a0 + r;
      As[d][r] = (a < na && d0 + d < pr.dim) ? A[(int64_t)a * lda + pr.a_off + d0 + d] : 0.f;
      int b = b0 + r;
      Bs[d][r] = (b < pr.nb && d0 + d < pr.dim) ? pr.B[(int64_t)b * pr.dim + d0 + d] : 0.f;
    }
    __syncthreads();
    const int dn = min(BK, pr.dim - d0);
    for (int d = 0; d < dn; ++d) {
      float av[4], bv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) av[r] = As[d][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) bv[c] = Bs[d][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if (MODE == MODE_SQ) {
            float t = av[r] - bv[c];
            acc[r][c] = fmaf(t, t, acc[r][c]);
          } else {
            float t = fmaf(-2.f, av[r], bv[c]);
            acc[r][c] = fmaf(bv[c], t, acc[r][c]);
          }
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    int a = a0 + ty + 16 * r;
    if (a >= na) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      int b = b0 + tx + 16 * c;
      if (b < pr.nb) pr.out[(int64_t)a * pr.ldo + pr.o_off + b] = acc[r][c];
    }
  }
}

// X[i][k][t] = 2 * sum_d C[i][k*s + d] * R[kbase + k][t][d]
__global__ void cross_table_kernel(const float* __restrict__ C, const float* __restrict__ R, int T,
                                   int m2, int s, int h, int kbase, float* __restrict__ X) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t n = (int64_t)T * m2 * KSUB;
  if (e >= n) return;
  int t = (int)(e % KSUB);
  int k = (int)((e / KSUB) % m2);
  int i = (int)(e / ((int64_t)KSUB * m2));
  const float* c = C + (int64_t)i * h + k * s;
  const float* r = R + ((int64_t)(kbase + k) * KSUB + t) * s;
  float acc = 0.f;
  for (int d = 0; d < s; ++d) acc = fmaf(c[d], r[d], acc);
  X[e] = 2.f * acc;
}

// bpq_search_shortlist step 1: per query, lo_k = min_t lut[k][t], step
// s = max_k (max_t lut[k][t] - lo_k) / 255 (1 if that is 0), and
// q8[k][t] = round_half_even((lut[k][t] - lo_k) / s), all in IEEE FP32.
template <int M>
__global__ void __launch_bounds__(256) quant_lut_kernel(const float* __restrict__ lut, int64_t nq,
                                                        uint8_t* __restrict__ lut8, float* __restrict__ scale) {
  __shared__ float lo_s[M];
  __shared__ unsigned int range_bits;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t q = blockIdx.x; q < nq; q += gridDim.x) {
    const float* L = lut + q * M * KSUB;
    __syncthreads();
    if (threadIdx.x == 0) range_bits = 0u;
    __syncthreads();
    for (int k = warp; k < M; k += 8) {
      float mn = __int_as_float(0x7f800000), mx = -__int_as_float(0x7f800000);
      for (int t = lane; t < KSUB; t += 32) {
        const float v = L[k * KSUB + t];
        mn = fminf(mn, v);
        mx = fmaxf(mx, v);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      }
      if (lane == 0) {
        lo_s[k] = mn;
        atomicMax(&range_bits, __float_as_uint(__fsub_rn(mx, mn)));  // >= 0: bit order = value order
      }
    }
    __syncthreads();
    const float range = __uint_as_float(range_bits);
    const float s = range > 0.f ? __fdiv_rn(range, 255.f) : 1.f;
    for (int e = threadIdx.x; e < M * KSUB; e += 256) {
      const float x = __fsub_rn(L[e], lo_s[e / KSUB]);
      const int v = __float2int_rn(__fdiv_rn(x, s));
      lut8[q * M * KSUB + e] = (uint8_t)min(255, max(0, v));
    }
    if (threadIdx.x == 0) scale[q] = s;
  }
}

}  // namespace

void launch_quant_lut(const float* lut, int M, int64_t nq, uint8_t* lut8, float* scale, cudaStream_t st) {
  if (nq <= 0) return;
  const int grid = (int)std::min<int64_t>(nq, 1 << 20);
  if (M == 8) quant_lut_kernel<8><<<grid, 256, 0, st>>>(lut, nq, lut8, scale);
  else if (M == 16) quant_lut_kernel<16><<<grid, 256, 0, st>>>(lut, nq, lut8, scale);
  else throw Error(BPQ_EINVAL, "the int8 table is built for M = 8 or 16");
  check_launch("table quantization kernel");
}

void launch_query_tables(const bpq_index& ix, const float* q, int64_t nq, float* d1, float* d2,
                         float* lut, cudaStream_t st) {
  if (nq <= 0) return;
  const int D = ix.p.D, T = ix.p.T, M = ix.p.M;
  const int gy = (int)((nq + BM - 1) / BM);
  BPQ_CHECK(nq < (int64_t)65535 * BM, BPQ_EINVAL, "too many queries in one table launch");
  if (d1 || d2) {
    PairProblems pp{};
    int np = 0;
    if (d1) pp.p[np++] = PairProblem{ix.C1.as<float>(), d1, 0, T, ix.h, T, 0};
    if (d2) pp.p[np++] = PairProblem{ix.C2.as<float>(), d2, ix.h, T, ix.h, T, 0};
    dim3 grid((T + BN - 1) / BN, gy, np);
    pair_table_kernel<MODE_SQ><<<grid, 256, 0, st>>>(q, D, (int)nq, pp);
    check_launch("coarse table kernel");
  }
  if (lut) {
    BPQ_CHECK(M <= MAXP, BPQ_EINVAL, "M too large for the table kernel");
    PairProblems pp{};
    for (int k = 0; k < M; ++k)
      pp.p[k] = PairProblem{ix.R.as<float>() + (int64_t)k * KSUB * ix.s, lut, k * ix.s, KSUB, ix.s,
                            M * KSUB, k * KSUB};
    dim3 grid(KSUB / BN, gy, M);
    pair_table_kernel<MODE_LUT><<<grid, 256, 0, st>>>(q, D, (int)nq, pp);
    check_launch("pq table kernel");
  }
}

void build_fbpq_tables(bpq_index& ix, cudaStream_t st) {
  const int T = ix.p.T;
  const int64_t n = (int64_t)T * ix.m2 * KSUB;
  ix.X1.alloc(n * sizeof(float));
  ix.X2.alloc(n * sizeof(float));
  const int blocks = (int)((n + 255) / 256);
  cross_table_kernel<<<blocks, 256, 0, st>>>(ix.C1.as<float>(), ix.R.as<float>(), T, ix.m2, ix.s, ix.h,
                                             0, ix.X1.as<float>());
  cross_table_kernel<<<blocks, 256, 0, st>>>(ix.C2.as<float>(), ix.R.as<float>(), T, ix.m2, ix.s, ix.h,
                                             ix.m2, ix.X2.as<float>());
  check_launch("fbpq cross table kernel");
}

}  // namespace bpq
