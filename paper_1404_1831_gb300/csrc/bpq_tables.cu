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
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "bpq_internal.cuh"

namespace bpq {
namespace {

constexpr int MAXP = 18; // problems per launch (2 halves, or up to 16 sub-quantizers)

enum { MODE_SQ = 0, MODE_LUT = 1 };

// ---------------------------------------------------------------------------
// Tensor-core tables (tcgen05, BF16 operands, FP32 accumulation in tensor
// memory).  One CTA of 128 threads computes a tile of 128 queries x up to 256
// codewords of one problem: D = A B^T with A the query slice and B the codewords
// (BF16 copies made at index build), then out = ||a||^2 + ||b||^2 - 2 D (coarse
// tables) or ||b||^2 - 2 D (PQ table).  Integer inputs of magnitude <= 256 are
// exact in BF16, every product is below 2^16 and every partial sum below 2^24,
// so the FP32 accumulation and the epilogue are exact.  Real-valued queries (OPQ
// rotations) against exact codewords are split into three BF16 planes
// a = a_hi + a_mid + a_lo (a_mid, a_lo the BF16 roundings of what is left), which
// carry a's 24-bit mantissa; the three products with the same codewords are exact
// and accumulate into one FP32 result, as accurate as an FP32 dot product (`split`,
// when the launch gives the planes' shared memory).  Any other tile whose operands
// BF16 cannot hold is computed in FP32 on the CUDA cores, so the tables never lose
// precision.
// Operands are K-major in shared memory without swizzle: 8-row x 16-byte core
// matrices, core (row group g, column group c) at byte 128 (g * KB + c).
// ---------------------------------------------------------------------------
constexpr int TC_M = 128, TC_N = 256;

struct TcProblem {
  const __nv_bfloat16* Bb;  // nb x kpad BF16, zero padded
  const float* B;           // nb x dim FP32
  const float* bn;          // nb squared norms
  float* out;               // out[a * ldo + o_off + b]
  int a_off, nb, dim, kpad, ldo, o_off;
  int b_planes;             // BF16 planes that hold B exactly: 1, 2 (Bb + Bb2), or 0 (none: CUDA cores)
  const __nv_bfloat16* Bb2; // second plane B - bf16(B) (b_planes == 2)
};
struct TcProblems {
  TcProblem p[MAXP];
};

template <int MODE>
__global__ void __launch_bounds__(128) tc_table_kernel(const float* __restrict__ A, int lda, int na,
                                                       TcProblems probs, int32_t* status, int split, int bsplit) {
  extern __shared__ __align__(1024) unsigned char tsm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ float bn_s[TC_N];
  const TcProblem pr = probs.p[blockIdx.z];
  const int n0 = blockIdx.x * TC_N;
  if (n0 >= pr.nb) return;
  const int a0 = blockIdx.y * TC_M;
  const int nt = min(TC_N, (pr.nb - n0 + 31) & ~31);  // tile columns: MMA N, a multiple of 32
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int kpad = pr.kpad, KB = kpad >> 3;
  unsigned char* sA = tsm;
  unsigned char* sB = tsm + TC_M * kpad * 2;
  unsigned char* sA2 = sB + TC_N * kpad * 2;  // split planes of A (when `split`)
  unsigned char* sA3 = sA2 + TC_M * kpad * 2;
  unsigned char* sB2 = split ? sA3 + TC_M * kpad * 2 : sA2;  // second plane of B (when `bsplit`)
  int bad = 0;
  // query slices, four values per step (float4 loads when aligned; kpad is a
  // multiple of 16): the BF16 value, and with `split` the next two planes
  const bool vec4 = ((pr.dim | lda | pr.a_off) & 3) == 0;
  const int q4 = kpad >> 2;
  auto pack = [](const __nv_bfloat16* b) {
    uint2 pk;
    pk.x = (uint32_t)__bfloat16_as_ushort(b[0]) | ((uint32_t)__bfloat16_as_ushort(b[1]) << 16);
    pk.y = (uint32_t)__bfloat16_as_ushort(b[2]) | ((uint32_t)__bfloat16_as_ushort(b[3]) << 16);
    return pk;
  };
  // four steps' loads are issued before any of them is converted and stored
  constexpr int GL = 4;
  for (int e0 = tid; e0 < TC_M * q4; e0 += 128 * GL) {
    float v[GL][4];
#pragma unroll
    for (int g = 0; g < GL; ++g) {
      const int e = e0 + g * 128;
      const int r = e / q4, k = (e - r * q4) << 2;
#pragma unroll
      for (int j = 0; j < 4; ++j) v[g][j] = 0.f;
      if (e < TC_M * q4 && a0 + r < na) {
        const float* src = A + (int64_t)(a0 + r) * lda + pr.a_off + k;
        if (vec4) {
          if (k < pr.dim) {
            const float4 f = *reinterpret_cast<const float4*>(src);
            v[g][0] = f.x;
            v[g][1] = f.y;
            v[g][2] = f.z;
            v[g][3] = f.w;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j) v[g][j] = k + j < pr.dim ? src[j] : 0.f;
        }
      }
    }
#pragma unroll
    for (int g = 0; g < GL; ++g) {
      const int e = e0 + g * 128;
      if (e >= TC_M * q4) break;
      const int r = e / q4, k = (e - r * q4) << 2;
      __nv_bfloat16 b1[4], b2[4], b3[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        b1[j] = __float2bfloat16_rn(v[g][j]);
        const float r1 = __fsub_rn(v[g][j], __bfloat162float(b1[j]));
        bad |= r1 != 0.f;
        b2[j] = __float2bfloat16_rn(r1);
        b3[j] = __float2bfloat16_rn(__fsub_rn(r1, __bfloat162float(b2[j])));
      }
      *reinterpret_cast<uint2*>(sA + core_off(r, k, KB)) = pack(b1);
      if (split) {
        *reinterpret_cast<uint2*>(sA2 + core_off(r, k, KB)) = pack(b2);
        *reinterpret_cast<uint2*>(sA3 + core_off(r, k, KB)) = pack(b3);
      }
    }
  }
  const int bpl = (pr.b_planes == 2 && !bsplit) ? 0 : pr.b_planes;  // a second plane needs its smem
  {  // codewords: one 16-byte core row per step (and the second plane)
    const int q8 = kpad >> 3;
    for (int e0 = tid; e0 < nt * q8; e0 += 128 * GL) {
      uint4 v[GL], v2[GL];
#pragma unroll
      for (int g = 0; g < GL; ++g) {
        const int e = e0 + g * 128;
        const int r = e / q8, k = (e - r * q8) << 3;
        v[g] = make_uint4(0u, 0u, 0u, 0u);
        v2[g] = make_uint4(0u, 0u, 0u, 0u);
        if (e < nt * q8 && n0 + r < pr.nb) {
          v[g] = *reinterpret_cast<const uint4*>(pr.Bb + (int64_t)(n0 + r) * kpad + k);
          if (bpl == 2) v2[g] = *reinterpret_cast<const uint4*>(pr.Bb2 + (int64_t)(n0 + r) * kpad + k);
        }
      }
#pragma unroll
      for (int g = 0; g < GL; ++g) {
        const int e = e0 + g * 128;
        if (e >= nt * q8) break;
        const int r = e / q8, k = (e - r * q8) << 3;
        *reinterpret_cast<uint4*>(sB + core_off(r, k, KB)) = v[g];
        if (bpl == 2) *reinterpret_cast<uint4*>(sB2 + core_off(r, k, KB)) = v2[g];
      }
    }
  }
  for (int c = tid; c < nt; c += 128) bn_s[c] = n0 + c < pr.nb ? pr.bn[n0 + c] : 0.f;
  bad = __syncthreads_or(bad);
  // A inexact (real-valued queries): three planes when the launch allows them; B in
  // one or two exact planes; otherwise the CUDA cores
  const bool use_split = bad && split && bpl > 0;
  bad = (bad && !use_split) || bpl == 0;
  const int planes = use_split ? 3 : 1;
  const int row = warp * 32 + lane, ga = a0 + row;
  bool done = false;
  if (!bad) {
    const uint32_t ncols = nt <= 32 ? 32u : (nt <= 64 ? 64u : (nt <= 128 ? 128u : 256u));
    if (warp == 0) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                   "r"(ncols));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
      asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tm = tmem_base;
    // D FP32 (bits 4-5), A and B BF16 (bits 7-9, 10-12), both K-major, N >> 3 (bits 17-22), M >> 4 (bits 24-28)
    const uint32_t idesc =
        (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(nt >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
    if (tid == 0) {
      for (int pl = 0; pl < planes; ++pl) {
        const unsigned char* ap = pl == 0 ? sA : (pl == 1 ? sA2 : sA3);
        for (int pb = 0; pb < bpl; ++pb) {
          const unsigned char* bp = pb == 0 ? sB : sB2;
          for (int kk = 0; kk < kpad / 16; ++kk) {
            const uint64_t ad = smem_desc(smem_u32(ap) + kk * 256, 128, KB * 128);
            const uint64_t bd = smem_desc(smem_u32(bp) + kk * 256, 128, KB * 128);
            asm volatile(
                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                ::"r"(tm), "l"(ad), "l"(bd), "r"(idesc), "r"((pl > 0 || pb > 0 || kk > 0) ? 1u : 0u));
          }
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&mbar)));
    }
    // bounded: an MMA group takes microseconds
    done = __syncthreads_and(mbar_wait_bounded(&mbar, 0, 1 << 24));
    if (!done) {
      // the wait gave up: report it, and give the MMA a second bounded wait before
      // the tensor memory it writes is released; the tile is then recomputed on
      // the CUDA cores below
      if (tid == 0 && status) atomicOr(status, STATUS_TIMEOUT);
      __syncthreads_and(mbar_wait_bounded(&mbar, 0, 1 << 24));
    }
    if (done) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      float an = 0.f;
      if (MODE == MODE_SQ) {
        if (use_split) {  // ||a||^2 of the FP32 row
          if (ga < na)
            for (int k = 0; k < pr.dim; ++k) {
              const float v = A[(int64_t)ga * lda + pr.a_off + k];
              an = fmaf(v, v, an);
            }
        } else {
          for (int k = 0; k < pr.dim; ++k) {
            const float v = __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(sA + core_off(row, k, KB)));
            an = fmaf(v, v, an);
          }
        }
      }
      const bool vec = ((pr.ldo | pr.o_off) & 3) == 0;
      for (int c0 = 0; c0 < nt; c0 += 32) {
        uint32_t r[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
              "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(tm + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        if (ga < na) {
          float* o = pr.out + (int64_t)ga * pr.ldo + pr.o_off + n0 + c0;
          float v[32];
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const float bn = bn_s[c0 + j];
            const float d2 = 2.f * __uint_as_float(r[j]);
            v[j] = (MODE == MODE_SQ) ? __fsub_rn(__fadd_rn(an, bn), d2) : __fsub_rn(bn, d2);
          }
          if (vec && n0 + c0 + 32 <= pr.nb) {
#pragma unroll
            for (int j = 0; j < 32; j += 4) *reinterpret_cast<float4*>(o + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (n0 + c0 + j < pr.nb) o[j] = v[j];
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(ncols));
  }
  if (!done && ga < na) {  // FP32 on the CUDA cores: sum (a - b)^2, or sum b (b - 2a)
    const float* a = A + (int64_t)ga * lda + pr.a_off;
    for (int b = n0; b < min(pr.nb, n0 + nt); ++b) {
      const float* bb = pr.B + (int64_t)b * pr.dim;
      float acc = 0.f;
      for (int d = 0; d < pr.dim; ++d) {
        if (MODE == MODE_SQ) {
          const float t = a[d] - bb[d];
          acc = fmaf(t, t, acc);
        } else {
          acc = fmaf(bb[d], fmaf(-2.f, a[d], bb[d]), acc);
        }
      }
      pr.out[(int64_t)ga * pr.ldo + pr.o_off + b] = acc;
    }
  }
}

// BF16 copy (K padded to kpad) and squared norms of n rows of dim floats; sets
// *inexact if a value is not exactly representable in BF16.
__global__ void bf16_rows_kernel(const float* __restrict__ X, int64_t n, int dim, int kpad,
                                 __nv_bfloat16* __restrict__ Xb, float* __restrict__ norms, int* inexact,
                                 __nv_bfloat16* __restrict__ Xb2, int* inexact2) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  float s = 0.f;
  int bad = 0, bad2 = 0;
  for (int k = 0; k < kpad; ++k) {
    const float v = k < dim ? X[r * dim + k] : 0.f;
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    const float rest = __fsub_rn(v, __bfloat162float(b));
    const __nv_bfloat16 b2 = __float2bfloat16_rn(rest);
    bad |= __bfloat162float(b) != v;
    bad2 |= __bfloat162float(b2) != rest;
    Xb[r * kpad + k] = b;
    Xb2[r * kpad + k] = b2;
    s = fmaf(v, v, s);
  }
  norms[r] = s;
  if (bad) atomicExch(inexact, 1);
  if (bad2) atomicExch(inexact2, 1);
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

// bpq_search_shortlist step 1: per query, lo_k = min_t lut[k][t] and the
// widest shifted table range = max_k (max_t lut[k][t] - lo_k), all in IEEE FP32.
//  int8: step s = range / 255 (1 if range is 0), q8[k][t] = round_half_even((lut[k][t] - lo_k) / s);
//  fp16: step s = the smallest power of two >= 1 with range <= 65504 s (exact scaling),
//        h[k][t] = the FP16 value nearest to (lut[k][t] - lo_k) / s (ties to even).
template <int M, bool F16>
__global__ void __launch_bounds__(256) quant_lut_kernel(const float* __restrict__ lut, int64_t nq,
                                                        void* __restrict__ out, float* __restrict__ scale) {
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
    float s;
    if (F16) {
      s = 1.f;
      while (range > __fmul_rn(65504.f, s)) s = __fmul_rn(s, 2.f);  // range is finite: at most 128 doublings
    } else {
      s = range > 0.f ? __fdiv_rn(range, 255.f) : 1.f;
    }
    for (int e = threadIdx.x; e < M * KSUB; e += 256) {
      const float x = __fsub_rn(L[e], lo_s[e / KSUB]);
      if (F16) {
        static_cast<uint16_t*>(out)[q * M * KSUB + e] = __half_as_ushort(__float2half_rn(__fdiv_rn(x, s)));
      } else {
        const int v = __float2int_rn(__fdiv_rn(x, s));
        static_cast<uint8_t*>(out)[q * M * KSUB + e] = (uint8_t)min(255, max(0, v));
      }
    }
    if (threadIdx.x == 0) scale[q] = s;
  }
}

}  // namespace

void launch_quant_lut(const float* lut, int M, int64_t nq, void* out, float* scale, bool f16, cudaStream_t st) {
  if (nq <= 0) return;
  const int grid = (int)std::min<int64_t>(nq, 1 << 20);
  if (M == 8 && f16) quant_lut_kernel<8, true><<<grid, 256, 0, st>>>(lut, nq, out, scale);
  else if (M == 8) quant_lut_kernel<8, false><<<grid, 256, 0, st>>>(lut, nq, out, scale);
  else if (M == 16 && f16) quant_lut_kernel<16, true><<<grid, 256, 0, st>>>(lut, nq, out, scale);
  else if (M == 16) quant_lut_kernel<16, false><<<grid, 256, 0, st>>>(lut, nq, out, scale);
  else throw Error(BPQ_EINVAL, "the reduced-precision table is built for M = 8 or 16");
  check_launch("table quantization kernel");
}

void launch_query_tables(const bpq_index& ix, const float* q, int64_t nq, float* d1, float* d2,
                         float* lut, cudaStream_t st, int32_t* status, const float* q_lut) {
  if (!q_lut) q_lut = q;
  if (nq <= 0) return;
  const int D = ix.p.D, T = ix.p.T, M = ix.p.M;
  const int ty = (int)((nq + TC_M - 1) / TC_M);
  BPQ_CHECK(nq < (int64_t)65535 * TC_M, BPQ_EINVAL, "too many queries in one table launch");
  if (d1 || d2) {
    TcProblems pp{};
    int np = 0;
    const int bp = ix.coarse_bf16_exact ? 1 : (ix.coarse_bf16x2_exact ? 2 : 0);
    if (d1)
      pp.p[np++] = TcProblem{ix.C1b.as<__nv_bfloat16>(), ix.C1.as<float>(), ix.n1.as<float>(), d1, 0, T, ix.h, ix.kh,
                             T, 0, bp, ix.C1b2.as<__nv_bfloat16>()};
    if (d2)
      pp.p[np++] = TcProblem{ix.C2b.as<__nv_bfloat16>(), ix.C2.as<float>(), ix.n2.as<float>(), d2, ix.h, T, ix.h,
                             ix.kh, T, 0, bp, ix.C2b2.as<__nv_bfloat16>()};
    // the split planes of real-valued queries (OPQ) and the codewords' second plane,
    // when they fit beside the operands
    const size_t base = (size_t)(TC_M + TC_N) * ix.kh * 2, planes = (size_t)2 * TC_M * ix.kh * 2;
    const size_t bplane = bp == 2 ? (size_t)TC_N * ix.kh * 2 : 0;
    const int split = ix.opq && base + planes + bplane <= 220 * 1024;
    const int bsplit = bp == 2 && base + (split ? planes : 0) + bplane <= 220 * 1024;
    const size_t smem = base + (split ? planes : 0) + (bsplit ? bplane : 0);
    BPQ_CUDA(cudaFuncSetAttribute(tc_table_kernel<MODE_SQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((T + TC_N - 1) / TC_N, ty, np);
    tc_table_kernel<MODE_SQ><<<grid, 128, smem, st>>>(q, D, (int)nq, pp, status, split, bsplit);
    check_launch("coarse table kernel");
  }
  if (lut) {
    BPQ_CHECK(M <= MAXP, BPQ_EINVAL, "M too large for the table kernel");
    TcProblems pp{};
    const int bp = ix.R_bf16_exact ? 1 : (ix.R_bf16x2_exact ? 2 : 0);
    for (int k = 0; k < M; ++k)
      pp.p[k] = TcProblem{ix.Rb.as<__nv_bfloat16>() + (int64_t)k * KSUB * ix.ks, ix.R.as<float>() + (int64_t)k * KSUB * ix.s,
                          ix.nR.as<float>() + (int64_t)k * KSUB, lut, k * ix.s, KSUB, ix.s, ix.ks, M * KSUB, k * KSUB,
                          bp, ix.Rb2.as<__nv_bfloat16>() + (int64_t)k * KSUB * ix.ks};
    const size_t base = (size_t)(TC_M + TC_N) * ix.ks * 2, planes = (size_t)2 * TC_M * ix.ks * 2;
    const size_t bplane = bp == 2 ? (size_t)TC_N * ix.ks * 2 : 0;
    const int split = ix.opq && base + planes + bplane <= 220 * 1024;
    const int bsplit = bp == 2 && base + (split ? planes : 0) + bplane <= 220 * 1024;
    const size_t smem = base + (split ? planes : 0) + (bsplit ? bplane : 0);
    BPQ_CUDA(cudaFuncSetAttribute(tc_table_kernel<MODE_LUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid(1, ty, M);
    tc_table_kernel<MODE_LUT><<<grid, 128, smem, st>>>(q_lut, D, (int)nq, pp, status, split, bsplit);
    check_launch("pq table kernel");
  }
}

void build_fbpq_tables(bpq_index& ix, cudaStream_t st) {
  const int T = ix.p.T;
  const int64_t n = (int64_t)T * ix.m2 * KSUB;
  ix.X1.alloc(n * sizeof(float));
  ix.X2.alloc(n * sizeof(float));
  const int blocks = (int)((n + 255) / 256);
  // with OPQ the dot products of Eq. 9 are in the residual space: rotated centroids B c
  const float* c1 = ix.opq ? ix.C1r.as<float>() : ix.C1.as<float>();
  const float* c2 = ix.opq ? ix.C2r.as<float>() : ix.C2.as<float>();
  cross_table_kernel<<<blocks, 256, 0, st>>>(c1, ix.R.as<float>(), T, ix.m2, ix.s, ix.h, 0, ix.X1.as<float>());
  cross_table_kernel<<<blocks, 256, 0, st>>>(c2, ix.R.as<float>(), T, ix.m2, ix.s, ix.h, ix.m2, ix.X2.as<float>());
  check_launch("fbpq cross table kernel");
  // tensor-core operands of the query tables
  ix.kh = (ix.h + 15) & ~15;
  ix.ks = (ix.s + 15) & ~15;
  BPQ_CHECK(ix.kh <= 192 && ix.ks <= 64, BPQ_EINVAL, "table operand widths: D/2 <= 192 and D/M <= 64");
  const int64_t nR = (int64_t)ix.p.M * KSUB;
  ix.C1b.alloc((size_t)T * ix.kh * 2);
  ix.C2b.alloc((size_t)T * ix.kh * 2);
  ix.Rb.alloc((size_t)nR * ix.ks * 2);
  ix.C1b2.alloc((size_t)T * ix.kh * 2);
  ix.C2b2.alloc((size_t)T * ix.kh * 2);
  ix.Rb2.alloc((size_t)nR * ix.ks * 2);
  ix.n1.alloc((size_t)T * 4);
  ix.n2.alloc((size_t)T * 4);
  ix.nR.alloc((size_t)nR * 4);
  DevBuf flags;
  flags.alloc(16);
  BPQ_CUDA(cudaMemsetAsync(flags.p, 0, 16, st));
  int* fl = flags.as<int>();  // [coarse, R] one plane inexact, [coarse, R] two planes inexact
  bf16_rows_kernel<<<(T + 255) / 256, 256, 0, st>>>(ix.C1.as<float>(), T, ix.h, ix.kh, ix.C1b.as<__nv_bfloat16>(),
                                                    ix.n1.as<float>(), fl, ix.C1b2.as<__nv_bfloat16>(), fl + 2);
  bf16_rows_kernel<<<(T + 255) / 256, 256, 0, st>>>(ix.C2.as<float>(), T, ix.h, ix.kh, ix.C2b.as<__nv_bfloat16>(),
                                                    ix.n2.as<float>(), fl, ix.C2b2.as<__nv_bfloat16>(), fl + 2);
  bf16_rows_kernel<<<(int)((nR + 255) / 256), 256, 0, st>>>(ix.R.as<float>(), nR, ix.s, ix.ks,
                                                            ix.Rb.as<__nv_bfloat16>(), ix.nR.as<float>(), fl + 1,
                                                            ix.Rb2.as<__nv_bfloat16>(), fl + 3);
  check_launch("table operand kernel");
  int h_fl[4] = {1, 1, 1, 1};
  BPQ_CUDA(cudaMemcpyAsync(h_fl, fl, 16, cudaMemcpyDeviceToHost, st));
  BPQ_CUDA(cudaStreamSynchronize(st));
  ix.coarse_bf16_exact = h_fl[0] == 0;
  ix.R_bf16_exact = h_fl[1] == 0;
  ix.coarse_bf16x2_exact = h_fl[2] == 0;
  ix.R_bf16x2_exact = h_fl[3] == 0;
}

}  // namespace bpq
