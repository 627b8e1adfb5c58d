// HBPQ per-half-cell lookup tables (§3.2, Eqs. 10-12), built for the half-cells
// that the queries of a batch visit, as one grouped tensor-core contraction per
// half-cell.
//
// The HBPQ distance of a point with code [c_1 .. c_M] in cell (i, j) -- the
// reconstruction with the local codebooks Q^i_k, S^j_k of §3.2 -- regroups exactly:
//   ||q - xhat||^2 = d1[i] + d2[j] + sum_{k<M/2} A_i[k][c_k] + sum_{k<M/2} B_j[k][c_{M/2+k}]
//   A_i[k][t] = E1[i][k][t] - 2 <q_k, Q^i_k[t]>,   E1[i][k][t] = ||Q^i_k[t]||^2 + 2 <c^1_i|k, Q^i_k[t]>
// (B_j likewise with S^j, c^2_j and the second half of q; c^1_i|k is block k of
// c^1_i).  A candidate then costs M table lookups instead of the O(D) distance of
// the paper's HBPQ.  E1 and E2 are query-independent and built with the index; the
// query terms <q_k, Q^i_k[t]> of every (query, visited half-cell) pair are one BF16
// tcgen05 MMA per sub-quantizer over a tile of the queries that visit the
// half-cell (M = 128 queries, N = 256 codewords, K = D/M = 16), FP32 accumulation
// in tensor memory.  Queries and codebooks on the integer grid (|v| <= 256) are
// exact in BF16 and every product and partial sum is an integer below 2^24, so
// the tables equal the FP64 definition exactly; a tile whose operands BF16 cannot
// hold, and every shape with D/M != 16, is tabulated in FP32 on the CUDA cores.
//
// Per search chunk:
//  1. hbpq_pairs_kernel (one warp per query): the distinct rows i and columns j of
//     the query's visited cells, as bitmaps; table slots base .. base + R + C - 1
//     (rows in increasing i, then columns in increasing j) are taken from a
//     counter; a query whose slots do not fit the table area is listed for the
//     O(D) reconstruction scan instead.  Each (query, half-cell) pair sets the
//     query's bit in the half-cell's bitmap of visiting queries.
//  2. hbpq_table_kernel (one CTA per half-cell and half): walks that bitmap in
//     tiles of 128 queries and writes their tables to their slots.
#include <cuda_bf16.h>

#include <algorithm>

#include "bpq_internal.cuh"

namespace bpq {
namespace {

// BF16 copies (K padded with zeros to ks) of the local codebooks and the
// query-independent table terms E[i][k][t] = ||W[t]||^2 + 2 <c_i|k, W[t]> with
// W = Q^i_k (or S^j_k): one thread per codeword row (i, k, t).
__global__ void hbpq_operand_kernel(const float* __restrict__ W, const float* __restrict__ C, int64_t nrows,
                                    int m2, int s, int ks, int H, __nv_bfloat16* __restrict__ Wb,
                                    float* __restrict__ E, int* inexact) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  const int64_t i = r / ((int64_t)m2 * KSUB);
  const int k = (int)((r / KSUB) % m2);
  const float* w = W + r * s;
  const float* c = C + i * H + k * s;
  float nrm = 0.f, dot = 0.f;
  int bad = 0;
  for (int d = 0; d < ks; ++d) {
    const float v = d < s ? w[d] : 0.f;
    const __nv_bfloat16 b = __float2bfloat16_rn(v);
    bad |= __bfloat162float(b) != v;
    Wb[r * ks + d] = b;
    if (d < s) {
      nrm = fmaf(v, v, nrm);
      dot = fmaf(c[d], v, dot);
    }
  }
  E[r] = __fadd_rn(nrm, 2.f * dot);
  if (bad) atomicExch(inexact, 1);
}

constexpr int PAIR_WARPS = 4;

__global__ void __launch_bounds__(PAIR_WARPS * 32) hbpq_pairs_kernel(HbpqArgs h) {
  __shared__ uint32_t bits_s[PAIR_WARPS][2][MAX_T / 32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t q = (int64_t)blockIdx.x * PAIR_WARPS + w;
  if (q >= h.nq) return;  // uniform over the warp; no block barrier follows
  const int T = h.T, TW = (T + 31) >> 5;
  uint32_t* rb = bits_s[w][0];
  uint32_t* cb = bits_s[w][1];
  for (int x = lane; x < TW; x += 32) {
    rb[x] = 0u;
    cb[x] = 0u;
  }
  __syncwarp();
  const int nc = max(0, h.ncells[q]);
  const bpq_cell* cl = h.cells + q * (int64_t)h.cap;
  for (int c = lane; c < nc; c += 32) {
    const uint32_t cell = cl[c].cell;
    const uint32_t i = cell / (uint32_t)T, j = cell - i * (uint32_t)T;
    atomicOr(&rb[i >> 5], 1u << (i & 31));
    atomicOr(&cb[j >> 5], 1u << (j & 31));
  }
  __syncwarp();
  int R = 0, C = 0;
  for (int x = lane; x < TW; x += 32) {
    R += __popc(rb[x]);
    C += __popc(cb[x]);
  }
  R = warp_sum(R);
  C = warp_sum(C);
  long long base = 0;
  if (lane == 0) {
    base = (long long)atomicAdd(h.slot_counter, (unsigned long long)(R + C));
    if (base + R + C > h.slot_cap) {
      base = -1;
      h.fallback[atomicAdd(h.fb_count, 1)] = (int32_t)q;
    }
    h.qbase[q] = (int32_t)base;
    h.qrows[q] = R;
  }
  base = __shfl_sync(0xffffffffu, base, 0);
  if (base < 0) return;
  uint32_t* qb = h.qbits + q * 2 * TW;
  for (int x = lane; x < TW; x += 32) {
    qb[x] = rb[x];
    qb[TW + x] = cb[x];
  }
  const int64_t QW = (h.nq + 31) >> 5;
  const uint32_t qbit = 1u << (q & 31);
  const int64_t qw = q >> 5;
  for (int x = lane; x < TW; x += 32) {
    for (uint32_t m = rb[x]; m; m &= m - 1u)
      atomicOr(&h.hmap[(int64_t)(x * 32 + __ffs(m) - 1) * QW + qw], qbit);
    for (uint32_t m = cb[x]; m; m &= m - 1u)
      atomicOr(&h.hmap[((int64_t)T + x * 32 + __ffs(m) - 1) * QW + qw], qbit);
  }
}

// Exclusive scan of one int per thread over a block of 128 threads; *total gets
// the sum.  tmp: 5 ints of shared memory.
__device__ int excl_scan128(int x, int* tmp, int* total) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  int v = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, v, o);
    if (l >= o) v += y;
  }
  __syncthreads();
  if (l == 31) tmp[w] = v;
  __syncthreads();
  int before = 0;
#pragma unroll
  for (int x2 = 0; x2 < 4; ++x2) before += (x2 < w) ? tmp[x2] : 0;
  *total = tmp[0] + tmp[1] + tmp[2] + tmp[3];
  return before + v - x;
}

struct TabArgs {
  HbpqArgs h;
  const __nv_bfloat16* Wb[2];  // Qb, Sb: T x M/2 x 256 x 16
  const float* W[2];           // Q, S: T x M/2 x 256 x D/M (FP32)
  const float* E[2];           // E1, E2: T x M/2 x 256
  int m2, s, H;
  int tensor;                  // 1: tcgen05 path allowed (D/M == 16, exact BF16 codebooks)
};

constexpr int HT_M = 128;   // queries per tile (MMA M)
constexpr int HT_N = 256;   // codewords per sub-quantizer (MMA N)
constexpr int HT_COLS = 256;  // tensor-memory columns: one sub-quantizer's 128 x 256 FP32 block

__global__ void __launch_bounds__(128) hbpq_table_kernel(TabArgs a) {
  extern __shared__ __align__(1024) unsigned char hsm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int32_t tq[HT_M];
  __shared__ int64_t tslot[HT_M];
  __shared__ int scan_tmp[5];
  const HbpqArgs& h = a.h;
  const int i = blockIdx.x, half = blockIdx.y;
  const int T = h.T, m2 = a.m2, s = a.s, H = a.H, TW = (T + 31) >> 5;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t QW = (h.nq + 31) >> 5;
  const uint32_t* bm = h.hmap + ((int64_t)half * T + i) * QW;
  {  // any visiting query?
    int mine = 0;
    for (int64_t x = tid; x < QW; x += 128) mine |= bm[x] != 0u;
    if (!__syncthreads_or(mine)) return;
  }

  const int KBA = H >> 3;                      // A: 128 x H BF16, column groups of 8
  unsigned char* sA = hsm;                     // HT_M * H * 2 bytes
  unsigned char* sB = sA + HT_M * H * 2;       // m2 x (256 x 16 BF16) = m2 x 8 KB
  float* Es = reinterpret_cast<float*>(sB + (a.tensor ? m2 * HT_N * 32 : 0));  // m2 x 256
  float* stage = Es + m2 * KSUB + warp * (32 * 33);  // per warp: 32 rows x 32 columns (+1 pad)
  const float* E = a.E[half] + (int64_t)i * m2 * KSUB;
  for (int e = tid; e < m2 * KSUB; e += 128) Es[e] = E[e];
  bool tc = a.tensor != 0;
  if (tc) {
    // B operand of sub-quantizer k: 256 codewords x 16 BF16, one 16-byte core row per step
    const __nv_bfloat16* Wb = a.Wb[half] + (int64_t)i * m2 * KSUB * 16;
    for (int e = tid; e < m2 * KSUB * 2; e += 128) {
      const int row = e >> 1, kc = (e & 1) << 3;  // row = k * 256 + t
      const int k = row >> 8, t = row & 255;
      *reinterpret_cast<uint4*>(sB + k * (HT_N * 32) + core_off(t, kc, 2)) =
          *reinterpret_cast<const uint4*>(Wb + (int64_t)row * 16 + kc);
    }
    if (warp == 0) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                   "r"((uint32_t)HT_COLS));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
      asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
  }
  __syncthreads();
  if (tc) asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tm = tc ? tmem_base : 0u;
  // D FP32 (bits 4-5), A and B BF16 (bits 7-9, 10-12), both K-major, N >> 3 (bits 17-22), M >> 4 (bits 24-28)
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(HT_N >> 3) << 17) |
                         ((uint32_t)(HT_M >> 4) << 24);
  uint32_t phase = 0;
  const float* Wf = a.W[half] + (int64_t)i * m2 * KSUB * s;
  const int r = tid;  // tile row of this thread = tensor-memory lane

  for (int64_t w0 = 0; w0 < QW; w0 += 128) {
    const uint32_t word = (w0 + tid < QW) ? bm[w0 + tid] : 0u;
    int total;
    const int ex = excl_scan128(__popc(word), scan_tmp, &total);
    for (int ts = 0; ts < total; ts += HT_M) {
      const int nt = min(HT_M, total - ts);
      __syncthreads();  // the previous tile's rows are no longer read
      {
        int p = ex;
        for (uint32_t m = word; m; m &= m - 1u, ++p)
          if (p >= ts && p < ts + HT_M) tq[p - ts] = (int32_t)((w0 + tid) * 32 + __ffs(m) - 1);
      }
      __syncthreads();
      int bad = 0;
      if (r < nt) {
        const int64_t q = tq[r];
        const uint32_t* bits = h.qbits + q * 2 * TW + half * TW;
        int rank = __popc(bits[i >> 5] & ((1u << (i & 31)) - 1u));
        for (int x = 0; x < (i >> 5); ++x) rank += __popc(bits[x]);
        tslot[r] = (int64_t)h.qbase[q] + (half ? h.qrows[q] : 0) + rank;
        if (tc) {  // query half as BF16 rows of A
          const float* qv = h.queries + q * h.D + half * H;
          for (int d = 0; d < H; d += 4) {
            const float4 v = *reinterpret_cast<const float4*>(qv + d);
            const __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
            bad |= __low2float(lo) != v.x || __high2float(lo) != v.y || __low2float(hi) != v.z ||
                   __high2float(hi) != v.w;
            uint2 pk;
            pk.x = *reinterpret_cast<const uint32_t*>(&lo);
            pk.y = *reinterpret_cast<const uint32_t*>(&hi);
            *reinterpret_cast<uint2*>(sA + core_off(r, d, KBA)) = pk;
          }
        }
      }
      if (tc) asm volatile("fence.proxy.async.shared::cta;");
      bad = __syncthreads_or(bad);
      bool done = false;
      if (tc && !bad) {
        done = true;
        for (int k = 0; k < m2 && done; ++k) {
          asm volatile("tcgen05.fence::after_thread_sync;");
          if (tid == 0) {
            const uint64_t ad = smem_desc(smem_u32(sA) + k * 256, 128, KBA * 128);
            const uint64_t bd = smem_desc(smem_u32(sB) + k * (HT_N * 32), 128, 256);
            asm volatile(
                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tm),
                "l"(ad), "l"(bd), "r"(idesc), "r"(0u));
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&mbar)));
          }
          // bounded: one MMA takes well under a microsecond
          done = __syncthreads_and(mbar_wait_bounded(&mbar, phase, 1 << 24));
          if (!done) {
            // report, give the MMA a second bounded wait before its tensor memory is
            // released, and finish this batch on the CUDA cores
            if (tid == 0 && h.status) atomicOr(h.status, STATUS_TIMEOUT);
            __syncthreads_and(mbar_wait_bounded(&mbar, phase, 1 << 24));
            tc = false;
            break;
          }
          phase ^= 1u;
          asm volatile("tcgen05.fence::after_thread_sync;");
          for (int c0 = 0; c0 < HT_N; c0 += 32) {
            uint32_t v[32];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                  "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                  "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(tm + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            // lane = tile row: stage the 32 x 32 block, then write it row by row so
            // that each store instruction covers four whole 128-byte rows
#pragma unroll
            for (int j = 0; j < 32; ++j) stage[lane * 33 + j] = __uint_as_float(v[j]);
            __syncwarp();
            const float* e = Es + k * KSUB + c0 + (lane & 7) * 4;
#pragma unroll
            for (int rr = 0; rr < 32; rr += 4) {
              const int row = rr + (lane >> 3), trow = warp * 32 + row;
              if (trow < nt) {
                const float* sv = stage + row * 33 + (lane & 7) * 4;
                float4 o;
                o.x = __fsub_rn(e[0], 2.f * sv[0]);
                o.y = __fsub_rn(e[1], 2.f * sv[1]);
                o.z = __fsub_rn(e[2], 2.f * sv[2]);
                o.w = __fsub_rn(e[3], 2.f * sv[3]);
                *reinterpret_cast<float4*>(h.tables + tslot[trow] * (int64_t)(m2 * KSUB) + k * KSUB + c0 +
                                           (lane & 7) * 4) = o;
              }
            }
            __syncwarp();
          }
          // every lane's tensor-memory reads are complete before the next MMA writes
          asm volatile("tcgen05.fence::before_thread_sync;");
          __syncthreads();
        }
      }
      if (!done && r < nt) {  // FP32 on the CUDA cores: E - 2 <q_k, W[t]>
        const float* qv = h.queries + (int64_t)tq[r] * h.D + half * H;
        float* out = h.tables + tslot[r] * (int64_t)(m2 * KSUB);
        for (int k = 0; k < m2; ++k)
          for (int t = 0; t < KSUB; ++t) {
            const float* wv = Wf + ((int64_t)k * KSUB + t) * s;
            float acc = 0.f;
            for (int d = 0; d < s; ++d) acc = fmaf(qv[k * s + d], wv[d], acc);
            out[k * KSUB + t] = __fsub_rn(Es[k * KSUB + t], 2.f * acc);
          }
      }
    }
  }
  if (a.tensor) {  // the allocation is held whether or not a wait gave up
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"((uint32_t)HT_COLS));
  }
}

}  // namespace

bool hbpq_tensor_shape(const bpq_index& ix) { return ix.s == 16 && ix.m2 <= 8; }

void build_hbpq_tables(bpq_index& ix, cudaStream_t st) {
  if (ix.p.variant != BPQ_VARIANT_LOCAL) return;
  const int T = ix.p.T, m2 = ix.m2, s = ix.s;
  const int ks = (s + 15) & ~15;
  const int64_t nrows = (int64_t)T * m2 * KSUB;
  ix.Qb.alloc((size_t)nrows * ks * 2);
  ix.Sb.alloc((size_t)nrows * ks * 2);
  ix.E1.alloc((size_t)nrows * 4);
  ix.E2.alloc((size_t)nrows * 4);
  DevBuf flag;
  flag.alloc(4);
  BPQ_CUDA(cudaMemsetAsync(flag.p, 0, 4, st));
  const int blocks = (int)((nrows + 255) / 256);
  hbpq_operand_kernel<<<blocks, 256, 0, st>>>(ix.Q.as<float>(), ix.C1.as<float>(), nrows, m2, s, ks, ix.h,
                                              ix.Qb.as<__nv_bfloat16>(), ix.E1.as<float>(), flag.as<int>());
  hbpq_operand_kernel<<<blocks, 256, 0, st>>>(ix.S.as<float>(), ix.C2.as<float>(), nrows, m2, s, ks, ix.h,
                                              ix.Sb.as<__nv_bfloat16>(), ix.E2.as<float>(), flag.as<int>());
  check_launch("hbpq operand kernel");
  int h_flag = 1;
  BPQ_CUDA(cudaMemcpyAsync(&h_flag, flag.p, 4, cudaMemcpyDeviceToHost, st));
  BPQ_CUDA(cudaStreamSynchronize(st));
  ix.local_bf16_exact = h_flag == 0;
}

void launch_hbpq_pairs(const HbpqArgs& h, cudaStream_t st) {
  if (h.nq <= 0) return;
  BPQ_CHECK(h.T <= MAX_T, BPQ_EINVAL, "T too large for the HBPQ pair kernel");
  const int64_t grid = (h.nq + PAIR_WARPS - 1) / PAIR_WARPS;
  BPQ_CHECK(grid < (1LL << 31), BPQ_EINVAL, "too many queries in one HBPQ chunk");
  hbpq_pairs_kernel<<<(unsigned)grid, PAIR_WARPS * 32, 0, st>>>(h);
  check_launch("hbpq pair kernel");
}

void launch_hbpq_tables(const bpq_index& ix, const HbpqArgs& h, cudaStream_t st) {
  if (h.nq <= 0) return;
  TabArgs a{};
  a.h = h;
  a.Wb[0] = ix.Qb.as<__nv_bfloat16>();
  a.Wb[1] = ix.Sb.as<__nv_bfloat16>();
  a.W[0] = ix.Q.as<float>();
  a.W[1] = ix.S.as<float>();
  a.E[0] = ix.E1.as<float>();
  a.E[1] = ix.E2.as<float>();
  a.m2 = ix.m2;
  a.s = ix.s;
  a.H = ix.h;
  a.tensor = (hbpq_tensor_shape(ix) && ix.local_bf16_exact && (ix.p.D & 3) == 0 &&
              (reinterpret_cast<uintptr_t>(h.queries) & 15) == 0) ? 1 : 0;
  const size_t smem = (size_t)HT_M * ix.h * 2 + (a.tensor ? (size_t)ix.m2 * HT_N * 32 : 0) + (size_t)ix.m2 * KSUB * 4 +
                      (size_t)4 * 32 * 33 * 4;
  BPQ_CHECK(smem <= 200 * 1024, BPQ_EINVAL, "HBPQ table kernel: shape too large for shared memory");
  BPQ_CUDA(cudaFuncSetAttribute(hbpq_table_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid(h.T, 2);
  hbpq_table_kernel<<<grid, 128, smem, st>>>(a);
  check_launch("hbpq table kernel");
}

}  // namespace bpq
