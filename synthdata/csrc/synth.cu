// Device copy of the seeded point generator of synthdata/__init__.py (counter-based
// SplitMix64 words, Irwin-Hall(4) draws, low-rank Gaussian mixture with integer
// tables).  It holds no arithmetic of the search method; it only lets large
// workloads be generated where they are used.  Produces the same bytes as the
// numpy generator (checked by the tests).
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr uint64_t GAMMA = 0x9E3779B97F4A7C15ull;
constexpr int NF = 16;  // latent factors
constexpr int SCALE = 166;
constexpr int NOISE = 8;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t word(uint64_t seedk, uint64_t stream, uint64_t n, uint64_t w) {
  const uint64_t ctr = (stream << 48) | (n << 8) | w;
  return mix64(seedk + (ctr + 1) * GAMMA);
}

__device__ __forceinline__ int irwin_hall(uint32_t half) {
  return (int)(half & 0xff) + (int)((half >> 8) & 0xff) + (int)((half >> 16) & 0xff) + (int)(half >> 24) - 510;
}

__device__ __forceinline__ long long floordiv(long long a, long long b) {
  long long q = a / b;
  if ((a % b != 0) && (a < 0)) --q;
  return q;
}

__global__ void points_kernel(const int32_t* __restrict__ mu, const int32_t* __restrict__ sigma,
                              const uint64_t* __restrict__ cum, const int32_t* __restrict__ B, int n_comp, int dim,
                              uint64_t seedk, uint64_t stream, int64_t start, int64_t count, float* out_f,
                              uint8_t* out_u8) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= count) return;
  const uint64_t n = (uint64_t)(start + p);
  const uint64_t r = word(seedk, stream, n, 0) >> 32;
  int lo = 0, hi = n_comp - 1;  // first c with cum[c] > r
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (cum[mid] > r) hi = mid; else lo = mid + 1;
  }
  const int c = lo;
  int lat[NF];
#pragma unroll
  for (int w = 0; w < NF / 2; ++w) {
    const uint64_t v = word(seedk, stream, n, 1 + w);
    lat[2 * w] = irwin_hall((uint32_t)v);
    lat[2 * w + 1] = irwin_hall((uint32_t)(v >> 32));
  }
  const long long sg = sigma[c];
  for (int d2 = 0; d2 < dim / 2; ++d2) {
    const uint64_t v = word(seedk, stream, n, 1 + NF / 2 + d2);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int d = 2 * d2 + h;
      const int e = irwin_hall(h ? (uint32_t)(v >> 32) : (uint32_t)v);
      long long acc = 0;
#pragma unroll
      for (int f = 0; f < NF; ++f) acc += (long long)B[d * NF + f] * lat[f];
      const long long a = sg * acc + (long long)NOISE * e;
      long long x = mu[(int64_t)c * dim + d] + floordiv(a + SCALE / 2, SCALE);
      x = x < 0 ? 0 : (x > 255 ? 255 : x);
      if (out_f) out_f[p * dim + d] = (float)x;
      if (out_u8) out_u8[p * dim + d] = (uint8_t)x;
    }
  }
}

}  // namespace

extern "C" int synth_points(const int32_t* mu, const int32_t* sigma, const uint64_t* cum, const int32_t* B,
                            int n_comp, int dim, uint64_t seedk, int stream, int64_t start, int64_t count,
                            float* out_f32, uint8_t* out_u8, void* cuda_stream) {
  if (count <= 0) return 0;
  const int threads = 128;
  const int64_t blocks = (count + threads - 1) / threads;
  points_kernel<<<(unsigned)blocks, threads, 0, (cudaStream_t)cuda_stream>>>(
      mu, sigma, cum, B, n_comp, dim, seedk, (uint64_t)stream, start, count, out_f32, out_u8);
  return (int)cudaGetLastError();
}
