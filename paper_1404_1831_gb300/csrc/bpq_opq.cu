// OPQ rotations (the "optimized" OMulti-D-OADC of §2.3; parametric OPQ learner).
//
// An OPQ index carries rot0 (D x D), applied to vectors before the coarse
// quantization, and rot1, rot2 (D/2 x D/2), applied to the two halves of the
// displacement before the residual PQ; B = blockdiag(rot1, rot2).  For a vector v
// the library works with v' = rot0 v (coarse space: cells and the keys d1, d2) and
// v~ = B rot0 v (residual space: PQ codes, the PQ table, the query displacement of
// the reconstruction scorer), and with the rotated coarse centroids B c (the FBPQ
// cross terms of Eq. 9).  All rotations are orthogonal, so every distance equals
// the distance to the reconstruction rot0^T (c + B^T r) in the original space.
//
// Learner (parametric OPQ): a rotation's rows are the eigenvectors of the data's
// covariance, dealt in descending eigenvalue order to the subspace (the two
// halves for rot0, the M/2 sub-quantizers of a half for rot1 / rot2) with the
// smallest sum of log eigenvalues so far (ties to the lower subspace); each
// eigenvector's largest-magnitude component is made positive.  Covariances are
// accumulated on the GPU in FP64 (exact for the integer inputs); the symmetric
// eigenproblem is solved on the host by cyclic Jacobi rotations.  The rotated
// learn vectors and displacements are rounded half up to the integer grid before
// K-means, so the codebooks stay integral in their spaces.
#include <algorithm>
#include <cmath>
#include <vector>

#include "bpq_internal.cuh"

namespace bpq {
namespace {

// S[a][b] += sum_p x_p[a] x_p[b], s1[a] += sum_p x_p[a] over rows p of X (n x ld, the
// d columns starting at col).  One CTA per 32 x 32 output tile and chunk of points.
constexpr int CT = 32;
__global__ void __launch_bounds__(256) cov_kernel(const float* __restrict__ X, int64_t n, int64_t ld, int col, int d,
                                                  int64_t chunk, double* __restrict__ S, double* __restrict__ s1) {
  __shared__ float xa[CT][CT + 1];
  __shared__ float xb[CT][CT + 1];
  const int a0 = blockIdx.x * CT, b0 = blockIdx.y * CT;
  const int64_t p0 = (int64_t)blockIdx.z * chunk, p1 = min(n, p0 + chunk);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads: 4 outputs each
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  double sum = 0.0;
  for (int64_t p = p0; p < p1; p += CT) {
    for (int e = threadIdx.x; e < CT * CT; e += 256) {
      const int r = e / CT, c = e % CT;
      const int64_t pp = p + r;
      xa[r][c] = (pp < p1 && a0 + c < d) ? X[pp * ld + col + a0 + c] : 0.f;
      xb[r][c] = (pp < p1 && b0 + c < d) ? X[pp * ld + col + b0 + c] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < CT; ++r) {
      const double va = xa[r][tx];
#pragma unroll
      for (int m = 0; m < 4; ++m) acc[m] = fma(va, (double)xb[r][ty + 8 * m], acc[m]);
      if (ty == 0) sum += va;
    }
    __syncthreads();
  }
  if (a0 + tx < d) {
#pragma unroll
    for (int m = 0; m < 4; ++m)
      if (b0 + ty + 8 * m < d) atomicAdd(&S[(int64_t)(a0 + tx) * d + b0 + ty + 8 * m], acc[m]);
    if (ty == 0 && blockIdx.y == 0) atomicAdd(&s1[a0 + tx], sum);
  }
}

// Y[p][i] = sum_j R[i][j] X[p][j] within blocks of w = D / nblk dimensions (R given as
// nblk transposed blocks Rt[b][j][i]), accumulated in FP64; rounded half up when
// `round` (the integer grid of the training sets), else stored as FP32.
__global__ void rotate_kernel(const float* __restrict__ X, int64_t n, int D, const double* __restrict__ Rt, int nblk,
                              int round, float* __restrict__ Y) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * D) return;
  const int64_t p = e / D;
  const int i = (int)(e - p * D);
  const int w = D / nblk, b = i / w, ii = i - b * w;
  const double* rt = Rt + (int64_t)b * w * w;
  const float* x = X + p * D + b * w;
  double acc = 0.0;
  for (int j = 0; j < w; ++j) acc = fma(rt[(int64_t)j * w + ii], (double)x[j], acc);
  Y[e] = round ? (float)floor(acc + 0.5) : (float)acc;
}

// Cyclic Jacobi eigendecomposition of a symmetric d x d matrix A (row-major,
// overwritten): eigenvalues lam[i], eigenvectors as the columns of V.
void jacobi_eigen(std::vector<double>& A, int d, std::vector<double>& lam, std::vector<double>& V) {
  V.assign((size_t)d * d, 0.0);
  for (int i = 0; i < d; ++i) V[(size_t)i * d + i] = 1.0;
  double norm = 0.0;
  for (double v : A) norm += v * v;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < d; ++p)
      for (int q = p + 1; q < d; ++q) off += A[(size_t)p * d + q] * A[(size_t)p * d + q];
    if (off <= 1e-30 * norm || off == 0.0) break;
    for (int p = 0; p < d; ++p)
      for (int q = p + 1; q < d; ++q) {
        const double apq = A[(size_t)p * d + q];
        if (apq == 0.0) continue;
        const double app = A[(size_t)p * d + p], aqq = A[(size_t)q * d + q];
        // the rotation in the (p, q) plane that zeroes A[p][q]
        const double tau = (aqq - app) / (2.0 * apq);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < d; ++k) {  // A <- J^T A J (rows / columns p and q)
          const double akp = A[(size_t)k * d + p], akq = A[(size_t)k * d + q];
          A[(size_t)k * d + p] = c * akp - s * akq;
          A[(size_t)k * d + q] = s * akp + c * akq;
        }
        for (int k = 0; k < d; ++k) {
          const double apk = A[(size_t)p * d + k], aqk = A[(size_t)q * d + k];
          A[(size_t)p * d + k] = c * apk - s * aqk;
          A[(size_t)q * d + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < d; ++k) {
          const double vkp = V[(size_t)k * d + p], vkq = V[(size_t)k * d + q];
          V[(size_t)k * d + p] = c * vkp - s * vkq;
          V[(size_t)k * d + q] = s * vkp + c * vkq;
        }
      }
  }
  lam.resize(d);
  for (int i = 0; i < d; ++i) lam[i] = A[(size_t)i * d + i];
}

// Rotation (row-major d x d, FP64) of the covariance of the d columns at `col` of
// X (n x ld, device) for `groups` subspaces.
std::vector<double> learn_rotation(const float* X, int64_t n, int64_t ld, int col, int d, int groups,
                                   cudaStream_t st) {
  DevBuf S, s1;
  S.alloc((size_t)d * d * 8);
  s1.alloc((size_t)d * 8);
  BPQ_CUDA(cudaMemsetAsync(S.p, 0, S.bytes, st));
  BPQ_CUDA(cudaMemsetAsync(s1.p, 0, s1.bytes, st));
  const int tiles = (d + CT - 1) / CT;
  const int64_t chunk = 16384;
  dim3 grid(tiles, tiles, (unsigned)((n + chunk - 1) / chunk));
  cov_kernel<<<grid, 256, 0, st>>>(X, n, ld, col, d, chunk, S.as<double>(), s1.as<double>());
  check_launch("covariance kernel");
  std::vector<double> A((size_t)d * d), mu(d);
  BPQ_CUDA(cudaMemcpyAsync(A.data(), S.p, S.bytes, cudaMemcpyDeviceToHost, st));
  BPQ_CUDA(cudaMemcpyAsync(mu.data(), s1.p, s1.bytes, cudaMemcpyDeviceToHost, st));
  BPQ_CUDA(cudaStreamSynchronize(st));
  for (int a = 0; a < d; ++a) mu[a] /= (double)n;
  for (int a = 0; a < d; ++a)
    for (int b = 0; b < d; ++b) A[(size_t)a * d + b] = A[(size_t)a * d + b] / (double)n - mu[a] * mu[b];
  std::vector<double> lam, V;
  jacobi_eigen(A, d, lam, V);
  // eigenvalue allocation: descending order (ties by index), to the non-full
  // subspace with the smallest sum of logs (ties to the lower subspace)
  std::vector<int> order(d);
  for (int i = 0; i < d; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return lam[x] > lam[y]; });
  const int cap = d / groups;
  std::vector<std::vector<int>> buckets(groups);
  std::vector<double> logsum(groups, 0.0);
  for (int i : order) {
    int best = -1;
    for (int g = 0; g < groups; ++g)
      if ((int)buckets[g].size() < cap && (best < 0 || logsum[g] < logsum[best])) best = g;
    buckets[best].push_back(i);
    logsum[best] += std::log(std::max(lam[i], 1e-12));
  }
  std::vector<double> R((size_t)d * d);
  int row = 0;
  for (int g = 0; g < groups; ++g)
    for (int i : buckets[g]) {
      int am = 0;
      for (int k = 1; k < d; ++k)
        if (std::fabs(V[(size_t)k * d + i]) > std::fabs(V[(size_t)am * d + i])) am = k;
      const double sg = V[(size_t)am * d + i] < 0 ? -1.0 : 1.0;
      for (int k = 0; k < d; ++k) R[(size_t)row * d + k] = sg * V[(size_t)k * d + i];
      ++row;
    }
  return R;
}

// Uploads nblk transposed square blocks (block b = rows/cols b*w .. of a
// block-diagonal matrix given as its blocks, row-major) for rotate_kernel.
void upload_transposed(DevBuf& dst, const std::vector<const double*>& blocks, int w) {
  std::vector<double> t((size_t)blocks.size() * w * w);
  for (size_t b = 0; b < blocks.size(); ++b)
    for (int i = 0; i < w; ++i)
      for (int j = 0; j < w; ++j) t[b * w * w + (size_t)j * w + i] = blocks[b][(size_t)i * w + j];
  dst.alloc(t.size() * 8);
  BPQ_CUDA(cudaMemcpy(dst.p, t.data(), t.size() * 8, cudaMemcpyHostToDevice));
}

}  // namespace

void rotate_rows(const float* X, int64_t n, int D, const double* Rt, int nblk, bool round, float* Y, cudaStream_t st) {
  if (n <= 0) return;
  const int64_t total = n * D;
  rotate_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(X, n, D, Rt, nblk, round ? 1 : 0, Y);
  check_launch("rotation kernel");
}

void set_opq_rotations(bpq_index& ix, const double* R0, const double* R1, const double* R2, cudaStream_t st) {
  const int D = ix.p.D, h = ix.h, T = ix.p.T;
  ix.h_rot0.assign(R0, R0 + (size_t)D * D);
  ix.h_rot1.assign(R1, R1 + (size_t)h * h);
  ix.h_rot2.assign(R2, R2 + (size_t)h * h);
  // device: rot0 (one block), B (two blocks) and P = B rot0 (one block), transposed
  upload_transposed(ix.rot0t, {R0}, D);
  upload_transposed(ix.rotBt, {R1, R2}, h);
  std::vector<double> P((size_t)D * D, 0.0);
  for (int i = 0; i < D; ++i) {
    const int b = i / h, ii = i - b * h;
    const double* Rb = b ? R2 : R1;
    for (int j = 0; j < D; ++j) {
      double acc = 0.0;
      for (int t = 0; t < h; ++t) acc += Rb[(size_t)ii * h + t] * R0[(size_t)(b * h + t) * D + j];
      P[(size_t)i * D + j] = acc;
    }
  }
  upload_transposed(ix.rotPt, {P.data()}, D);
  {  // FP32 copies (transposed) of rot0 and P for the queries
    std::vector<float> a((size_t)D * D), b((size_t)D * D);
    for (int i = 0; i < D; ++i)
      for (int j = 0; j < D; ++j) {
        a[(size_t)j * D + i] = (float)R0[(size_t)i * D + j];
        b[(size_t)j * D + i] = (float)P[(size_t)i * D + j];
      }
    ix.rot0tf.alloc(a.size() * 4);
    ix.rotPtf.alloc(b.size() * 4);
    BPQ_CUDA(cudaMemcpy(ix.rot0tf.p, a.data(), a.size() * 4, cudaMemcpyHostToDevice));
    BPQ_CUDA(cudaMemcpy(ix.rotPtf.p, b.data(), b.size() * 4, cudaMemcpyHostToDevice));
  }
  // rotated coarse centroids B c (T x h per half) for the cross terms and the reconstruction scorer
  ix.C1r.alloc((size_t)T * h * 4);
  ix.C2r.alloc((size_t)T * h * 4);
  DevBuf t1, t2;
  upload_transposed(t1, {R1}, h);
  upload_transposed(t2, {R2}, h);
  rotate_rows(ix.C1.as<float>(), T, h, t1.as<double>(), 1, false, ix.C1r.as<float>(), st);
  rotate_rows(ix.C2.as<float>(), T, h, t2.as<double>(), 1, false, ix.C2r.as<float>(), st);
  BPQ_CUDA(cudaStreamSynchronize(st));
  ix.opq = true;
}

void rotate_for_index(const bpq_index& ix, const float* x, int64_t n, float* xc, float* xr, cudaStream_t st) {
  if (xc) rotate_rows(x, n, ix.p.D, ix.rot0t.as<double>(), 1, false, xc, st);
  if (xr) rotate_rows(x, n, ix.p.D, ix.rotPt.as<double>(), 1, false, xr, st);
}

namespace {
// Queries: both rotations at once in FP32 (a query's D floats staged in shared
// memory, one thread per output); rot0 and P = B rot0 as FP32 transposed copies.
__global__ void rotate_queries_kernel(const float* __restrict__ X, int64_t n, int D, const float* __restrict__ R0t,
                                      const float* __restrict__ Pt, float* __restrict__ yc, float* __restrict__ yr) {
  extern __shared__ float xs[];
  const int64_t p = blockIdx.x;
  if (p >= n) return;
  for (int j = threadIdx.x; j < D; j += blockDim.x) xs[j] = X[p * D + j];
  __syncthreads();
  for (int i = threadIdx.x; i < D; i += blockDim.x) {
    float a = 0.f, b = 0.f;
    for (int j = 0; j < D; ++j) {
      a = fmaf(R0t[(int64_t)j * D + i], xs[j], a);
      b = fmaf(Pt[(int64_t)j * D + i], xs[j], b);
    }
    yc[p * D + i] = a;
    yr[p * D + i] = b;
  }
}
}  // namespace

void rotate_queries(const bpq_index& ix, const float* q, int64_t n, float* qc, float* qr, cudaStream_t st) {
  if (n <= 0) return;
  BPQ_CHECK(n < (1LL << 31), BPQ_EINVAL, "too many queries for the rotation kernel");
  const int D = ix.p.D;
  rotate_queries_kernel<<<(unsigned)n, 128, (size_t)D * 4, st>>>(q, n, D, ix.rot0tf.as<float>(),
                                                                 ix.rotPtf.as<float>(), qc, qr);
  check_launch("query rotation kernel");
}

std::vector<double> opq_learn_rotation(const float* X, int64_t n, int64_t ld, int col, int d, int groups,
                                       cudaStream_t st) {
  return learn_rotation(X, n, ld, col, d, groups, st);
}

}  // namespace bpq
