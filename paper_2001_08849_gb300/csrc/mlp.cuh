// Generic kernels of the small MLPs of the learned corrections (learned.cu:
// per-patch network; cnet.cu: coarse network): FP32 GEMM, bias + GELU,
// squared-error loss, GELU backward, column sums, Adam, BF16 rounding, the
// counter-based generator of the initial weights.  Internal linkage: each
// translation unit that includes this header has its own copy.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "reduce.cuh"
#include "sfem_internal.cuh"

namespace sfem {

// out[z] = op(A)[M x K-range z] op(B); row-major; op(A) = A^T when TA (A is
// stored K x M), op(B) = B^T when TB (B stored N x K).  64x64 tiles, 4x4
// outputs per thread, K split over gridDim.z ranges of k_split.
template <bool TA, bool TB>
static __global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const float *__restrict__ A, int lda,
                                              const float *__restrict__ B, int ldb, float *__restrict__ out,
                                              int ldo, int64_t out_stride, int k_split) {
  __shared__ float As[16][68];
  __shared__ float Bs[16][68];
  const int tid = threadIdx.x;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int kb = blockIdx.z * k_split, ke = min(K, kb + k_split);
  const int tm = (tid >> 4) * 4, tn = (tid & 15) * 4;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = kb; k0 < ke; k0 += 16) {
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int e = tid + l * 256;
      const int mm = TA ? (e & 63) : (e >> 4), kk = TA ? (e >> 6) : (e & 15);
      const int gm = m0 + mm, gk = k0 + kk;
      float v = 0.f;
      if (gm < M && gk < ke) v = TA ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk];
      As[kk][mm] = v;
    }
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int e = tid + l * 256;
      const int nn = TB ? (e >> 4) : (e & 63), kk = TB ? (e & 15) : (e >> 6);
      const int gn = n0 + nn, gk = k0 + kk;
      float v = 0.f;
      if (gn < N && gk < ke) v = TB ? B[(int64_t)gn * ldb + gk] : B[(int64_t)gk * ldb + gn];
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = As[kk][tm + i];
        b[i] = Bs[kk][tn + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  float *o = out + (int64_t)blockIdx.z * out_stride;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gm = m0 + tm + i, gn = n0 + tn + j;
      if (gm < M && gn < N) o[(int64_t)gm * ldo + gn] = acc[i][j];
    }
}

// C[M x N] = sum over z of part[z] (fixed order)
static __global__ void k_sum_splits(const float *__restrict__ part, int splits, int M, int N, float *__restrict__ C, int ldc) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)M * N) return;
  float s = 0.f;
  for (int z = 0; z < splits; ++z) s += part[(int64_t)z * M * N + i];
  C[(i / N) * ldc + i % N] = s;
}

static __device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
static __device__ __forceinline__ float gelu_d(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// a += bias (per column); h = GELU(a) when h is not null
static __global__ void k_bias_gelu(float *a, float *h, const float *bias, int64_t rows, int cols) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows * cols) return;
  const float v = a[i] + bias[i % cols];
  a[i] = v;
  if (h) h[i] = gelu_f(v);
}

// dy = 2 (y - T) / rows; loss[0] = sum((y - T)^2) / rows; loss[1] += sum
static __global__ void __launch_bounds__(256) k_mse(const float *y, const float *T, int64_t n, int64_t rows, float *dy,
                                             double *partials, unsigned int *ticket, double *loss) {
  const float inv = 1.f / (float)rows;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
    const float d = y[i] - T[i];
    dy[i] = 2.f * d * inv;
    s += (double)d * d;
  }
  double vv[1] = {s};
  if (grid_sum<256, 1>(vv, partials, ticket, nullptr) && threadIdx.x == 0) {
    loss[0] = vv[0] / (double)rows;
    loss[1] += vv[0];
  }
}

static __global__ void k_gelu_back(float *d, const float *a, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] *= gelu_d(a[i]);
}

// out[c] = sum over rows of M[r, c] (FP64 accumulation, fixed order)
static __global__ void __launch_bounds__(256) k_colsum(const float *M, int64_t rows, int cols, float *out) {
  const int c = blockIdx.x;
  double s = 0.0;
  for (int64_t r = threadIdx.x; r < rows; r += 256) s += M[r * cols + c];
  s = block_sum<256>(s);
  if (threadIdx.x == 0) out[c] = (float)s;
}

static __global__ void k_adam(float *theta, const float *g, float *m, float *v, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2, __nv_bfloat16 *wbf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float th = theta[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  theta[i] = th;
  wbf[i] = __float2bfloat16_rn(th);
}

static __global__ void k_to_bf16(const float *theta, __nv_bfloat16 *wbf, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) wbf[i] = __float2bfloat16_rn(theta[i]);
}

// splitmix64 (Steele, Lea, Flood 2014)
static __host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

// C = op(A) op(B) (row-major, FP32) by k_gemm, split over K for small grids
// (partial products in `split`, grown as needed, summed in a fixed order)
static void mlp_gemm(Allocator &mem, float *&split, size_t &split_floats, cudaStream_t st, int M, int N, int K,
                     const float *A, int lda, bool tA, const float *B, int ldb, bool tB, float *C, int ldc) {
  const int tiles = ((M + 63) / 64) * ((N + 63) / 64);
  int splits = 1;
  if (tiles < 64 && K >= 512) splits = std::min(64, std::max(1, K / 256));
  const int k_split = ((K + splits - 1) / splits + 15) / 16 * 16;
  splits = (K + k_split - 1) / k_split;
  dim3 grid((N + 63) / 64, (M + 63) / 64, splits);
  float *out = C;
  int ldo = ldc;
  int64_t stride = 0;
  if (splits > 1) {
    const size_t need = (size_t)splits * M * N;
    if (need > split_floats) {
      if (split) mem.drop(split);
      split = mem.get<float>(need);
      split_floats = need;
    }
    out = split;
    ldo = N;
    stride = (int64_t)M * N;
  }
  if (tA && tB)
    k_gemm<true, true><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, out, ldo, stride, k_split);
  else if (tA)
    k_gemm<true, false><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, out, ldo, stride, k_split);
  else if (tB)
    k_gemm<false, true><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, out, ldo, stride, k_split);
  else
    k_gemm<false, false><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, out, ldo, stride, k_split);
  SFEM_CHECK_LAUNCH();
  if (splits > 1) {
    k_sum_splits<<<grid_for((int64_t)M * N, 256), 256, 0, st>>>(split, splits, M, N, C, ldc);
    SFEM_CHECK_LAUNCH();
  }
}

}  // namespace sfem
