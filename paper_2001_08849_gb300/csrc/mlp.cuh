// Generic kernels of the small MLPs of the learned corrections (learned.cu:
// per-patch network; cnet.cu: coarse network): FP32 GEMM on the tensor
// cores (tc_gemm.cuh), bias + GELU,
// squared-error loss, GELU backward, column sums, Adam, BF16 rounding, the
// counter-based generator of the initial weights.  Internal linkage: each
// translation unit that includes this header has its own copy.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "reduce.cuh"
#include "sfem_internal.cuh"
#include "tc_gemm.cuh"

namespace sfem {

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

template <bool TA, bool TB>
static void launch_gemm_tc(dim3 grid, cudaStream_t st, int M, int N, int K, const float *A, int lda, const float *B,
                           int ldb, float *out, int ldo, int64_t stride, int k_split, int *err) {
  static bool attr[64] = {};  // the shared-memory attribute, set once per device
  int dev = 0;
  SFEM_CUDA(cudaGetDevice(&dev));
  if (dev >= 64 || !attr[dev]) {
    SFEM_CUDA(cudaFuncSetAttribute(k_gemm_tc<TA, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem));
    if (dev < 64) attr[dev] = true;
  }
  k_gemm_tc<TA, TB><<<grid, kTcThreads, kTcSmem, st>>>(M, N, K, A, lda, B, ldb, out, ldo, stride, k_split, err);
}

// C = op(A) op(B) (row-major, FP32) by k_gemm_tc, split over K when the
// output tiles alone would leave SMs idle (partial products in `split`,
// grown as needed, summed in a fixed order).  *err (device) is set when a
// CTA's wait for its MMAs ran out.
static void mlp_gemm(Allocator &mem, float *&split, size_t &split_floats, cudaStream_t st, int M, int N, int K,
                     const float *A, int lda, bool tA, const float *B, int ldb, bool tB, float *C, int ldc, int *err) {
  int dev = 0, sms = 0;
  SFEM_CUDA(cudaGetDevice(&dev));
  SFEM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int tiles = ((M + kTcBM - 1) / kTcBM) * ((N + kTcBN - 1) / kTcBN);
  int splits = 1;
  if (tiles < sms && K >= 4 * kTcBK) splits = std::min((sms + tiles - 1) / tiles, K / (2 * kTcBK));
  const int k_split = ((K + splits - 1) / splits + kTcBK - 1) / kTcBK * kTcBK;
  splits = k_split > 0 ? (K + k_split - 1) / k_split : 1;
  dim3 grid((N + kTcBN - 1) / kTcBN, (M + kTcBM - 1) / kTcBM, splits);
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
    launch_gemm_tc<true, true>(grid, st, M, N, K, A, lda, B, ldb, out, ldo, stride, k_split, err);
  else if (tA)
    launch_gemm_tc<true, false>(grid, st, M, N, K, A, lda, B, ldb, out, ldo, stride, k_split, err);
  else if (tB)
    launch_gemm_tc<false, true>(grid, st, M, N, K, A, lda, B, ldb, out, ldo, stride, k_split, err);
  else
    launch_gemm_tc<false, false>(grid, st, M, N, K, A, lda, B, ldb, out, ldo, stride, k_split, err);
  SFEM_CHECK_LAUNCH();
  if (splits > 1) {
    k_sum_splits<<<grid_for((int64_t)M * N, 256), 256, 0, st>>>(split, splits, M, N, C, ldc);
    SFEM_CHECK_LAUNCH();
  }
}

// throws SFEM_ETIMEOUT when a tensor-core GEMM since the last check reported
// a wait that ran out (the word is cleared)
static void check_gemm_err(int *err, cudaStream_t st) {
  int h = 0;
  SFEM_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  SFEM_CUDA(cudaStreamSynchronize(st));
  if (h) {
    SFEM_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    throw Error{SFEM_ETIMEOUT, "a tensor-core GEMM gave up waiting for its MMAs"};
  }
}

}  // namespace sfem
