// Deterministic FP64 block and grid reductions.
//
// Every block reduces its values with warp shuffles, writes one partial per
// quantity, and the last block to finish (ticket counter) sums the
// partials in block order.  For a fixed grid the result is bitwise
// reproducible.  Partials are read with ld.global.cg (L2) because they
// were written by other SMs.
#pragma once

#include <cuda_runtime.h>

namespace sfem {

template <int BS>
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[BS / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  v = (threadIdx.x < BS / 32) ? sh[threadIdx.x] : 0.0;
  if (wid == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;  // valid in thread 0
}

// FP32 variant of block_sum
template <int BS>
__device__ __forceinline__ float block_sum_f(float v) {
  __shared__ float shf[BS / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) shf[wid] = v;
  __syncthreads();
  v = (threadIdx.x < BS / 32) ? shf[threadIdx.x] : 0.f;
  if (wid == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;  // valid in thread 0
}

// Sum K quantities over the whole grid.  partials holds K * gridDim.x
// doubles, ticket is zero on entry and reset by the last block, which
// stores the K sums to out[0..K) (if out is not null), leaves them in v[]
// of all its threads and returns true there.
template <int BS, int K>
__device__ __forceinline__ bool grid_sum(double (&v)[K], double *partials, unsigned int *ticket, double *out) {
  __shared__ bool last;
  __shared__ double res[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = block_sum<BS>(v[k]);
    if (threadIdx.x == 0) partials[k * gridDim.x + blockIdx.x] = s;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = 0.0;
    for (unsigned int i = threadIdx.x; i < gridDim.x; i += BS) s += __ldcg(&partials[k * gridDim.x + i]);
    s = block_sum<BS>(s);
    if (threadIdx.x == 0) {
      res[k] = s;
      if (out) out[k] = s;
    }
  }
  if (threadIdx.x == 0) *ticket = 0u;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) v[k] = res[k];
  return true;
}

}  // namespace sfem
