// FP32 GEMM of the learned corrections' training on the fifth-generation
// tensor cores: tcgen05.mma of kind tf32 issued by one thread per CTA,
// operands in shared memory, the 128 x 128 FP32 accumulator tile in tensor
// memory (TMEM), read back by tcgen05.ld and stored through shared memory
// as coalesced rows.
//
// Accuracy: the 3xTF32 split of Ootomo and Yokota (2022, "Recovering single
// precision accuracy from Tensor Cores while surpassing the FP32 theoretical
// peak performance").  Each operand element x = hi + lo, hi = x with the 13
// low mantissa bits cleared (a TF32 value) and lo = x - hi (exact in FP32);
// A B is accumulated as lo_A hi_B + hi_A lo_B + hi_A hi_B, three MMAs per K
// step, which leaves an error near that of an FP32 GEMM (lo_A lo_B and the
// TF32 truncation of lo are below 2^-21 relative).
//
// Shared-memory operand layout (K-major, 128-byte swizzle): an operand tile
// of 128 rows x 32 K elements stores row r in the 128 bytes at r * 128, its
// 16-byte chunk c (elements 4c .. 4c + 3) at chunk position c ^ (r % 8);
// groups of 8 rows are 1024 bytes apart.  A warp stages one row per step
// when K is contiguous in global memory (a coalesced 128-byte load), else 8
// rows x 4 K values (four 32-byte loads); either way its 32 stores hit 32
// distinct banks.  One MMA
// consumes K = 8 (32 bytes of every row): its descriptor starts 32 bytes
// further per step, the hardware applying the same swizzle.
//
// Waits on the MMA-completion mbarriers are bounded (async.cuh); a CTA whose
// wait runs out writes no output, sets *err, waits (bounded) once more for
// its own MMAs and releases its TMEM.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "async.cuh"

namespace sfem {

constexpr int kTcBM = 128;                           // rows of A (and TMEM lanes) per CTA
constexpr int kTcBN = 128;                           // columns of B (TMEM columns) per CTA
constexpr int kTcBK = 32;                            // K elements per stage
constexpr int kTcThreads = 128;                      // four warps: one TMEM lane quarter each
constexpr int kTcOpBytes = kTcBM * kTcBK * 4;        // one operand tile, 16 KB
constexpr int kTcStageBytes = 4 * kTcOpBytes;        // A hi, A lo, B hi, B lo
constexpr int kTcSmem = 2 * kTcStageBytes + 64;      // two stages, two mbarriers, the TMEM address
static_assert(kTcBM == kTcBN, "the operand staging serves A and B tiles of one shape");
static_assert(kTcBM * (kTcBN + 1) * 4 <= 2 * kTcStageBytes, "the epilogue tile fits in the stage buffers");

// kind::tf32 instruction descriptor: FP32 accumulator (bits 4-5 = 1), A and B
// TF32 (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 in bits
// 17-22, M >> 4 in bits 24-28; dense, no negation, no saturation
constexpr uint32_t kTcIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcBN >> 3) << 17) |
                              ((uint32_t)(kTcBM >> 4) << 24);

// shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading
// byte offset (bits 16-29: unused by a swizzled K-major operand whose MMA K
// extent lies inside one 128-byte row; 1 by convention), stride byte offset
// >> 4 (bits 32-45: adjacent 8-row groups, 1024 B), descriptor version 1
// (bits 46-47), base offset 0 (tiles are 1024-byte aligned), 128-byte
// swizzle (bits 61-63 = 2)
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3fffu) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
         (2ull << 61);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// whole warp: allocates `cols` TMEM columns (a power of two, >= 32) and
// writes their address to *slot
__device__ __forceinline__ void tc_alloc(uint32_t *slot, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)), "r"(cols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// whole warp (the allocating one)
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}

// D (+)= A B^T for one K = 8 step; D is overwritten when accumulate == 0
__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(kTcIdesc), "r"(accumulate)
      : "memory");
}

// one arrival on `bar` once every MMA this thread issued so far has completed
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

// this thread's TMEM lane (row), 16 consecutive 32-bit columns from taddr
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// x = hi + lo, hi a TF32 value (low 13 mantissa bits cleared), lo exact
__device__ __forceinline__ void tf32_split(float x, float &hi, float &lo) {
  hi = __uint_as_float(__float_as_uint(x) & 0xffffe000u);
  lo = x - hi;
}

// byte offset of element (row r, K index k) of an operand tile
__device__ __forceinline__ int tc_off(int r, int k) { return r * 128 + ((((k >> 2) ^ r) & 7) << 4) + ((k & 3) << 2); }

// Element (row, k) of this thread's i-th slot (i = 0..31) of an operand
// tile.  KMajor (K contiguous in global memory, X[row * ld + k]): warp w
// takes rows 4i + w, lane = k: one load reads a 128-byte row and the 32
// stores hit 32 banks.  Otherwise (X[k * ld + row]): slot i of warp w is the
// group of 8 rows x 4 k with index P = 4i + w (rows 8 (P % 16) .., k
// 4 (P / 16) ..), lane l = row % 8 + 8 (k % 4): one load reads four 32-byte
// runs of rows, and the swizzle sends the 32 stores to 32 banks.
template <bool KMajor>
__device__ __forceinline__ void tc_slot(int i, int &row, int &k) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (KMajor) {
    row = 4 * i + warp;
    k = lane;
  } else {
    const int P = 4 * i + warp;
    row = 8 * (P & 15) + (lane & 7);
    k = 4 * (P >> 4) + (lane >> 3);
  }
}

// This thread's 32 elements of one operand tile for the K chunk at k0:
// element (r0 + row, k) of op(X) for A (rows = M) or of op(B)^T for B (rows
// = N), slots as tc_slot.
template <bool KMajor>
__device__ __forceinline__ void tc_fetch(const float *__restrict__ X, int ld, int r0, int rows, int k0, int kend,
                                         float (&v)[32]) {
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    int row, k;
    tc_slot<KMajor>(i, row, k);
    const int r = r0 + row, kk = k0 + k;
    v[i] = 0.f;
    if (r < rows && kk < kend) v[i] = KMajor ? __ldg(X + (int64_t)r * ld + kk) : __ldg(X + (int64_t)kk * ld + r);
  }
}

// writes the fetched elements, split into hi and lo, at their swizzled
// positions (the same element order as tc_fetch)
template <bool KMajor>
__device__ __forceinline__ void tc_stage(const float (&v)[32], uint8_t *hi, uint8_t *lo) {
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    int row, k;
    tc_slot<KMajor>(i, row, k);
    const int off = tc_off(row, k);
    float h, l;
    tf32_split(v[i], h, l);
    *reinterpret_cast<float *>(hi + off) = h;
    *reinterpret_cast<float *>(lo + off) = l;
  }
}

// out[z] = op(A)[M x K-range z] op(B); row-major; op(A) = A^T when TA (A is
// stored K x M), op(B) = B^T when TB (B stored N x K).  CTA (x, y, z): the
// 128 x 128 output tile (y, x) over K range z of k_split elements.
template <bool TA, bool TB>
static __global__ void __launch_bounds__(kTcThreads, 1)
    k_gemm_tc(int M, int N, int K, const float *__restrict__ A, int lda, const float *__restrict__ B, int ldb,
              float *__restrict__ out, int ldo, int64_t out_stride, int k_split, int *err) {
  extern __shared__ __align__(1024) uint8_t tc_smem[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(tc_smem + 2 * kTcStageBytes);
  uint32_t *slot = reinterpret_cast<uint32_t *>(bar + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * kTcBM, n0 = blockIdx.x * kTcBN;
  const int kb = blockIdx.z * k_split, ke = min(K, kb + k_split);
  const int nchunks = ke > kb ? (ke - kb + kTcBK - 1) / kTcBK : 0;

  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
  }
  if (warp == 0) tc_alloc(slot, kTcBN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;

  float va[32], vb[32];
  if (nchunks > 0) {
    tc_fetch<!TA>(A, lda, m0, M, kb, ke, va);
    tc_fetch<TB>(B, ldb, n0, N, kb, ke, vb);
  }
  int issued = 0;  // chunks whose MMAs were issued and committed
  bool ok = true;
  for (int c = 0; c < nchunks; ++c) {
    const int buf = c & 1;
    // the MMAs of chunk c - 2 read this buffer: wait for their commit
    const bool free_ok = c < 2 || mbar_wait(&bar[buf], ((c - 2) >> 1) & 1);
    if (!__syncthreads_and(free_ok)) {
      ok = false;
      break;
    }
    uint8_t *st = tc_smem + buf * kTcStageBytes;
    tc_stage<!TA>(va, st, st + kTcOpBytes);
    tc_stage<TB>(vb, st + 2 * kTcOpBytes, st + 3 * kTcOpBytes);
    if (c + 1 < nchunks) {
      const int k0 = kb + (c + 1) * kTcBK;
      tc_fetch<!TA>(A, lda, m0, M, k0, ke, va);
      tc_fetch<TB>(B, ldb, n0, N, k0, ke, vb);
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a_hi = smem_addr(st), a_lo = a_hi + kTcOpBytes;
      const uint32_t b_hi = a_hi + 2 * kTcOpBytes, b_lo = a_hi + 3 * kTcOpBytes;
#pragma unroll
      for (int s = 0; s < kTcBK / 8; ++s) {
        const uint32_t o = s * 32;  // K = 8 FP32 elements per MMA
        tc_mma(tmem, tc_desc(a_lo + o), tc_desc(b_hi + o), (c | s) != 0);
        tc_mma(tmem, tc_desc(a_hi + o), tc_desc(b_lo + o), 1u);
        tc_mma(tmem, tc_desc(a_hi + o), tc_desc(b_hi + o), 1u);
      }
      tc_commit(&bar[buf]);
    }
    issued = c + 1;
  }
  // the last commit covers every MMA issued before it
  bool done = true;
  if (issued > 0) done = mbar_wait(&bar[(issued - 1) & 1], ((issued - 1) >> 1) & 1);
  done = __syncthreads_and(done);
  tc_fence_after();
  if (ok && done) {
    // accumulator rows -> shared memory (the stage buffers are idle now;
    // rows padded to kTcBN + 1 floats: conflict-free), then each warp
    // stores its own 32 rows with coalesced row writes
    float *o = out + (int64_t)blockIdx.z * out_stride;
    float *tile = reinterpret_cast<float *>(tc_smem);
    constexpr int kLd = kTcBN + 1;
    const int row = warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < kTcBN; c0 += 16) {
      float v[16];
      if (issued > 0)
        tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      else
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = 0.f;
#pragma unroll
      for (int i = 0; i < 16; ++i) tile[row * kLd + c0 + i] = v[i];
    }
    __syncwarp();
#pragma unroll 1
    for (int rr = 0; rr < 32; ++rr) {
      const int r = warp * 32 + rr;
      if (m0 + r >= M) break;
#pragma unroll
      for (int cc = lane; cc < kTcBN; cc += 32)
        if (n0 + cc < N) o[(int64_t)(m0 + r) * ldo + n0 + cc] = tile[r * kLd + cc];
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, kTcBN);
}

}  // namespace sfem
