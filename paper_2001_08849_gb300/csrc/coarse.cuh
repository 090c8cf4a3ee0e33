// Device view of the two-level preconditioner's coarse space (coarse.cu),
// shared with the CG kernels of solve.cu.
//
// Coarse space: one trilinear function per patch centre and displacement
// component on a d0 x d1 x d2 grid of centres over the mesh's bounding box.
// Each node lies in one interpolation cell (between 2 x 2 x 2 centres,
// clamped at the outermost centres) and carries its three fractional
// coordinates in that cell.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sfem {

constexpr int kChunkNodes = 2048;  // nodes per block of the restriction in the two-level iterations
constexpr int kSubNodes = 512;     // nodes per update item of the batched solver (batch.cu)

struct CoarseDev {
  int d[3];                // centres per axis
  int cd[3];               // interpolation cells per axis, max(d - 1, 1)
  int nc, npad, ncell;     // coarse DOFs (3 P), padded order of C, cells
  const int32_t *cell;     // n_nodes: interpolation cell of each node
  const int32_t *cinfo;    // n_nodes: centre of the cell's lower corner (bits 0-23) and
                           // whether the upper corner is a different centre on x, y, z
                           // (bits 24, 25, 26; not where the grid has one centre)
  const float *frac;       // n_nodes x 3: fractional position in the cell
  const int32_t *glist;    // nc x 8: cellsum entries summed into each coarse DOF (-1: none)
  const int32_t *cnodes;   // node ids grouped by cell (ascending within a cell)
  const int32_t *coff;     // ncell + 1
  const int4 *chunk;       // nchunk: (cell, first, end) ranges of cnodes, <= kChunkNodes nodes each
  int nchunk;
  const int4 *sub;         // nsub: the same ranges split to <= kSubNodes nodes
  int nsub;
  float *cellsum;          // ncell x 24 partial restrictions (8 corners x 3)
  float *rc, *yc;          // coarse residual and correction (npad)
  const float *C;          // A_c^-1 (symmetric, FP32): lower 64 x 64 blocks, block (a, b) at
                           // (a (a + 1) / 2 + b) * 4096, row-major
  const float *Ap;         // A_c itself in FP32, the same packed layout (the learned coarse
                           // correction's step length, cnet.cu)
};

// weight of corner k (bits: x = 4, y = 2, z = 1) at fractions f
__device__ __forceinline__ float cs_weight(const float f[3], int k) {
  return ((k & 4) ? f[0] : 1.f - f[0]) * ((k & 2) ? f[1] : 1.f - f[1]) * ((k & 1) ? f[2] : 1.f - f[2]);
}

// centre index of corner k of cell `cell`
__device__ __forceinline__ int cs_corner(const CoarseDev &cs, int cell, int k) {
  const int iz = cell % cs.cd[2], iy = (cell / cs.cd[2]) % cs.cd[1], ix = cell / (cs.cd[1] * cs.cd[2]);
  const int jx = min(ix + ((k >> 2) & 1), cs.d[0] - 1);
  const int jy = min(iy + ((k >> 1) & 1), cs.d[1] - 1);
  const int jz = min(iz + (k & 1), cs.d[2] - 1);
  return (jx * cs.d[1] + jy) * cs.d[2] + jz;
}

// reduce-scatter of 32 values over the warp by recursive halving (31
// shuffles instead of 5 per value): returns, in lane l, the warp total of
// value l (the restrictions' 24 corner sums)
__device__ __forceinline__ float warp_reduce_scatter32(float (&v)[32]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      const float send = upper ? v[i] : v[i + o];
      const float keep = upper ? v[i + o] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0];
}

// (Pi y)_i for DOF i = 3 node + c (not masked), y given by the caller
__device__ __forceinline__ float cs_prolong_y(const CoarseDev &cs, const float *yc, int64_t i) {
  const int64_t node = i / 3;
  const int c = (int)(i - 3 * node);
  const int ci = cs.cinfo[node];
  const int base = ci & 0xFFFFFF;
  const int ox = ((ci >> 24) & 1) ? 3 * cs.d[1] * cs.d[2] : 0;
  const int oy = ((ci >> 25) & 1) ? 3 * cs.d[2] : 0;
  const int oz = ((ci >> 26) & 1) ? 3 : 0;
  const float f[3] = {cs.frac[3 * node], cs.frac[3 * node + 1], cs.frac[3 * node + 2]};
  const float *y = yc + 3 * base + c;
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k)
    s = fmaf(cs_weight(f, k), y[((k & 4) ? ox : 0) + ((k & 2) ? oy : 0) + ((k & 1) ? oz : 0)], s);
  return s;
}

// (Pi yc)_i with the coarse space's own correction vector
__device__ __forceinline__ float cs_prolong(const CoarseDev &cs, int64_t i) { return cs_prolong_y(cs, cs.yc, i); }

}  // namespace sfem
