// Two-level preconditioner for the PCG solves: Jacobi plus a Galerkin coarse
// correction (the paper has no counterpart: it calls a direct solver).
//
//   M^-1 = D^-1 + Pi A_c^-1 Pi^T,   A_c = Pi^T A Pi,
//
// Pi: one trilinear function per patch centre and component on a regular
// grid of centres over the bounding box, masked by P (see coarse.cuh).
//
// Setup (sfem_coarse_setup):
//   * nodes grouped by interpolation cell with their fractions (host, once);
//   * A_c tile by tile (k_cs_galerkin, below), or by probing (the fallback
//     and an option): the centres are split into colour classes with stride
//     s_a = min(5, d_a) per axis.  For every class and component the FP32
//     tiled operator is applied to the sum of the class's functions, and the
//     restricted response at centre i is attributed to the unique class
//     member j with |i_a - j_a| <= 2 on every axis.  The operator couples
//     nodes two element layers apart, so centres farther apart than two
//     cells are not coupled when patches span at least three elements, and
//     within a stride-5 class the members are 5 apart;
//   * A_c is symmetrised and factored by a blocked Cholesky (L) that skips
//     the zero blocks outside its band, in FP32 by default (FP64 on a
//     non-positive pivot or on request, sfem_coarse_opts.factor), inverted
//     to W = L^-1 and C = W^T W = A_c^-1 in FP32 (blocked, 64 x 64 tiles;
//     only the lower blocks of the symmetric C are stored).
// Per PCG iteration (coarse_correction): rc = Pi^T r (FP32 atomics per run
// of nodes of one interpolation cell in the solve's fused kernels;
// fixed-order sums and a fixed-order gather per centre at initialisation,
// reliable updates and sfem_coarse_apply), yc = C rc (FP32 product with
// the L2-resident packed C), and the CG kernels add P Pi yc to D^-1 r.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "reduce.cuh"
#include "sfem_internal.cuh"
#include "tile_apply.cuh"

namespace sfem {

constexpr int kCB = 64;           // dense block order
static_assert(kCB == 64, "k_cs_symv maps 128 threads to 64 x 64 blocks");
constexpr int64_t kMaxCoarse = 8192;  // coarse DOFs (3 per centre)
constexpr int kRestrictThreads = 256;

// ---- restriction -----------------------------------------------------------

// cellsum[cell][3k + c] = sum over the cell's nodes of w_k(x) v_c(x)
// (v masked by dmask when dmask is given)
template <class TV>
__global__ void __launch_bounds__(kRestrictThreads) k_cs_restrict(const TV *__restrict__ v,
                                                                 const uint8_t *__restrict__ dmask, CoarseDev cs,
                                                                 const int *done) {
  if (done && *done) return;
  const int cell = blockIdx.x;
  const int b = cs.coff[cell], e = cs.coff[cell + 1];
  float acc[24];
#pragma unroll
  for (int j = 0; j < 24; ++j) acc[j] = 0.f;
  for (int i = b + threadIdx.x; i < e; i += kRestrictThreads) {
    const int64_t n = cs.cnodes[i];
    const float f[3] = {cs.frac[3 * n], cs.frac[3 * n + 1], cs.frac[3 * n + 2]};
    float x[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) x[c] = (dmask && !dmask[3 * n + c]) ? 0.f : (float)v[3 * n + c];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float w = cs_weight(f, k);
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[3 * k + c] = fmaf(w, x[c], acc[3 * k + c]);
    }
  }
  __shared__ float sm[kRestrictThreads / 32][24];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < 24; ++j) {
    float s = acc[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) sm[wid][j] = s;
  }
  __syncthreads();
  if (threadIdx.x < 24) {
    float s = 0.f;
#pragma unroll
    for (int w = 0; w < kRestrictThreads / 32; ++w) s += sm[w][threadIdx.x];
    cs.cellsum[24 * (int64_t)cell + threadIdx.x] = s;
  }
}

// rc[3j + c] = sum over the cells having centre j as a corner (fixed order)
__global__ void k_cs_gather(CoarseDev cs, const int *done) {
  if (done && *done) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cs.npad) return;
  cs.yc[t] = 0.f;  // k_cs_symv accumulates into yc
  if (t >= cs.nc) {
    cs.rc[t] = 0.f;
    return;
  }
  // the (cell, corner) entries of this centre, listed at setup in a fixed order
  const int *g = cs.glist + 8 * (int64_t)t;
  double s = 0.0;
#pragma unroll
  for (int e = 0; e < 8; ++e)
    if (g[e] >= 0) s += (double)cs.cellsum[g[e]];
  cs.rc[t] = (float)s;
}

// yc += C rc with C = A_c^-1 symmetric, stored as its lower 64 x 64 blocks
// (block (a, b), a >= b, at (a (a + 1) / 2 + b) * 4096, row-major): half the
// bytes of the full matrix, which streams from DRAM every iteration (the
// operator's records evict it from L2; keeping it there with an evict-last
// policy, or marking the records evict-first, measured no faster).  One CTA
// per block: the block is read once with evict-first loads and applied
// twice, C_ab rc_b to yc_a (row sums from registers) and C_ab^T rc_a to yc_b
// (a > b; column sums from a shared-memory copy of the block), by FP32
// atomics; yc must be zero before.
// With rzc, rc.C rc is added to *rzc as well (rc_a.C_ab rc_b, twice for
// a > b; one FP64 atomic per block).
constexpr int kSymvThreads = 128;  // two rows per thread; 9 CTAs per SM: the 1275 blocks of 3150 DOFs in one wave

__global__ void __launch_bounds__(kSymvThreads, 9) k_cs_symv(CoarseDev cs, const int *done, double *rzc) {
  if (done && *done) return;
  const int t = blockIdx.x;
  int a = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((a + 1) * (a + 2) / 2 <= t) ++a;
  while (a * (a + 1) / 2 > t) --a;
  const int b = t - a * (a + 1) / 2;
  __shared__ float ra[kCB], rb[kCB];
  if (threadIdx.x < kCB) {
    ra[threadIdx.x] = cs.rc[a * kCB + threadIdx.x];
    rb[threadIdx.x] = cs.rc[b * kCB + threadIdx.x];
  }
  // thread: rows i and i + 32 (i = tid / 4), columns 16 q .. 16 q + 15 (q = tid % 4);
  // off-diagonal blocks are also copied to shared memory (rows padded to 65
  // floats) for the transposed product
  __shared__ float bs[kCB][kCB + 1];
  __shared__ float part[2][kCB];
  const int i = threadIdx.x >> 2, q = threadIdx.x & 3;
  const float4 *blk = reinterpret_cast<const float4 *>(cs.C + (int64_t)t * kCB * kCB) + i * (kCB / 4) + q * 4;
  float4 v[2][4];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int u = 0; u < 4; ++u) v[h][u] = __ldcs(blk + h * 32 * (kCB / 4) + u);
  if (a != b)
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        float *dst = &bs[i + 32 * h][16 * q + 4 * u];
        dst[0] = v[h][u].x;
        dst[1] = v[h][u].y;
        dst[2] = v[h][u].z;
        dst[3] = v[h][u].w;
      }
  __syncthreads();
  const float *rbq = rb + 16 * q;
  float s[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    float x = 0.f;
#pragma unroll
    for (int u = 0; u < 4; ++u)
      x = fmaf(v[h][u].x, rbq[4 * u],
               fmaf(v[h][u].y, rbq[4 * u + 1], fmaf(v[h][u].z, rbq[4 * u + 2], fmaf(v[h][u].w, rbq[4 * u + 3], x))));
    x += __shfl_xor_sync(0xffffffffu, x, 1);
    x += __shfl_xor_sync(0xffffffffu, x, 2);
    s[h] = x;
    if (q == 0) atomicAdd(&cs.yc[a * kCB + i + 32 * h], x);
  }
  if (rzc) {  // whole block (rzc is uniform)
    float e = q == 0 ? (ra[i] * s[0] + ra[i + 32] * s[1]) * (a == b ? 1.f : 2.f) : 0.f;
    e = block_sum_f<kSymvThreads>(e);
    if (threadIdx.x == 0) atomicAdd(rzc, (double)e);
  }
  if (a == b) return;  // a whole block: uniform
  // C_ab^T ra: thread (column j = tid % 64, rows 32 p .. 32 p + 31 with
  // p = tid / 64) sums C_ab[i][j] ra[i]; then the two halves are added
  const int j = threadIdx.x & (kCB - 1), p = threadIdx.x / kCB;
  float x = 0.f;
#pragma unroll
  for (int r = 0; r < 32; ++r) x = fmaf(bs[32 * p + r][j], ra[32 * p + r], x);
  part[p][j] = x;
  __syncthreads();
  if (threadIdx.x < kCB) atomicAdd(&cs.yc[b * kCB + threadIdx.x], part[0][threadIdx.x] + part[1][threadIdx.x]);
}

// ---- probing -----------------------------------------------------------------

// v = P Pi (sum of the class's functions in component comp), FP32
__global__ void k_cs_probe(CoarseDev cs, int64_t n_nodes, const uint8_t *__restrict__ dmask, int comp, int3 res,
                           int3 str, float *__restrict__ v) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= n_nodes) return;
  const int cell = cs.cell[n];
  const float f[3] = {cs.frac[3 * n], cs.frac[3 * n + 1], cs.frac[3 * n + 2]};
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int j = cs_corner(cs, cell, k);
    const int jz = j % cs.d[2], jy = (j / cs.d[2]) % cs.d[1], jx = j / (cs.d[1] * cs.d[2]);
    if (jx % str.x == res.x && jy % str.y == res.y && jz % str.z == res.z) s += cs_weight(f, k);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) v[3 * n + c] = (c == comp && dmask[3 * n + c]) ? s : 0.f;
}

// Ac[(3i + c'), (3j + comp)] = rc[3i + c'] for the class member j near i
__global__ void k_cs_attrib(CoarseDev cs, int comp, int3 res, int3 str, double *__restrict__ Ac) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cs.nc) return;
  const int i = t / 3;
  const int iz = i % cs.d[2], iy = (i / cs.d[2]) % cs.d[1], ix = i / (cs.d[1] * cs.d[2]);
  const int ia[3] = {ix, iy, iz}, ra[3] = {res.x, res.y, res.z}, sa[3] = {str.x, str.y, str.z};
  int ja[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (sa[a] < 5) {
      ja[a] = ra[a];  // stride = d: the class has one member on this axis
    } else {
      // the member of residue class ra (mod 5) within distance 2 of ia
      int off = ((ra[a] - ia[a]) % 5 + 5) % 5;  // 0 .. 4
      if (off > 2) off -= 5;                    // -2 .. 2
      ja[a] = ia[a] + off;
      if (ja[a] < 0 || ja[a] >= cs.d[a]) return;
    }
  }
  const int j = (ja[0] * cs.d[1] + ja[1]) * cs.d[2] + ja[2];
  Ac[(int64_t)t * cs.npad + 3 * j + comp] = (double)cs.rc[t];
}

// ---- Galerkin coarse matrix, tile by tile ------------------------------------

constexpr int kGalMaxCells = 64;    // interpolation cells a tile may touch (4 per axis)
constexpr int kGalMaxCentres = 125; // centres of those cells (5 per axis)

// Every tile applies its part of the FP32 operator (own tets, halo strains)
// to each coarse function P Pi_J whose centre is a corner of a cell touched
// by the tile's nodes, and restricts the tile's masked nodal forces against
// the same centres; the contributions of all tiles add up to
// A_c = Pi^T P K P Pi (FP64 atomics into the dense A_c).
//
// The three components of one centre share a pass where every tile node has
// all or none of its DOFs free (the clamped beam: every tile): the field
// u = w_J e_c has displacement gradient e_c (x) grad w_J, so one pass forms
// V grad w_J per tet (own and halo), its face average over the smoothing
// domains, and from it the smoothed strain of each component (e_c (x) g in
// Voigt form); only stress, nodal forces and restriction run per component.
// Tiles with partly prescribed nodes apply the operator per (centre,
// component).
//
// Restriction: the tile's nodes are grouped by interpolation cell (stable
// order); one warp per cell sums w_k(x) f(x) over its nodes for the cell's
// 8 corners and 3 components, and each local centre sums the (cell,
// corner) entries that map to it in a fixed order.
// Dynamic shared memory: the tile layout (stage_off float4 units), then per
// tile node a float4 stage (local cell: index in bits 0-7, coordinates in
// bits 8-13; free-DOF mask in bits 28-30; the three fractions), a float4 of
// masked nodal forces and a uint16 order.  Sets *overflow for a tile that touches more than 4 cells on an
// axis.
constexpr int kGalWarps = kTileThreads / 32;

// 1D hat weight of local centre coordinate jc for a node in local cell
// coordinate lc at fraction f (upper corner clamped to the last centre)
__device__ __forceinline__ float gal_w1(int jc, int lc, int c0, int d, float f) {
  const int lo = c0 + lc, hi = min(lo + 1, d - 1), j = c0 + jc;
  return (j == lo ? 1.f - f : 0.f) + (j == hi ? f : 0.f);
}

__global__ void __launch_bounds__(kTileThreads, 3) k_cs_galerkin(TileArgs A, CoarseDev cs,
                                                              const uint8_t *__restrict__ dmask, float lam,
                                                              float mu, int stage_off, double *__restrict__ Ac,
                                                              int *overflow, int *maxdist) {
  extern __shared__ float4 smem_t[];
  __shared__ int bb[6], coff[kGalMaxCells + 1], mixed, tile_md;
  __shared__ float cellacc[kGalMaxCells][24];
  __shared__ short gat[kGalMaxCentres][8];
  const int tile = blockIdx.x;
  TileRegs R;
  tile_load(A, tile, R);
  const TileView T = tile_view(A, tile, smem_t);
  float4 *stage = smem_t + stage_off;
  float4 *nf = stage + T.L;  // masked nodal forces (the tile's force slots overlay su)
  uint16_t *order = reinterpret_cast<uint16_t *>(nf + T.L);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < 3) {
    bb[threadIdx.x] = 1 << 30;
    bb[3 + threadIdx.x] = -1;
  }
  if (threadIdx.x == 0) {
    mixed = 0;
    tile_md = 0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < T.L; i += kTileThreads) {
    const int64_t node = A.tile_nodes[T.n0 + i];
    const int cell = cs.cell[node];
    const int m = (dmask[3 * node] ? 1 : 0) | (dmask[3 * node + 1] ? 2 : 0) | (dmask[3 * node + 2] ? 4 : 0);
    stage[i] = make_float4(__int_as_float(cell | (m << 28)), cs.frac[3 * node], cs.frac[3 * node + 1],
                           cs.frac[3 * node + 2]);
    T.snode[i] = A.node_inc[T.n0 + i];
    if (m != 0 && m != 7) mixed = 1;
    const int iz = cell % cs.cd[2], iy = (cell / cs.cd[2]) % cs.cd[1], ix = cell / (cs.cd[1] * cs.cd[2]);
    atomicMin(&bb[0], ix);
    atomicMin(&bb[1], iy);
    atomicMin(&bb[2], iz);
    atomicMax(&bb[3], ix);
    atomicMax(&bb[4], iy);
    atomicMax(&bb[5], iz);
  }
  __syncthreads();
  const int c0[3] = {bb[0], bb[1], bb[2]};
  const int ncl[3] = {bb[3] - bb[0] + 1, bb[4] - bb[1] + 1, bb[5] - bb[2] + 1};
  if (ncl[0] > 4 || ncl[1] > 4 || ncl[2] > 4) {
    if (threadIdx.x == 0) atomicExch(overflow, 1);
    return;
  }
  const int nlc = ncl[0] * ncl[1] * ncl[2];
  // local centres: corners of the local cells, clamped to the grid
  int nj[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) nj[a] = min(c0[a] + ncl[a], cs.d[a] - 1) - c0[a] + 1;
  const int nloc = nj[0] * nj[1] * nj[2];
  // local cell of every node (index, coordinates), mask kept
  for (int i = threadIdx.x; i < T.L; i += kTileThreads) {
    const int cm = __float_as_int(stage[i].x);
    const int cell = cm & 0x0FFFFFFF;
    const int iz = cell % cs.cd[2], iy = (cell / cs.cd[2]) % cs.cd[1], ix = cell / (cs.cd[1] * cs.cd[2]);
    const int lx = ix - c0[0], ly = iy - c0[1], lz = iz - c0[2];
    const int lc = (lx * ncl[1] + ly) * ncl[2] + lz;
    stage[i].x = __int_as_float(lc | (lx << 8) | (ly << 10) | (lz << 12) | (cm & 0x70000000));
  }
  // per local centre the (cell, corner) pairs that restrict onto it, in a
  // fixed order
  for (int il = threadIdx.x; il < nloc; il += kTileThreads) {
    const int jx = il / (nj[1] * nj[2]), jy = (il / nj[2]) % nj[1], jz = il % nj[2];
    int n = 0;
    for (int lc = 0; lc < nlc; ++lc) {
      const int lx = lc / (ncl[1] * ncl[2]), ly = (lc / ncl[2]) % ncl[1], lz = lc % ncl[2];
      for (int k = 0; k < 8; ++k) {
        const int gx = min(c0[0] + lx + ((k >> 2) & 1), cs.d[0] - 1) - c0[0];
        const int gy = min(c0[1] + ly + ((k >> 1) & 1), cs.d[1] - 1) - c0[1];
        const int gz = min(c0[2] + lz + (k & 1), cs.d[2] - 1) - c0[2];
        if (gx == jx && gy == jy && gz == jz && n < 8) gat[il][n++] = (short)((lc << 3) | k);
      }
    }
    for (; n < 8; ++n) gat[il][n] = -1;
  }
  __syncthreads();
  // stable grouping of the tile's nodes by local cell: rank = earlier nodes
  // of the same cell
  if (threadIdx.x <= nlc) coff[threadIdx.x] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < T.L; i += kTileThreads) atomicAdd(&coff[(__float_as_int(stage[i].x) & 0xFF) + 1], 1);
  __syncthreads();
  if (threadIdx.x == 0)
    for (int q = 0; q < nlc; ++q) coff[q + 1] += coff[q];
  __syncthreads();
  for (int i = threadIdx.x; i < T.L; i += kTileThreads) {
    const int lc = __float_as_int(stage[i].x) & 0xFF;
    int rank = 0;
    for (int t = 0; t < i; ++t) rank += ((__float_as_int(stage[t].x) & 0xFF) == lc);
    order[coff[lc] + rank] = (uint16_t)i;
  }
  __syncthreads();

  // restriction of the masked nodal forces in nf against the local centres,
  // added to column `col` of A_c (all threads; ends with a barrier)
  auto restrict_add = [&](int col) {
    // (lower and upper x corners in two sweeps: 12 accumulators per lane)
    for (int t = warp; t < 2 * nlc; t += kGalWarps) {
      const int lc = t >> 1, k0 = 4 * (t & 1);
      float a[12];
#pragma unroll
      for (int q = 0; q < 12; ++q) a[q] = 0.f;
      for (int e = coff[lc] + lane; e < coff[lc + 1]; e += 32) {
        const int i = order[e];
        const float4 st = stage[i];
        const float f[3] = {st.y, st.z, st.w};
        const float4 fi = nf[i];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float w = cs_weight(f, k0 + k);
          a[3 * k] = fmaf(w, fi.x, a[3 * k]);
          a[3 * k + 1] = fmaf(w, fi.y, a[3 * k + 1]);
          a[3 * k + 2] = fmaf(w, fi.z, a[3 * k + 2]);
        }
      }
#pragma unroll
      for (int q = 0; q < 12; ++q) {
        float v = a[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) cellacc[lc][3 * k0 + q] = v;
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 3 * nloc; t += kTileThreads) {
      const int il = t / 3, cc = t - 3 * il;
      float v = 0.f;
#pragma unroll
      for (int n = 0; n < 8; ++n) {
        const int g = gat[il][n];
        if (g >= 0) v += cellacc[g >> 3][3 * (g & 7) + cc];
      }
      if (v != 0.f) {
        const int ix = c0[0] + il / (nj[1] * nj[2]), iy = c0[1] + (il / nj[2]) % nj[1], iz = c0[2] + il % nj[2];
        const int I = (ix * cs.d[1] + iy) * cs.d[2] + iz;
        atomicAdd(&Ac[(int64_t)(3 * I + cc) * cs.npad + col], (double)v);
        atomicMax(&tile_md, abs(3 * I + cc - col));
      }
    }
    __syncthreads();
  };
  // masked nodal forces of the tile into nf (all threads; ends with a barrier)
  auto node_forces = [&]() {
    for (int i = threadIdx.x; i < T.L; i += kTileThreads) {
      float fx, fy, fz;
      tile_node_force(T, i, fx, fy, fz);
      const int m = __float_as_int(stage[i].x) >> 28;
      nf[i] = make_float4((m & 1) ? fx : 0.f, (m & 2) ? fy : 0.f, (m & 4) ? fz : 0.f, 0.f);
    }
    __syncthreads();
  };
  // value of the local centre's hat function at node i
  auto hat = [&](int i, int jx, int jy, int jz) {
    const float4 st = stage[i];
    const int cm = __float_as_int(st.x);
    return gal_w1(jx, (cm >> 8) & 3, c0[0], cs.d[0], st.y) * gal_w1(jy, (cm >> 10) & 3, c0[1], cs.d[1], st.z) *
           gal_w1(jz, (cm >> 12) & 3, c0[2], cs.d[2], st.w);
  };

  for (int jl = 0; jl < nloc; ++jl) {
    const int jx = jl / (nj[1] * nj[2]), jy = (jl / nj[2]) % nj[1], jz = jl % nj[2];
    const int J = ((c0[0] + jx) * cs.d[1] + c0[1] + jy) * cs.d[2] + c0[2] + jz;
    if (!mixed) {
      // scalar field w_J on the free nodes
      for (int i = threadIdx.x; i < T.L; i += kTileThreads) {
        const float v = (__float_as_int(stage[i].x) >> 28) ? hat(i, jx, jy, jz) : 0.f;
        T.su[i] = make_float4(v, 0.f, 0.f, 0.f);
      }
      __syncthreads();
      // (V grad w, V) of own and halo tets
#pragma unroll
      for (int r = 0; r < kTilePer; ++r) {
        const int j = threadIdx.x + r * kTileThreads;
        if (j < T.n_own) {
          TetGeo G;
          uint2 lc;
          rec_unpack(R.rr[r], G, lc);
          const int l[4] = {(int)(lc.x & 0xFFFF), (int)(lc.x >> 16), (int)(lc.y & 0xFFFF), (int)(lc.y >> 16)};
          float g[3] = {0.f, 0.f, 0.f};
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const float w = T.su[l[a]].x;
#pragma unroll
            for (int q = 0; q < 3; ++q) g[q] = fmaf(w, G.g[a][q], g[q]);
          }
          T.swa[j] = make_float4(g[0], g[1], g[2], G.V);
        }
      }
      for (int h = threadIdx.x; h < T.H; h += kTileThreads) {
        TetGeo G;
        uint2 lc;
        load_rec(A.rec, A.rs, A.halo_tet[T.h0 + h], G, lc, nullptr);
        lc = A.halo_lconn[T.h0 + h];
        const int l[4] = {(int)(lc.x & 0xFFFF), (int)(lc.x >> 16), (int)(lc.y & 0xFFFF), (int)(lc.y >> 16)};
        float g[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const float w = T.su[l[a]].x;
#pragma unroll
          for (int q = 0; q < 3; ++q) g[q] = fmaf(w, G.g[a][q], g[q]);
        }
        T.swa[T.n_own + h] = make_float4(g[0], g[1], g[2], G.V);
      }
      __syncthreads();
      // face-averaged V grad w of the own tets (kept in registers)
      float Sg[kTilePer][3];
#pragma unroll
      for (int r = 0; r < kTilePer; ++r) {
        Sg[r][0] = Sg[r][1] = Sg[r][2] = 0.f;
        const int j = threadIdx.x + r * kTileThreads;
        if (j >= T.n_own) continue;
        const uint2 nb2 = make_uint2(__float_as_uint(R.rr[r][3].x), __float_as_uint(R.rr[r][3].y));
        const int nb[4] = {(int)(nb2.x & 0xFFFF), (int)(nb2.x >> 16), (int)(nb2.y & 0xFFFF), (int)(nb2.y >> 16)};
        const float4 we = T.swa[j];
        float ks = 0.f;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          if (nb[a] != kNoNbr) {
            const float4 wn = T.swa[nb[a]];
            const float k = __fdividef(0.25f, we.w + wn.w);
            ks += k;
            Sg[r][0] = fmaf(k, wn.x, Sg[r][0]);
            Sg[r][1] = fmaf(k, wn.y, Sg[r][1]);
            Sg[r][2] = fmaf(k, wn.z, Sg[r][2]);
          } else {
            ks += __fdividef(0.25f, we.w);
          }
        }
        Sg[r][0] = fmaf(ks, we.x, Sg[r][0]);
        Sg[r][1] = fmaf(ks, we.y, Sg[r][1]);
        Sg[r][2] = fmaf(ks, we.z, Sg[r][2]);
      }
      for (int comp = 0; comp < 3; ++comp) {
        // smoothed strain of w_J e_comp (Voigt xx yy zz yz zx xy), stress,
        // nodal force slots
#pragma unroll
        for (int r = 0; r < kTilePer; ++r) {
          const int j = threadIdx.x + r * kTileThreads;
          if (j >= T.n_own) continue;
          TetGeo G;
          uint2 lc;
          rec_unpack(R.rr[r], G, lc);
          const float g0 = Sg[r][0], g1 = Sg[r][1], g2 = Sg[r][2];
          const float S[6] = {comp == 0 ? g0 : 0.f, comp == 1 ? g1 : 0.f, comp == 2 ? g2 : 0.f,
                              comp == 1 ? g2 : (comp == 2 ? g1 : 0.f), comp == 0 ? g2 : (comp == 2 ? g0 : 0.f),
                              comp == 0 ? g1 : (comp == 1 ? g0 : 0.f)};
          const float tr = S[0] + S[1] + S[2];
          const float st[6] = {lam * tr + 2.f * mu * S[0], lam * tr + 2.f * mu * S[1], lam * tr + 2.f * mu * S[2],
                               mu * S[3], mu * S[4], mu * S[5]};
#pragma unroll
          for (int a = 0; a < 4; ++a) store_slot_force(T, R.rr[r][3], a, G.g[a], st);
        }
        __syncthreads();
        node_forces();
        restrict_add(3 * J + comp);
      }
    } else {
      for (int comp = 0; comp < 3; ++comp) {
        // synthetic displacements P Pi_J e_comp at the tile's nodes
        for (int i = threadIdx.x; i < T.L; i += kTileThreads) {
          const float v = ((__float_as_int(stage[i].x) >> (28 + comp)) & 1) ? hat(i, jx, jy, jz) : 0.f;
          T.su[i] = make_float4(comp == 0 ? v : 0.f, comp == 1 ? v : 0.f, comp == 2 ? v : 0.f, 0.f);
        }
        __syncthreads();
        TileOwnW Wn;
        tile_strains(A, R, T, Wn);
        __syncthreads();
        tile_forces(R, T, Wn, lam, mu);
        __syncthreads();
        node_forces();
        restrict_add(3 * J + comp);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) atomicMax(maxdist, tile_md);
}

// A <- (A + A^T) / 2 on the nc x nc block; padding: identity; a zero
// diagonal (a function on prescribed DOFs only) becomes 1
__global__ void k_cs_symmetrize(double *A, int nc, int npad) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)npad * npad) return;
  const int i = (int)(e / npad), j = (int)(e % npad);
  if (i >= nc || j >= nc) {
    A[e] = (i == j) ? 1.0 : 0.0;
    return;
  }
  if (i == j) {
    if (!(A[e] > 0.0)) A[e] = 1.0;
    return;
  }
  if (j < i) {
    const double s = 0.5 * (A[e] + A[(int64_t)j * npad + i]);
    A[e] = s;
    A[(int64_t)j * npad + i] = s;
  }
}

// ---- dense blocked Cholesky (FP64), triangular inverse and W^T W (FP32) --------

template <class T>
struct Tile64 {
  T v[kCB][kCB + 1];
};

// acc += op(A) op(B) over one 64-deep slice; A, B 64 x 64 tiles in smem;
// thread owns rows tm..tm+3 and columns tn..tn+3 of the output
template <class T, bool TA, bool TB>
__device__ __forceinline__ void mm64(T (&acc)[4][4], const Tile64<T> &As, const Tile64<T> &Bs, int tm, int tn) {
#pragma unroll 8
  for (int k = 0; k < kCB; ++k) {
    T a[4], b[4];
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      a[x] = TA ? As.v[k][tm + x] : As.v[tm + x][k];
      b[x] = TB ? Bs.v[tn + x][k] : Bs.v[k][tn + x];
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
  }
}

template <class T>
__device__ __forceinline__ void load64(Tile64<T> &S, const T *A, int64_t ld, int bi, int bj) {
  for (int e = threadIdx.x; e < kCB * kCB; e += blockDim.x)
    S.v[e / kCB][e % kCB] = A[(int64_t)(bi * kCB + e / kCB) * ld + bj * kCB + e % kCB];
}

// factor the diagonal block k, right-looking one column at a time: thread
// (r = tid % 64, q0 = tid / 64) keeps L[r][q0 + 4m] (m < 16) in registers; at
// column j the owners of column j publish it (double-buffered), and after one
// barrier every thread applies the rank-1 update scaled by 1 / L_jj.  Then
// W_kk = L_kk^-1 the same way with thread (c = tid % 64, g = tid / 64)
// holding W[g + 4m][c]: row j is final after the rows above it, divided by
// L_jj and published.  Loops over j and m are unrolled so that the register
// arrays are indexed by constants.  L_kk back to A, W_kk to Wd[k].  A
// non-positive or non-finite pivot sets *info and is replaced by 1.
template <class T>
__global__ void __launch_bounds__(256) k_potrf_diag(T *A, T *Wd, int npad, int k, int *info) {
  extern __shared__ __align__(16) unsigned char dyn_raw[];
  Tile64<T> &L = *reinterpret_cast<Tile64<T> *>(dyn_raw);
  __shared__ T buf[2][kCB];
  const int tid = threadIdx.x;
  load64(L, A, npad, k, k);
  __syncthreads();
  const int r = tid & 63, q0 = tid >> 6;
  T a[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) a[m] = L.v[r][q0 + 4 * m];
  bool bad = false;
#pragma unroll
  for (int j = 0; j < kCB; ++j) {
    T *cj = buf[j & 1];
    if (q0 == (j & 3) && r >= j) cj[r] = a[j >> 2];  // column j below the diagonal, and L_jj
    __syncthreads();
    T d = cj[j];
    if (!(d > T(0)) || !isfinite(d)) {
      bad = true;
      d = T(1);
    }
    const T sd = sqrt(d), inv = T(1) / sd, inv2 = inv * inv;
    if (r > j) {
      const T cr = cj[r] * inv2;
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const int q = q0 + 4 * m;
        if (q > j && q <= r) a[m] -= cr * cj[q];
      }
    }
    if (q0 == (j & 3) && r >= j) a[j >> 2] = (r == j) ? sd : a[j >> 2] * inv;
  }
  if (bad && tid == 0) atomicExch(info, 1);
  __syncthreads();
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    const int q = q0 + 4 * m;
    L.v[r][q] = (q <= r) ? a[m] : T(0);
  }
  __syncthreads();
  // W = L^-1 (lower)
  const int c = r, g = q0;
  T w[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) w[m] = (g + 4 * m == c) ? T(1) : T(0);
#pragma unroll
  for (int j = 0; j < kCB; ++j) {
    T *rj = buf[j & 1];
    if (g == (j & 3)) {
      w[j >> 2] = (c <= j) ? w[j >> 2] / L.v[j][j] : T(0);
      rj[c] = w[j >> 2];
    }
    __syncthreads();
    const T wj = rj[c];
#pragma unroll
    for (int m = 0; m < 16; ++m)
      if (g + 4 * m > j) w[m] -= L.v[g + 4 * m][j] * wj;
  }
  for (int e = tid; e < kCB * kCB; e += blockDim.x) {
    const int i = e / kCB, l = e % kCB;
    A[(int64_t)(k * kCB + i) * npad + k * kCB + l] = L.v[i][l];
  }
#pragma unroll
  for (int m = 0; m < 16; ++m) Wd[(int64_t)k * kCB * kCB + (g + 4 * m) * kCB + c] = w[m];
}

// L[i][k] = A[i][k] W_kk^T for the row blocks k < i <= k + bwb
template <class T>
__global__ void __launch_bounds__(256) k_trsm_panel(T *A, const T *Wd, int npad, int k) {
  extern __shared__ __align__(16) unsigned char dyn_raw[];
  Tile64<T> &X = *reinterpret_cast<Tile64<T> *>(dyn_raw);
  Tile64<T> &Wk = *reinterpret_cast<Tile64<T> *>(dyn_raw + sizeof(Tile64<T>));
  const int bi = k + 1 + blockIdx.x;
  load64(X, A, npad, bi, k);
  load64(Wk, Wd + (int64_t)k * kCB * kCB, kCB, 0, 0);
  __syncthreads();
  const int tm = (threadIdx.x >> 4) * 4, tn = (threadIdx.x & 15) * 4;
  T acc[4][4] = {};
  mm64<T, false, true>(acc, X, Wk, tm, tn);
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) A[(int64_t)(bi * kCB + tm + x) * npad + k * kCB + tn + y] = acc[x][y];
}

// A[i][j] -= L[i][k] L[j][k]^T for k < j <= i <= k + m (block pairs enumerated)
template <class T>
__global__ void __launch_bounds__(256) k_syrk_update(T *A, int npad, int k, int m) {
  extern __shared__ __align__(16) unsigned char dyn_raw[];
  Tile64<T> &Li = *reinterpret_cast<Tile64<T> *>(dyn_raw);
  Tile64<T> &Lj = *reinterpret_cast<Tile64<T> *>(dyn_raw + sizeof(Tile64<T>));
  const int t = blockIdx.x;
  int ii = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((ii + 1) * (ii + 2) / 2 <= t) ++ii;
  while (ii * (ii + 1) / 2 > t) --ii;
  const int jj = t - ii * (ii + 1) / 2;
  if (ii >= m || jj > ii) return;
  const int bi = k + 1 + ii, bj = k + 1 + jj;
  load64(Li, A, npad, bi, k);
  load64(Lj, A, npad, bj, k);
  __syncthreads();
  const int tm = (threadIdx.x >> 4) * 4, tn = (threadIdx.x & 15) * 4;
  T acc[4][4] = {};
  mm64<T, false, true>(acc, Li, Lj, tm, tn);
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) A[(int64_t)(bi * kCB + tm + x) * npad + bj * kCB + tn + y] -= acc[x][y];
}

__global__ void k_lower_to_f32(const double *A, float *L, int npad) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)npad * npad) return;
  const int i = (int)(e / npad), j = (int)(e % npad);
  L[e] = (j <= i) ? (float)A[e] : 0.f;
}

// W = L^-1 (FP32), one block per block column j, walking down the column:
// W_jj from Wd, then W_ij = -W_ii sum_{l} L_il W_lj over the band of L
__global__ void __launch_bounds__(256) k_trtri_cols(const float *L, const float *Wd, float *W, int npad, int nb,
                                                    int bwb) {
  __shared__ Tile64<float> As, Bs;
  const int bj = blockIdx.x;
  const int tm = (threadIdx.x >> 4) * 4, tn = (threadIdx.x & 15) * 4;
  for (int e = threadIdx.x; e < kCB * kCB; e += blockDim.x)
    W[(int64_t)(bj * kCB + e / kCB) * npad + bj * kCB + e % kCB] = Wd[(int64_t)bj * kCB * kCB + e];
  for (int bi = bj + 1; bi < nb; ++bi) {
    float acc[4][4] = {};
    for (int l = max(bj, bi - bwb); l < bi; ++l) {
      __syncthreads();  // W_lj of the previous steps is in global memory
      load64(As, L, npad, bi, l);
      load64(Bs, W, npad, l, bj);
      __syncthreads();
      mm64<float, false, false>(acc, As, Bs, tm, tn);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < kCB * kCB; e += blockDim.x)
      As.v[e / kCB][e % kCB] = Wd[(int64_t)bi * kCB * kCB + e];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) Bs.v[tm + x][tn + y] = acc[x][y];
    __syncthreads();
    float out[4][4] = {};
    mm64<float, false, false>(out, As, Bs, tm, tn);
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) W[(int64_t)(bi * kCB + tm + x) * npad + bj * kCB + tn + y] = -out[x][y];
  }
}

// The same column recurrence with the column's last bwb blocks W_lj kept in
// a shared-memory ring (slot l mod bwb), so that a step loads only its L
// blocks and W_ii, all issued together.  Shared memory: 2 bwb + 2 tiles.
__global__ void __launch_bounds__(256) k_trtri_ring(const float *L, const float *Wd, float *W, int npad, int nb,
                                                    int bwb) {
  extern __shared__ __align__(16) unsigned char dyn_raw[];
  Tile64<float> *ring = reinterpret_cast<Tile64<float> *>(dyn_raw);
  Tile64<float> *Lt = ring + bwb;
  Tile64<float> &D = Lt[bwb];
  Tile64<float> &S = Lt[bwb + 1];
  const int bj = blockIdx.x;
  const int tm = (threadIdx.x >> 4) * 4, tn = (threadIdx.x & 15) * 4;
  for (int e = threadIdx.x; e < kCB * kCB; e += blockDim.x) {
    const float v = Wd[(int64_t)bj * kCB * kCB + e];
    ring[bj % bwb].v[e / kCB][e % kCB] = v;
    W[(int64_t)(bj * kCB + e / kCB) * npad + bj * kCB + e % kCB] = v;
  }
  for (int bi = bj + 1; bi < nb; ++bi) {
    const int l0 = max(bj, bi - bwb);
    __syncthreads();  // the previous step's ring write and tile reads are done
    for (int l = l0; l < bi; ++l) load64(Lt[l - l0], L, npad, bi, l);
    load64(D, Wd + (int64_t)bi * kCB * kCB, kCB, 0, 0);
    __syncthreads();
    float acc[4][4] = {};
    for (int l = l0; l < bi; ++l) mm64<float, false, false>(acc, Lt[l - l0], ring[l % bwb], tm, tn);
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) S.v[tm + x][tn + y] = acc[x][y];
    __syncthreads();  // S complete; ring slot bi mod bwb (block bi - bwb) no longer read
    float out[4][4] = {};
    mm64<float, false, false>(out, D, S, tm, tn);
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        ring[bi % bwb].v[tm + x][tn + y] = -out[x][y];
        W[(int64_t)(bi * kCB + tm + x) * npad + bj * kCB + tn + y] = -out[x][y];
      }
  }
}

// C[a][b] = sum_{l >= a} W[l][a]^T W[l][b] for a >= b (packed lower blocks)
__global__ void __launch_bounds__(256) k_lauum(const float *W, float *C, int npad, int nb) {
  __shared__ Tile64<float> As, Bs;
  const int t = blockIdx.x;
  int a = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((a + 1) * (a + 2) / 2 <= t) ++a;
  while (a * (a + 1) / 2 > t) --a;
  const int b = t - a * (a + 1) / 2;
  const int tm = (threadIdx.x >> 4) * 4, tn = (threadIdx.x & 15) * 4;
  float acc[4][4] = {};
  for (int l = a; l < nb; ++l) {
    __syncthreads();
    load64(As, W, npad, l, a);
    load64(Bs, W, npad, l, b);
    __syncthreads();
    mm64<float, true, false>(acc, As, Bs, tm, tn);
  }
  // packed lower blocks: block (a, b) at t = a (a + 1) / 2 + b
  float *Cb = C + (int64_t)t * kCB * kCB;
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) Cb[(tm + x) * kCB + tn + y] = acc[x][y];
}

// the lower 64 x 64 blocks of the dense FP64 matrix A (npad x npad) packed
// in FP32: block (a, b), a >= b, at (a (a + 1) / 2 + b) * 4096, row-major
__global__ void k_cs_pack_lower(const double *__restrict__ A, float *__restrict__ P, int npad, int nb) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)nb * (nb + 1) / 2 * kCB * kCB;
  if (e >= total) return;
  const int64_t t = e / (kCB * kCB);
  const int w = (int)(e - t * kCB * kCB), i = w / kCB, j = w % kCB;
  int a = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((int64_t)(a + 1) * (a + 2) / 2 <= t) ++a;
  while ((int64_t)a * (a + 1) / 2 > t) --a;
  const int b = (int)(t - (int64_t)a * (a + 1) / 2);
  P[e] = (float)A[(int64_t)(a * kCB + i) * npad + b * kCB + j];
}

// z = D^-1 r + P Pi yc
__global__ void k_cs_apply_z(CoarseDev cs, const double *__restrict__ r, const double *__restrict__ dinv,
                             const uint8_t *__restrict__ dmask, int64_t n, double *__restrict__ z) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] = dinv[i] * r[i] + (dmask[i] ? (double)cs_prolong(cs, i) : 0.0);
}

void coarse_gemv(const CoarseDev &cs, cudaStream_t st, const int *done, double *rzc) {
  const int nb = cs.npad / kCB;
  k_cs_symv<<<nb * (nb + 1) / 2, kSymvThreads, 0, st>>>(cs, done, rzc);
  SFEM_CHECK_LAUNCH();
}

template <class TV>
static void coarse_correction_t(Ctx &c, cudaStream_t st, const TV *r, const int *done) {
  const CoarseDev &cs = c.coarse->dev;
  k_cs_restrict<TV><<<cs.ncell, kRestrictThreads, 0, st>>>(r, nullptr, cs, done);
  SFEM_CHECK_LAUNCH();
  k_cs_gather<<<grid_for(cs.npad, 256), 256, 0, st>>>(cs, done);
  SFEM_CHECK_LAUNCH();
  coarse_gemv(cs, st, done);
}
void coarse_correction(Ctx &c, cudaStream_t st, const double *r, const int *done) {
  coarse_correction_t(c, st, r, done);
}
void coarse_restrict(Ctx &c, cudaStream_t st, const double *r, const int *done) {
  const CoarseDev &cs = c.coarse->dev;
  k_cs_restrict<double><<<cs.ncell, kRestrictThreads, 0, st>>>(r, nullptr, cs, done);
  SFEM_CHECK_LAUNCH();
  k_cs_gather<<<grid_for(cs.npad, 256), 256, 0, st>>>(cs, done);
  SFEM_CHECK_LAUNCH();
}
void coarse_correction(Ctx &c, cudaStream_t st, const float *r, const int *done) {
  coarse_correction_t(c, st, r, done);
}

// ---- coarse-space tables ---------------------------------------------------

struct CsGrid {
  double lo[3], ext[3];
  int d[3], cd[3];
};

// interpolation cell, lower-corner centre (with axis flags) and fractions
// of every node: t = (x - lo) / ext * d - 1/2 clamped to [0, d - 1], cell
// index floor(t) clamped to [0, d - 2]
__global__ void k_cs_locate(const double *__restrict__ xyz, int64_t n_nodes, CsGrid g, int32_t *__restrict__ cell,
                            int32_t *__restrict__ cinfo, float *__restrict__ frac) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  int i0[3];
  for (int a = 0; a < 3; ++a) {
    double t = (xyz[3 * i + a] - g.lo[a]) / g.ext[a] * g.d[a] - 0.5;
    t = fmin(fmax(t, 0.0), (double)max(g.d[a] - 1, 0));
    i0[a] = min(max((int)floor(t), 0), max(g.d[a] - 2, 0));
    frac[3 * i + a] = (float)(g.d[a] > 1 ? t - i0[a] : 0.0);
  }
  cell[i] = (i0[0] * g.cd[1] + i0[1]) * g.cd[2] + i0[2];
  cinfo[i] = ((i0[0] * g.d[1] + i0[1]) * g.d[2] + i0[2]) | ((i0[0] + 1 < g.d[0]) << 24) |
             ((i0[1] + 1 < g.d[1]) << 25) | ((i0[2] + 1 < g.d[2]) << 26);
}

constexpr int kGroupNodes = 1024;  // nodes per block of the grouping sort

// nodes of block b per cell, stored cell-major: hist[cell * nblk + b]
__global__ void k_cs_group_hist(const int32_t *__restrict__ cell, int64_t n_nodes, int ncell, int nblk,
                                int32_t *__restrict__ hist) {
  extern __shared__ int32_t gsm[];
  for (int q = threadIdx.x; q < ncell; q += blockDim.x) gsm[q] = 0;
  __syncthreads();
  const int64_t b0 = (int64_t)blockIdx.x * kGroupNodes;
  for (int k = threadIdx.x; k < kGroupNodes && b0 + k < n_nodes; k += blockDim.x) atomicAdd(&gsm[cell[b0 + k]], 1);
  __syncthreads();
  for (int q = threadIdx.x; q < ncell; q += blockDim.x) hist[(int64_t)q * nblk + blockIdx.x] = gsm[q];
}

// place block b's nodes in node order from the cell-major exclusive offsets
// (one thread walks the block: the order within a cell stays ascending)
__global__ void k_cs_group_place(const int32_t *__restrict__ cell, int64_t n_nodes, int ncell, int nblk,
                                 const int64_t *__restrict__ base, int32_t *__restrict__ nodes) {
  extern __shared__ int32_t gsm[];
  int32_t *cur = gsm, *cl = gsm + ncell;
  for (int q = threadIdx.x; q < ncell; q += blockDim.x) cur[q] = (int32_t)base[(int64_t)q * nblk + blockIdx.x];
  const int64_t b0 = (int64_t)blockIdx.x * kGroupNodes;
  const int m = (int)(n_nodes - b0 < kGroupNodes ? n_nodes - b0 : kGroupNodes);
  for (int k = threadIdx.x; k < m; k += blockDim.x) cl[k] = cell[b0 + k];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int k = 0; k < m; ++k) nodes[cur[cl[k]]++] = (int32_t)(b0 + k);
}

// first node of each cell in the grouped order; off[ncell] = n_nodes
__global__ void k_cs_group_off(const int64_t *__restrict__ base, int ncell, int nblk, int64_t n_nodes,
                               int32_t *__restrict__ off) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < ncell) off[q] = (int32_t)base[(int64_t)q * nblk];
  if (q == ncell) off[q] = (int32_t)n_nodes;
}

__global__ void k_cs_to_f32(const double *a, float *b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// blocked Cholesky of the band of A (lower blocks within bwb of the
// diagonal) in place, with the inverses of the diagonal blocks in Wd;
// false on a non-positive pivot.  (The whole band in one CTA, diagonal
// block, panel and trailing blocks per step in shared memory, took 3.7
// instead of 2.8 ms on the 2M-tet beam's 50 block steps: one SM's GEMM
// throughput; the diagonal factor with its j loops not unrolled, 3.2 ms.)
template <class T>
static bool banded_cholesky(Ctx &c, T *A, T *Wd, int npad, int nb, int bwb, int *dev_info) {
  const size_t sm2 = 2 * sizeof(Tile64<T>);
  SFEM_CUDA(cudaFuncSetAttribute(k_potrf_diag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
  SFEM_CUDA(cudaFuncSetAttribute(k_trsm_panel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
  SFEM_CUDA(cudaFuncSetAttribute(k_syrk_update<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
  SFEM_CUDA(cudaMemsetAsync(dev_info, 0, sizeof(int), c.stream));
  for (int k = 0; k < nb; ++k) {
    k_potrf_diag<T><<<1, 256, sm2, c.stream>>>(A, Wd, npad, k, dev_info);
    SFEM_CHECK_LAUNCH();
    const int m = std::min(nb - 1 - k, bwb);  // nonzero row blocks below the diagonal block
    if (m == 0) continue;
    k_trsm_panel<T><<<m, 256, sm2, c.stream>>>(A, Wd, npad, k);
    SFEM_CHECK_LAUNCH();
    k_syrk_update<T><<<m * (m + 1) / 2, 256, sm2, c.stream>>>(A, npad, k, m);
    SFEM_CHECK_LAUNCH();
  }
  int info = 0;
  SFEM_CUDA(cudaMemcpyAsync(&info, dev_info, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  SFEM_CUDA(cudaStreamSynchronize(c.stream));
  return info == 0;
}

static void setup_coarse(Ctx &c, const sfem_coarse_opts *opts) {
  cudaEvent_t e0, e1;
  SFEM_CUDA(cudaEventCreate(&e0));
  SFEM_CUDA(cudaEventCreate(&e1));
  SFEM_CUDA(cudaEventRecord(e0, c.stream));
  auto co = std::make_shared<Coarse>();
  // grid of centres over the nodes' bounding box (found with the tiles)
  const double *lo = c.bbox_lo, *hi = c.bbox_hi;
  const bool auto_pn = !(opts && opts->patch_nodes > 0);
  int pn = auto_pn ? 8 : opts->patch_nodes;
  const double box = std::max((hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2]), 1e-300);
  const double h_mean = std::cbrt(box / (double)c.n_nodes);
  CoarseDev &cs = co->dev;
  int64_t P = 1;
  for (;;) {
    P = 1;
    bool any_auto = false;
    for (int a = 0; a < 3; ++a) {
      co->g.lo[a] = lo[a];
      co->g.ext[a] = std::max(hi[a] - lo[a], 1e-300);
      const int req = opts ? opts->patch_dims[a] : 0;
      SFEM_REQUIRE(req >= 0 && req <= 4096, SFEM_EINVAL, "patch_dims out of range");
      any_auto |= req == 0;
      co->g.d[a] = req > 0 ? req : std::max(1, (int)std::ceil((hi[a] - lo[a]) / (pn * h_mean) - 1e-9));
      cs.d[a] = co->g.d[a];
      cs.cd[a] = std::max(cs.d[a] - 1, 1);
      P *= cs.d[a];
    }
    // the default patch width grows until the coarse space fits (large meshes)
    if (3 * P <= kMaxCoarse || !auto_pn || !any_auto || pn >= 4096) break;
    ++pn;
  }
  SFEM_REQUIRE(3 * P <= kMaxCoarse, SFEM_EINVAL, "coarse space larger than 8192 DOFs");
  // probing assumes centres three or more cells apart are uncoupled: patches
  // must span a few elements (checked against the mean node spacing)
  for (int a = 0; a < 3; ++a)
    SFEM_REQUIRE(cs.d[a] < 5 || co->g.ext[a] / cs.d[a] >= 2.5 * h_mean, SFEM_EINVAL,
                 "patches narrower than 2.5 node spacings");
  cs.nc = (int)(3 * P);
  cs.npad = (cs.nc + kCB - 1) / kCB * kCB;
  cs.ncell = cs.cd[0] * cs.cd[1] * cs.cd[2];
  // interpolation cell and fractions of every node (k_cs_locate); nodes
  // grouped by cell, ascending within a cell, by a stable counting sort
  // over blocks of kGroupNodes nodes (histogram per block, one scan over
  // the cell-major block histograms, then placement in node order)
  int32_t *d_cell = c.mem.get<int32_t>(c.n_nodes), *d_nodes = c.mem.get<int32_t>(c.n_nodes);
  int32_t *d_off = c.mem.get<int32_t>(cs.ncell + 1), *d_cinfo = c.mem.get<int32_t>(c.n_nodes);
  float *d_frac = c.mem.get<float>(3 * c.n_nodes);
  {
    CsGrid gr;
    for (int a = 0; a < 3; ++a) {
      gr.lo[a] = co->g.lo[a];
      gr.ext[a] = co->g.ext[a];
      gr.d[a] = cs.d[a];
      gr.cd[a] = cs.cd[a];
    }
    k_cs_locate<<<grid_for(c.n_nodes, 256), 256, 0, c.stream>>>(c.xyz, c.n_nodes, gr, d_cell, d_cinfo, d_frac);
    SFEM_CHECK_LAUNCH();
    const int nblk = (int)((c.n_nodes + kGroupNodes - 1) / kGroupNodes);
    const int64_t nh = (int64_t)cs.ncell * nblk;
    int32_t *hist = c.mem.get<int32_t>(nh);
    int64_t *base = c.mem.get<int64_t>(nh + 1);
    const size_t gsm = (size_t)cs.ncell * sizeof(int32_t) + kGroupNodes * sizeof(int32_t);
    SFEM_REQUIRE(gsm <= 200 * 1024, SFEM_EINVAL, "too many interpolation cells");
    SFEM_CUDA(cudaFuncSetAttribute(k_cs_group_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm));
    SFEM_CUDA(cudaFuncSetAttribute(k_cs_group_place, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm));
    k_cs_group_hist<<<nblk, 256, gsm, c.stream>>>(d_cell, c.n_nodes, cs.ncell, nblk, hist);
    SFEM_CHECK_LAUNCH();
    scan_counts(c, hist, nh, base);
    k_cs_group_place<<<nblk, 256, gsm, c.stream>>>(d_cell, c.n_nodes, cs.ncell, nblk, base, d_nodes);
    SFEM_CHECK_LAUNCH();
    k_cs_group_off<<<grid_for(cs.ncell + 1, 256), 256, 0, c.stream>>>(base, cs.ncell, nblk, c.n_nodes, d_off);
    SFEM_CHECK_LAUNCH();
    c.mem.drop(hist);
    c.mem.drop(base);
  }
  std::vector<int32_t> off(cs.ncell + 1);
  SFEM_CUDA(cudaMemcpyAsync(off.data(), d_off, off.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
  // per coarse DOF the cellsum entries (cell, corner) that restrict onto it
  std::vector<int32_t> glist(8 * (size_t)cs.nc, -1);
  for (int j = 0; j < (int)P; ++j) {
    const int jz = j % cs.d[2], jy = (j / cs.d[2]) % cs.d[1], jx = j / (cs.d[1] * cs.d[2]);
    int n = 0;
    for (int ix = std::max(0, jx - 1); ix <= std::min(cs.cd[0] - 1, jx); ++ix)
      for (int bx = 0; bx < 2; ++bx) {
        if (std::min(ix + bx, cs.d[0] - 1) != jx) continue;
        for (int iy = std::max(0, jy - 1); iy <= std::min(cs.cd[1] - 1, jy); ++iy)
          for (int by = 0; by < 2; ++by) {
            if (std::min(iy + by, cs.d[1] - 1) != jy) continue;
            for (int iz = std::max(0, jz - 1); iz <= std::min(cs.cd[2] - 1, jz); ++iz)
              for (int bz = 0; bz < 2; ++bz) {
                if (std::min(iz + bz, cs.d[2] - 1) != jz) continue;
                const int q = (ix * cs.cd[1] + iy) * cs.cd[2] + iz;
                const int k = (bx << 2) | (by << 1) | bz;
                SFEM_REQUIRE(n < 8, SFEM_EINVAL, "coarse gather list overflow");
                for (int cc = 0; cc < 3; ++cc) glist[8 * (size_t)(3 * j + cc) + n] = 24 * q + 3 * k + cc;
                ++n;
              }
          }
      }
  }
  SFEM_CUDA(cudaStreamSynchronize(c.stream));  // off
  // blocks of the restriction in the two-level iterations: runs of at most
  // kChunkNodes nodes of one cell (256 per warp)
  std::vector<int4> chunks;
  for (int q = 0; q < cs.ncell; ++q)
    for (int b = off[q]; b < off[q + 1]; b += kChunkNodes)
      chunks.push_back(make_int4(q, b, std::min(b + kChunkNodes, off[q + 1]), 0));
  cs.nchunk = (int)chunks.size();
  int4 *d_chunk = c.mem.get<int4>(chunks.size());
  SFEM_CUDA(cudaMemcpyAsync(d_chunk, chunks.data(), chunks.size() * sizeof(int4), cudaMemcpyHostToDevice, c.stream));
  cs.chunk = d_chunk;
  // the same runs split to at most kSubNodes nodes (update items of the
  // batched solver)
  std::vector<int4> subs;
  for (const int4 &ch : chunks)
    for (int b = ch.y; b < ch.z; b += kSubNodes) subs.push_back(make_int4(ch.x, b, std::min(b + kSubNodes, ch.z), 0));
  cs.nsub = (int)subs.size();
  int4 *d_sub = c.mem.get<int4>(subs.size());
  SFEM_CUDA(cudaMemcpyAsync(d_sub, subs.data(), subs.size() * sizeof(int4), cudaMemcpyHostToDevice, c.stream));
  cs.sub = d_sub;
  int32_t *d_glist = c.mem.get<int32_t>(glist.size());
  SFEM_CUDA(cudaMemcpyAsync(d_glist, glist.data(), glist.size() * 4, cudaMemcpyHostToDevice, c.stream));
  cs.cinfo = d_cinfo;
  cs.glist = d_glist;
  cs.cell = d_cell;
  cs.cnodes = d_nodes;
  cs.coff = d_off;
  cs.frac = d_frac;
  cs.cellsum = c.mem.get<float>(24 * (size_t)cs.ncell);
  cs.rc = c.mem.get<float>(cs.npad);
  cs.yc = c.mem.get<float>(cs.npad);
  SFEM_CUDA(cudaMemsetAsync(cs.rc, 0, cs.npad * sizeof(float), c.stream));
  SFEM_CUDA(cudaMemsetAsync(cs.yc, 0, cs.npad * sizeof(float), c.stream));
  // ---- A_c by probing with the FP32 tiled operator --------------------------
  const int64_t np2 = (int64_t)cs.npad * cs.npad;
  double *Ac = c.mem.get<double>(np2);
  SFEM_CUDA(cudaMemsetAsync(Ac, 0, np2 * sizeof(double), c.stream));
  int probes = 0, maxdist = 0;
  const int assembly = opts ? opts->assembly : 0;
  SFEM_REQUIRE(assembly == 0 || assembly == 1, SFEM_EINVAL, "assembly must be 0 or 1");
  if (assembly == 0) {
    // tile by tile (exact Galerkin entries, no colouring)
    int *ovf = c.mem.get<int>(2);  // [0] overflow, [1] largest |row - column|
    SFEM_CUDA(cudaMemsetAsync(ovf, 0, 2 * sizeof(int), c.stream));
    const int stage_off = (int)((c.tl.smem + 15) / 16);
    const size_t smem = (size_t)stage_off * 16 + (size_t)c.tl.max_nodes * (2 * sizeof(float4) + sizeof(uint16_t)) + 16;
    SFEM_REQUIRE(smem <= 227 * 1024, SFEM_EINVAL, "tile too large for the Galerkin assembly");
    SFEM_CUDA(cudaFuncSetAttribute(k_cs_galerkin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    TileArgs TA{c.tl.tile_start, c.tl.hoff, c.tl.noff, c.tl.halo_tet, c.tl.halo_lconn, c.tl.tile_nodes,
                c.tl.node_inc, c.tl.rec, c.n_tets, c.tl.slot_stride};
    k_cs_galerkin<<<(unsigned)c.tl.n_tiles, kTileThreads, smem, c.stream>>>(TA, cs, c.dmask, (float)c.lam,
                                                                              (float)c.mu, stage_off, Ac, ovf,
                                                                              ovf + 1);
    SFEM_CHECK_LAUNCH();
    int hovf[2] = {0, 0};
    SFEM_CUDA(cudaMemcpyAsync(hovf, ovf, sizeof hovf, cudaMemcpyDeviceToHost, c.stream));
    SFEM_CUDA(cudaStreamSynchronize(c.stream));
    c.mem.drop(ovf);
    if (hovf[0]) {
      SFEM_CUDA(cudaMemsetAsync(Ac, 0, np2 * sizeof(double), c.stream));  // probe instead
    } else {
      probes = -1;
      maxdist = hovf[1];
    }
  }
  if (probes >= 0)  // probing attributes entries to centres at most 2 cells apart per axis
    maxdist = 3 * (2 * cs.d[1] * cs.d[2] + 2 * cs.d[2] + 2) + 2;
  float *v = c.mem.get<float>(c.ndof), *y = c.mem.get<float>(c.ndof);
  const int3 str = make_int3(std::min(5, cs.d[0]), std::min(5, cs.d[1]), std::min(5, cs.d[2]));
  for (int comp = 0; comp < 3 && probes >= 0; ++comp)
    for (int rx = 0; rx < str.x; ++rx)
      for (int ry = 0; ry < str.y; ++ry)
        for (int rz = 0; rz < str.z; ++rz) {
          const int3 res = make_int3(rx, ry, rz);
          k_cs_probe<<<grid_for(c.n_nodes, 256), 256, 0, c.stream>>>(cs, c.n_nodes, c.dmask, comp, res, str, v);
          SFEM_CHECK_LAUNCH();
          SFEM_CUDA(cudaMemsetAsync(y, 0, c.ndof * sizeof(float), c.stream));
          launch_mf32_tiled<float, float>(c, c.stream, v, y, nullptr, nullptr);
          k_cs_restrict<float><<<cs.ncell, kRestrictThreads, 0, c.stream>>>(y, c.dmask, cs, nullptr);
          SFEM_CHECK_LAUNCH();
          k_cs_gather<<<grid_for(cs.npad, 256), 256, 0, c.stream>>>(cs, nullptr);
          SFEM_CHECK_LAUNCH();
          k_cs_attrib<<<grid_for(cs.nc, 256), 256, 0, c.stream>>>(cs, comp, res, str, Ac);
          SFEM_CHECK_LAUNCH();
          ++probes;
        }
  c.mem.drop(v);
  c.mem.drop(y);
  k_cs_symmetrize<<<grid_for(np2, 256), 256, 0, c.stream>>>(Ac, cs.nc, cs.npad);
  SFEM_CHECK_LAUNCH();
  {  // A_c itself, packed in FP32 (the learned coarse correction's step length)
    const int nbp = cs.npad / kCB;
    const int64_t tot = (int64_t)nbp * (nbp + 1) / 2 * kCB * kCB;
    float *Ap = c.mem.get<float>(tot);
    k_cs_pack_lower<<<grid_for(tot, 256), 256, 0, c.stream>>>(Ac, Ap, cs.npad, nbp);
    SFEM_CHECK_LAUNCH();
    cs.Ap = Ap;
  }
  // ---- banded blocked Cholesky ---------------------------------------------
  // FP32 (the inverse C is FP32 anyway: on the 26 x 6 x 6 grid of the 2M-tet
  // beam, cond(A_c) ~ 8e4, and C from an FP32 factor has C A_c within 1.4e-4
  // of I, as with an FP64 factor); FP64 when the FP32 factor meets a
  // non-positive pivot
  const int nb = cs.npad / kCB;
  int *dev_i = c.mem.get<int>(1);  // Cholesky info
  // block bandwidth: an entry |row - column| = m apart lies at most m/64 + 1
  // block rows below the diagonal block of its column
  const int bwb = std::min(std::max(maxdist / kCB + 1, 1), nb - 1 > 0 ? nb - 1 : 1);
  float *L32 = c.mem.get<float>(np2);
  float *Wd = c.mem.get<float>((size_t)nb * kCB * kCB);
  k_cs_to_f32<<<grid_for(np2, 256), 256, 0, c.stream>>>(Ac, L32, np2);
  SFEM_CHECK_LAUNCH();
  const int factor = opts ? opts->factor : 0;
  co->fp64_factor = factor == 1 || !banded_cholesky<float>(c, L32, Wd, cs.npad, nb, bwb, dev_i);
  if (co->fp64_factor) {
    double *Wd64 = c.mem.get<double>((size_t)nb * kCB * kCB);
    SFEM_REQUIRE(banded_cholesky<double>(c, Ac, Wd64, cs.npad, nb, bwb, dev_i), SFEM_EBREAKDOWN,
                 "coarse matrix is not positive definite");
    k_lower_to_f32<<<grid_for(np2, 256), 256, 0, c.stream>>>(Ac, L32, cs.npad);
    SFEM_CHECK_LAUNCH();
    k_cs_to_f32<<<grid_for((int64_t)nb * kCB * kCB, 256), 256, 0, c.stream>>>(Wd64, Wd, (int64_t)nb * kCB * kCB);
    SFEM_CHECK_LAUNCH();
    c.mem.drop(Wd64);
  }
  c.mem.drop(Ac);
  // ---- C = A_c^-1 = L^-T L^-1 (FP32) ----------------------------------------
  // (trtri reads only the strictly lower blocks of L and the diagonal blocks'
  // inverses Wd)
  float *W = c.mem.get<float>(np2);
  float *C = c.mem.get<float>((size_t)nb * (nb + 1) / 2 * kCB * kCB);
  SFEM_CUDA(cudaMemsetAsync(W, 0, np2 * sizeof(float), c.stream));
  const size_t smr = (2 * (size_t)bwb + 2) * sizeof(Tile64<float>);
  if (smr <= 200 * 1024) {  // 1.27 -> 0.91 ms on the 2M-tet beam's 3150 coarse DOFs
    SFEM_CUDA(cudaFuncSetAttribute(k_trtri_ring, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smr));
    k_trtri_ring<<<nb, 256, smr, c.stream>>>(L32, Wd, W, cs.npad, nb, bwb);
  } else {
    k_trtri_cols<<<nb, 256, 0, c.stream>>>(L32, Wd, W, cs.npad, nb, bwb);
  }
  SFEM_CHECK_LAUNCH();
  k_lauum<<<nb * (nb + 1) / 2, 256, 0, c.stream>>>(W, C, cs.npad, nb);
  SFEM_CHECK_LAUNCH();
  c.mem.drop(L32);
  c.mem.drop(W);
  c.mem.drop(Wd);
  c.mem.drop(dev_i);
  cs.C = C;
  co->probes = std::max(probes, 0);  // 0: assembled tile by tile
  SFEM_CUDA(cudaEventRecord(e1, c.stream));
  SFEM_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  SFEM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  co->setup_ms = ms;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c.coarse = co;
}

bool ensure_coarse(Ctx &c, int patch_nodes) {
  if (c.coarse) return true;
  if (patch_nodes > 0) {
    sfem_coarse_opts o{};
    o.patch_nodes = patch_nodes;
    try {
      setup_coarse(c, &o);
      return true;
    } catch (const Error &) {
      c.coarse.reset();  // e.g. A_c not positive definite with narrow patches: the default grid next
    }
  }
  try {
    setup_coarse(c, nullptr);
  } catch (const Error &) {
    c.coarse.reset();
    return false;  // no coarse space for this mesh (e.g. patches too narrow)
  }
  return true;
}

}  // namespace sfem

using namespace sfem;

extern "C" int sfem_coarse_setup(sfem_ctx *h, const sfem_coarse_opts *opts) {
  try {
    SFEM_REQUIRE(h && h->c.vol && h->c.tl.ready, SFEM_EINVAL, "context not set up");
    if (opts) {
      for (int r : opts->reserved) SFEM_REQUIRE(r == 0, SFEM_EINVAL, "reserved options must be zero");
      SFEM_REQUIRE(opts->assembly == 0 || opts->assembly == 1, SFEM_EINVAL, "assembly must be 0 or 1");
      SFEM_REQUIRE(opts->factor == 0 || opts->factor == 1, SFEM_EINVAL, "factor must be 0 or 1");
    }
    h->c.coarse.reset();
    setup_coarse(h->c, opts);
  } catch (const Error &err) {
    set_last_error(err.msg);
    return err.status;
  }
  return SFEM_OK;
}

extern "C" int sfem_coarse_info(const sfem_ctx *h, int *patch_dims, int *n_coarse, int *probes, double *setup_ms) {
  if (!h || !h->c.coarse) {
    set_last_error("no coarse space on this context");
    return SFEM_EINVAL;
  }
  const Coarse &co = *h->c.coarse;
  if (patch_dims)
    for (int a = 0; a < 3; ++a) patch_dims[a] = co.dev.d[a];
  if (n_coarse) *n_coarse = co.dev.nc;
  if (probes) *probes = co.probes;
  if (setup_ms) *setup_ms = co.setup_ms;
  return SFEM_OK;
}

extern "C" int sfem_coarse_apply(sfem_ctx *h, const double *r, double *z) {
  try {
    SFEM_REQUIRE(h && h->c.coarse && r && z, SFEM_EINVAL, "context with a coarse space, r and z are required");
    Ctx &c = h->c;
    coarse_correction(c, c.stream, r, nullptr);
    k_cs_apply_z<<<grid_for(c.ndof, 256), 256, 0, c.stream>>>(c.coarse->dev, r, c.dinv64, c.dmask, c.ndof, z);
    SFEM_CHECK_LAUNCH();
    SFEM_CUDA(cudaStreamSynchronize(c.stream));
  } catch (const Error &err) {
    set_last_error(err.msg);
    return err.status;
  }
  return SFEM_OK;
}
