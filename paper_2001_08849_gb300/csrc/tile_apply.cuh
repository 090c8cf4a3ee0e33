// Device side of the tiled single-pass FP32 operator (shared by the
// single-system kernel in tiles.cu and the batched persistent solver in
// batch.cu).  See tiles.cu for the method and the data layout.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "reduce.cuh"

namespace sfem {

constexpr int kTileMax = 512;            // tets per tile
constexpr int kTileThreads = 256;        // threads per tile CTA
constexpr int kTilePer = kTileMax / kTileThreads;
constexpr unsigned short kNoNbr = 0xFFFF;

// Nodal force slots of a tile.  Tile nodes are ordered by their number of
// own slots (slots 4j+a of the tile's tets j whose vertex a is the node),
// largest first, and taken in groups of 32 (one warp of the nodal-sum
// phase).  Slot k of node q lies at position
//   base(q / 32) + 32 k + ((q + k) mod 32)
// of three float arrays (x, y, z components, stride slot_stride): the warp
// summing 32 nodes reads one row of 32 banks per step, and the slots of one
// node fall in different banks, so the tets sharing a node write them
// without bank conflicts.  Each tet writes its four slot forces straight to
// their positions (stored in its record).  Per tile node, node_inc holds
// base(q / 32) | (count << 16).
struct TileArgs {
  const int32_t *tile_start;
  const int64_t *hoff, *noff;
  const int32_t *halo_tet;
  const uint2 *halo_lconn;
  const int32_t *tile_nodes;
  const uint32_t *node_inc;  // per tile node: base of its group | own-slot count << 16
  const float4 *rec;   // 64-byte per-tet records, tile order, as 4 planes of float4 (word 4q..4q+3 of
                       // tet t at rec[q * rs + t]): a warp's loads of one plane are contiguous
  int64_t rs;          // plane stride (the tet count)
  int slot_stride;     // floats per component array of the force slots (a multiple of 32)
};

struct TetGeo {
  float g[4][3];
  float V;
};

__device__ __forceinline__ void rec_unpack(const float4 (&q)[4], TetGeo &G, uint2 &lc) {
  G.g[1][0] = q[0].x, G.g[1][1] = q[0].y, G.g[1][2] = q[0].z;
  G.g[2][0] = q[0].w, G.g[2][1] = q[1].x, G.g[2][2] = q[1].y;
  G.g[3][0] = q[1].z, G.g[3][1] = q[1].w, G.g[3][2] = q[2].x;
  G.V = q[2].y;
  lc = make_uint2(__float_as_uint(q[2].z), __float_as_uint(q[2].w));
#pragma unroll
  for (int i = 0; i < 3; ++i) G.g[0][i] = -(G.g[1][i] + G.g[2][i] + G.g[3][i]);
}

__device__ __forceinline__ void load_rec(const float4 *__restrict__ rec, int64_t rs, int t, TetGeo &G, uint2 &lc,
                                         uint2 *lnb) {
  const float4 a = __ldg(rec + t), b = __ldg(rec + rs + t);
  const float4 c = __ldg(rec + 2 * rs + t);
  G.g[1][0] = a.x, G.g[1][1] = a.y, G.g[1][2] = a.z;
  G.g[2][0] = a.w, G.g[2][1] = b.x, G.g[2][2] = b.y;
  G.g[3][0] = b.z, G.g[3][1] = b.w, G.g[3][2] = c.x;
  G.V = c.y;
  lc = make_uint2(__float_as_uint(c.z), __float_as_uint(c.w));
  if (lnb) {
    const float4 d = __ldg(rec + 3 * rs + t);
    *lnb = make_uint2(__float_as_uint(d.x), __float_as_uint(d.y));
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) G.g[0][i] = -(G.g[1][i] + G.g[2][i] + G.g[3][i]);
}

// w = V_e eps_e (Voigt) from the tile's smem displacements; w[6] = V_e.
// The gradients of a tet sum to zero, so grad u = sum_{a>=1} (u_a - u_0)
// (x) grad N_a: the FP32 arithmetic acts on differences of displacements
// within the tet (no cancellation of a common rigid part).
__device__ __forceinline__ void strain_to(const float4 *su, uint2 lc, const TetGeo &G, float4 *w2) {
  const int l[4] = {(int)(lc.x & 0xFFFF), (int)(lc.x >> 16), (int)(lc.y & 0xFFFF), (int)(lc.y >> 16)};
  float H[3][3] = {};
  const float4 u0 = su[l[0]];
#pragma unroll
  for (int a = 1; a < 4; ++a) {
    const float4 ua = su[l[a]];
    const float dx = ua.x - u0.x, dy = ua.y - u0.y, dz = ua.z - u0.z;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      H[0][j] = fmaf(dx, G.g[a][j], H[0][j]);
      H[1][j] = fmaf(dy, G.g[a][j], H[1][j]);
      H[2][j] = fmaf(dz, G.g[a][j], H[2][j]);
    }
  }
  w2[0] = make_float4(H[0][0], H[1][1], H[2][2], H[1][2] + H[2][1]);
  w2[1] = make_float4(H[2][0] + H[0][2], H[0][1] + H[1][0], G.V, 0.f);
}

// own-tet records of a tile, kept in registers for both phases (and for
// every right-hand side of a batched apply); NT threads per tile, tet
// threadIdx.x + r NT in rr[r]
template <int NT>
struct TileRegsT {
  static constexpr int kPer = kTileMax / NT;
  float4 rr[kPer][4];
};
using TileRegs = TileRegsT<kTileThreads>;

// the strains (w0..w3 | w4, w5, V, 0) of a thread's own tets, kept in
// registers from the strain phase to the force phase (the shared-memory
// copies are for the neighbours; re-reading them cost 2 of the 10 float4
// loads per tet of the force phase)
template <int NT>
struct TileOwnWT {
  float4 w[TileRegsT<NT>::kPer][2];
};
using TileOwnW = TileOwnWT<kTileThreads>;

__device__ __forceinline__ void tile_load(const TileArgs &A, int tile, TileRegs &R) {
  const int s = A.tile_start[tile], n_own = A.tile_start[tile + 1] - s;
#pragma unroll
  for (int r = 0; r < kTilePer; ++r) {
    const int j = threadIdx.x + r * kTileThreads;
    if (j < n_own) {
      const float4 *rp = A.rec + (s + j);
#pragma unroll
      for (int q = 0; q < 4; ++q) R.rr[r][q] = __ldg(rp + q * A.rs);
    }
  }
}

// Shared-memory layout of one tile: displacements (L float4) sharing their
// space with the force slots (three arrays of slot_stride floats; written
// only after the strains have been formed), strains split in two float4
// arrays (w0..w3 | w4, w5, V, 0) over tile + halo tets, and the per-node
// slot position and count.
struct TileView {
  int n_own, H, L, nt, ns;
  int64_t h0, n0;
  float4 *su, *swa, *swb;
  float *sfx;       // x components of the slots; y at sfx + ns, z at sfx + 2 ns
  uint32_t *snode;
};

// float4 words taken by the displacement / force-slot region
__host__ __device__ __forceinline__ int tile_slot_words(int L, int slot_stride) {
  const int fw = (3 * slot_stride + 3) / 4;
  return L > fw ? L : fw;
}

__device__ __forceinline__ TileView tile_view(const TileArgs &A, int tile, float4 *smem) {
  TileView T;
  const int s = A.tile_start[tile];
  T.n_own = A.tile_start[tile + 1] - s;
  T.h0 = A.hoff[tile];
  T.n0 = A.noff[tile];
  T.H = (int)(A.hoff[tile + 1] - T.h0);
  T.L = (int)(A.noff[tile + 1] - T.n0);
  T.nt = T.n_own + T.H;
  T.ns = A.slot_stride;
  T.su = smem;
  T.sfx = reinterpret_cast<float *>(smem);                              // 3 * ns, over su
  T.swa = T.su + tile_slot_words(T.L, T.ns);
  T.swb = T.swa + T.nt;
  T.snode = reinterpret_cast<uint32_t *>(T.swb + T.nt);                 // L
  return T;
}

// position of the slot of vertex a of a tile tet; q3 is the tet record's
// fourth float4 (words 14, 15: four 16-bit positions)
__device__ __forceinline__ int slot_pos(const float4 &q3, int a) {
  const uint32_t w = __float_as_uint(a < 2 ? q3.z : q3.w);
  return (int)((a & 1) ? (w >> 16) : (w & 0xFFFF));
}

// nodal force (V_e grad N_a)^T sigma of vertex a into its slot
// (sigma in Voigt order xx yy zz yz zx xy)
__device__ __forceinline__ void store_slot_force(const TileView &T, const float4 &q3, int a, const float (&g)[3],
                                                 const float (&st)[6]) {
  const int p = slot_pos(q3, a);
  T.sfx[p] = g[0] * st[0] + g[1] * st[5] + g[2] * st[4];
  T.sfx[T.ns + p] = g[0] * st[5] + g[1] * st[1] + g[2] * st[3];
  T.sfx[2 * T.ns + p] = g[0] * st[4] + g[1] * st[3] + g[2] * st[2];
}

// strains of the tile's own and halo tets from the displacements in su
// (with kKeep the own tets' also into W)
template <bool kKeep = false>
__device__ __forceinline__ void tile_strains(const TileArgs &A, const TileRegs &R, const TileView &T, TileOwnW &W) {
#pragma unroll
  for (int r = 0; r < kTilePer; ++r) {
    const int j = threadIdx.x + r * kTileThreads;
    if (j < T.n_own) {
      TetGeo G;
      uint2 lc;
      rec_unpack(R.rr[r], G, lc);
      float4 w2[2];
      strain_to(T.su, lc, G, w2);
      T.swa[j] = w2[0];
      T.swb[j] = w2[1];
      if (kKeep) {
        W.w[r][0] = w2[0];
        W.w[r][1] = w2[1];
      }
    }
  }
  for (int h = threadIdx.x; h < T.H; h += kTileThreads) {
    TetGeo G;
    uint2 lc;
    load_rec(A.rec, A.rs, A.halo_tet[T.h0 + h], G, lc, nullptr);
    lc = A.halo_lconn[T.h0 + h];
    float4 w2[2];
    strain_to(T.su, lc, G, w2);
    T.swa[T.n_own + h] = w2[0];
    T.swb[T.n_own + h] = w2[1];
  }
}

// face-averaged stress of every own tet and its four nodal force slots
// (the neighbours' strains from shared memory, the own ones from Wn with
// kKeep, else from shared memory too; the kernels that keep them have the
// registers to spare); returns this thread's share of the energy sum w . t
template <int NT = kTileThreads, bool kKeep = false>
__device__ __forceinline__ float tile_forces(const TileRegsT<NT> &R, const TileView &T, const TileOwnWT<NT> &Wn,
                                             float lam, float mu) {
  float en = 0.f;  // this thread's tets
#pragma unroll
  for (int r = 0; r < TileRegsT<NT>::kPer; ++r) {
    const int j = threadIdx.x + r * NT;
    if (j >= T.n_own) continue;
    TetGeo G;
    uint2 lc;
    rec_unpack(R.rr[r], G, lc);
    const uint2 nb2 = make_uint2(__float_as_uint(R.rr[r][3].x), __float_as_uint(R.rr[r][3].y));
    const int nb[4] = {(int)(nb2.x & 0xFFFF), (int)(nb2.x >> 16), (int)(nb2.y & 0xFFFF), (int)(nb2.y >> 16)};
    const float4 w0 = kKeep ? Wn.w[r][0] : T.swa[j], w1 = kKeep ? Wn.w[r][1] : T.swb[j];
    const float W[6] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y};
    const float Ve = w1.z;
    // face weights kap_a = 1/(4 (V_e + V_nbr)), 1/(4 V_e) on exterior faces
    // (the hardware reciprocal: both tets of a face form the same sum and so
    // the same weight)
    float S[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float ks = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      if (nb[a] != kNoNbr) {
        const float4 n0v = T.swa[nb[a]], n1v = T.swb[nb[a]];
        const float k = __fdividef(0.25f, Ve + n1v.z);
        ks += k;
        S[0] = fmaf(k, n0v.x, S[0]);
        S[1] = fmaf(k, n0v.y, S[1]);
        S[2] = fmaf(k, n0v.z, S[2]);
        S[3] = fmaf(k, n0v.w, S[3]);
        S[4] = fmaf(k, n1v.x, S[4]);
        S[5] = fmaf(k, n1v.y, S[5]);
      } else {
        ks += __fdividef(0.25f, Ve);
      }
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) S[i] = fmaf(ks, W[i], S[i]);
    const float tr = S[0] + S[1] + S[2];
    const float st[6] = {lam * tr + 2.f * mu * S[0], lam * tr + 2.f * mu * S[1], lam * tr + 2.f * mu * S[2],
                         mu * S[3], mu * S[4], mu * S[5]};
    float el = 0.f;
#pragma unroll
    for (int i = 0; i < 6; ++i) el = fmaf(W[i], st[i], el);
    en += el;
#pragma unroll
    for (int a = 0; a < 4; ++a) store_slot_force(T, R.rr[r][3], a, G.g[a], st);
  }
  return en;
}

// the force at tile node i: its own slots summed in a fixed order (the
// tets' order in the tile) with compensation (the element forces at a node
// nearly cancel); false when the node has no slot in this tile.  Called by
// the 32 threads of a node group together, each step reads one bank row.
__device__ __forceinline__ bool tile_node_force(const TileView &T, int i, float &fx, float &fy, float &fz) {
  const uint32_t info = T.snode[i];
  const int b = (int)(info & 0xFFFF), n = (int)(info >> 16), lane = i & 31;
  fx = fy = fz = 0.f;
  if (n == 0) return false;
  float cx = 0.f, cy = 0.f, cz = 0.f;
  const float *px = T.sfx + b, *py = px + T.ns, *pz = py + T.ns;
  // compensated (Kahan) step: s += v
  auto add = [](float &s, float &c, float v) {
    const float yv = v - c;
    const float t = s + yv;
    c = __fsub_rn(__fsub_rn(t, s), yv);
    s = t;
  };
  int k = 0;
  // four slots' loads in flight at a time; the sums keep the order k = 0, 1, ...
  for (; k + 4 <= n; k += 4) {
    float vx[4], vy[4], vz[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int o = 32 * (k + q) + ((lane + k + q) & 31);
      vx[q] = px[o];
      vy[q] = py[o];
      vz[q] = pz[o];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      add(fx, cx, vx[q]);
      add(fy, cy, vy[q]);
      add(fz, cz, vz[q]);
    }
  }
  for (; k < n; ++k) {
    const int o = 32 * k + ((lane + k) & 31);
    add(fx, cx, px[o]);
    add(fy, cy, py[o]);
    add(fz, cz, pz[o]);
  }
  return true;
}

// y += K u over one tile (all threads of the block); returns this thread's
// share of u^T K u.  Starts and ends with a block barrier, so it can be
// called repeatedly on the same shared memory.
// kCoherentU: read u through L2 (ld.global.cg) instead of the read-only
// path; needed when u changes during the kernel (persistent solvers).
// energy_out: u^T K u of the tile added to *energy_out (one FP64 atomic per
// tile; the caller zeroes it before the launch).  A deterministic ticketed
// grid reduction here cost 26 us per apply on the 2M-tet beam (a memory
// fence and a returning atomic in each of the 4928 tiles).
template <class TU, class TY, bool kCoherentU = false>
__device__ __forceinline__ float tile_compute(const TileArgs &A, int tile, const TileRegs &R,
                                               const TU *__restrict__ u, TY *__restrict__ y, float lam, float mu,
                                               float4 *smem, double *energy_out = nullptr) {
  const TileView T = tile_view(A, tile, smem);
  // Strains are differences of nodal displacements, and K annihilates
  // constant fields (the shape-function gradients of a tet sum to zero), so
  // the tile subtracts the displacement of its first node (in the input's
  // precision) before the FP32 strain arithmetic: the rounding then acts on
  // the small tile-local differences instead of the full displacements,
  // which removes most of the cancellation error of the FP32 strains.
  // (With FP32 input the differences of nearby values are exact.)
  // (FP32 input needs no reference: the strains difference FP32 values
  // within each tet, see strain_to.)
  constexpr bool kRef = !std::is_same<TU, float>::value;
  TU ref[3] = {TU(0), TU(0), TU(0)};
  if (kRef) {
    const TU *rp = u + 3 * (int64_t)A.tile_nodes[T.n0];
#pragma unroll
    for (int c = 0; c < 3; ++c) ref[c] = kCoherentU ? __ldcg(rp + c) : __ldg(rp + c);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < T.L; i += kTileThreads) {
    const int64_t node = A.tile_nodes[T.n0 + i];
    const TU *up = u + 3 * node;
    if (kCoherentU)
      T.su[i] = make_float4((float)(__ldcg(up) - ref[0]), (float)(__ldcg(up + 1) - ref[1]),
                            (float)(__ldcg(up + 2) - ref[2]), 0.f);
    else
      T.su[i] = make_float4((float)(__ldg(up) - ref[0]), (float)(__ldg(up + 1) - ref[1]),
                            (float)(__ldg(up + 2) - ref[2]), 0.f);
    T.snode[i] = A.node_inc[T.n0 + i];
  }
  __syncthreads();
  TileOwnW Wn;
  tile_strains(A, R, T, Wn);
  __syncthreads();
  const float en = tile_forces(R, T, Wn, lam, mu);
  __shared__ float s_en[kTileThreads / 32];
  if (energy_out) {  // FP32 within the tile (512 terms), FP64 across tiles
    float e = en;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0) s_en[threadIdx.x >> 5] = e;
  }
  __syncthreads();
  if (energy_out && threadIdx.x == 0) {  // warp partials in a fixed order
    float e = 0.f;
#pragma unroll
    for (int w = 0; w < kTileThreads / 32; ++w) e += s_en[w];
    atomicAdd(energy_out, (double)e);
  }
  for (int i = threadIdx.x; i < T.L; i += kTileThreads) {
    float fx, fy, fz;
    if (!tile_node_force(T, i, fx, fy, fz)) continue;
    TY *yp = y + 3 * (int64_t)A.tile_nodes[T.n0 + i];
    atomicAdd(yp, (TY)fx);
    atomicAdd(yp + 1, (TY)fy);
    atomicAdd(yp + 2, (TY)fz);
  }
  __syncthreads();
  return en;
}

}  // namespace sfem
