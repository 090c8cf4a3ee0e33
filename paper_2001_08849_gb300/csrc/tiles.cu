// Tiled single-pass FP32 operator of FS-FEM-T4 (the hot kernel of the
// mixed-precision solve).
//
// Same arithmetic as the two-pass matrix-free operator (operator.cu):
//   w_e = V_e eps_e,  t_e = c sum_a kap_ea (w_e + w_nbr(a)),  y += (V_e B_e)^T t_e
// (Eq. 2-3 face averages on quarter-volume sub-tets, Eq. 9), but one CTA
// owns a tile of spatially close tets and keeps everything between the
// gather of u and the scatter of y in shared memory:
//   1. u at the tile's nodes -> smem (FP32);
//   2. strains of the tile's tets and of its halo (the neighbours across
//      the tile's outer faces, recomputed here) -> smem;
//   3. face-averaged stress per tile tet and its four nodal forces -> smem;
//   4. each tile node sums its slots in a fixed order and adds the sum to y
//      with one global atomic per component.  The slots are laid out at
//      setup so that this phase reads shared memory without bank conflicts
//      and without an index: nodes ordered by slot count and taken 32 at a
//      time, slot k of a node in bank row k of its group, in a bank rotated
//      by k; each tet writes its four slot forces to positions stored in
//      its record.
// Setup reorders tets by a coarse spatial binning of their centroids
// (counting sort on a Morton-free lexicographic bin grid), cuts bins into
// tiles of at most kTileMax tets, and builds per tile: the node list (in
// the order of the slot layout), 16-bit local connectivity, 16-bit local
// neighbour indices (into tile tets, then halo tets) and the halo list.  Per-tet data streamed by
// the kernel: one 64-byte record in four 16-byte planes (V_e-scaled
// gradients, V_e, local connectivity, local neighbours, slot positions);
// the face weights 1/(4 (V_e + V_nbr))
// are formed from the volumes staged in shared memory.

#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "reduce.cuh"
#include "sfem_internal.cuh"
#include "async.cuh"
#include "tile_apply.cuh"

namespace sfem {

constexpr int kTileTarget = 448;         // mean tets per spatial bin
constexpr int kHaloCand = 4 * kTileMax;  // neighbour candidates per tile

// ---------------------------------------------------------------------------
// setup kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ordered_bits(double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
static double from_ordered_bits(unsigned long long b) {
  b = (b & 0x8000000000000000ull) ? (b & 0x7fffffffffffffffull) : ~b;
  double d;
  memcpy(&d, &b, 8);
  return d;
}

// bounding box as ordered bit patterns: a grid-stride loop per thread, a
// warp reduction, then one atomic per warp and axis (launched with whole
// warps)
__global__ void k_bbox(const double *__restrict__ xyz, int64_t n_nodes, unsigned long long *mn,
                       unsigned long long *mx) {
  unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_nodes; i += (int64_t)gridDim.x * blockDim.x)
    for (int k = 0; k < 3; ++k) {
      const unsigned long long b = ordered_bits(xyz[3 * i + k]);
      lo[k] = min(lo[k], b);
      hi[k] = max(hi[k], b);
    }
  for (int k = 0; k < 3; ++k)
    for (int o = 16; o > 0; o >>= 1) {
      lo[k] = min(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
      hi[k] = max(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
    }
  if ((threadIdx.x & 31) == 0 && lo[0] != ~0ull)
    for (int k = 0; k < 3; ++k) {
      atomicMin(&mn[k], lo[k]);
      atomicMax(&mx[k], hi[k]);
    }
}

struct BinGrid {
  double lo[3], inv[3];
  int nb[3];
};

__global__ void k_bin_keys(const double *__restrict__ xyz, const int32_t *__restrict__ tets, int64_t n_tets,
                           BinGrid g, int32_t *__restrict__ key, int32_t *__restrict__ hist) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_tets) return;
  int4 t = reinterpret_cast<const int4 *>(tets)[e];
  int v[4] = {t.x, t.y, t.z, t.w};
  int b[3];
  for (int k = 0; k < 3; ++k) {
    double c = 0.25 * (xyz[3 * (int64_t)v[0] + k] + xyz[3 * (int64_t)v[1] + k] + xyz[3 * (int64_t)v[2] + k] +
                       xyz[3 * (int64_t)v[3] + k]);
    int q = (int)floor((c - g.lo[k]) * g.inv[k]);
    b[k] = min(max(q, 0), g.nb[k] - 1);
  }
  int kk = (b[0] * g.nb[1] + b[1]) * g.nb[2] + b[2];
  key[e] = kk;
  atomicAdd(&hist[kk], 1);
}

__global__ void k_bin_scatter(const int32_t *__restrict__ key, int64_t n_tets, unsigned long long *cursor,
                              int32_t *__restrict__ perm) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_tets) return;
  unsigned long long pos = atomicAdd(&cursor[key[e]], 1ull);
  perm[pos] = (int32_t)e;
}

__global__ void k_bin_tiles(const int64_t *__restrict__ bin_ptr, int64_t n_bins, int32_t *__restrict__ ntile) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_bins) return;
  int64_t c = bin_ptr[b + 1] - bin_ptr[b];
  ntile[b] = (int32_t)((c + kTileMax - 1) / kTileMax);
}

__global__ void k_tile_ranges(const int64_t *__restrict__ bin_ptr, const int64_t *__restrict__ tile_base,
                              int64_t n_bins, int64_t n_tiles, int32_t *__restrict__ tile_start) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n_bins) return;
  int64_t s = bin_ptr[b], e = bin_ptr[b + 1];
  int64_t t = tile_base[b];
  for (int64_t x = s; x < e; x += kTileMax, ++t) tile_start[t] = (int32_t)x;
  if (b == n_bins - 1) tile_start[n_tiles] = (int32_t)e;
}

// Per-tet record of the tiled operator (64 bytes, tile order), stored as four
// planes of float4 (words 4q..4q+3 of tet t at rec[q * n_tets + t], so one
// warp's load of a plane is 512 contiguous bytes):
//   [0..8]  V_e grad N_1..3 (node 1..3 by x, y, z) in FP32
//   [9]     V_e in FP32
//   [10,11] local connectivity (4 x 16 bit), written by k_tile_build
//   [12,13] local neighbours (4 x 16 bit, 0xFFFF exterior), k_tile_build
//   [14,15] positions (4 x 16 bit) of the tet's four nodal force slots in
//           the tile's slot arrays (see TileArgs), k_tile_build
__global__ void k_reorder(const int32_t *__restrict__ perm, int64_t n, const float *__restrict__ Gs32,
                          const double *__restrict__ vol, float4 *__restrict__ rec, int32_t *__restrict__ iperm) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t o = perm[i];
  iperm[o] = (int32_t)i;
  float g[9];
  for (int k = 0; k < 9; ++k) g[k] = Gs32[k * n + o];
  rec[i] = make_float4(g[0], g[1], g[2], g[3]);
  rec[n + i] = make_float4(g[4], g[5], g[6], g[7]);
  rec[2 * n + i] = make_float4(g[8], (float)vol[o], 0.f, 0.f);
  rec[3 * n + i] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// ascending bitonic sort of a[0..n) in shared memory; P a power of two >= n,
// a[n..P) is overwritten with padding
__device__ void block_bitonic_sort(int *a, int P, int n) {
  for (int i = n + threadIdx.x; i < P; i += blockDim.x) a[i] = INT_MAX;
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        int ixj = i ^ j;
        if (ixj > i) {
          int x = a[i], y = a[ixj];
          bool up = (i & k) == 0;
          if ((x > y) == up) {
            a[i] = y;
            a[ixj] = x;
          }
        }
      }
      __syncthreads();
    }
  }
}

// exclusive prefix sum of v over the block (blockDim.x a multiple of 32, at
// most 1024); *total receives the block's sum.  All threads must call it.
__device__ int block_exclusive_scan(int v, int *total) {
  __shared__ int wsum[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) wsum[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int w = lane < nw ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) wsum[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  *total = wsum[nw - 1];
  const int before = wid > 0 ? wsum[wid - 1] : 0;
  __syncthreads();
  return before + x - v;
}

// shared-memory hash sets of non-negative ints (INT_MAX marks a free slot;
// open addressing with linear probing; the table never fills: it holds at
// least twice as many slots as keys are inserted)
constexpr int kHaloHash = 4096;  // >= 2 * 4 * kTileMax, a multiple of the build block

__device__ __forceinline__ void hash_clear(int *t, int size) {
  for (int i = threadIdx.x; i < size; i += blockDim.x) t[i] = INT_MAX;
}
__device__ __forceinline__ void hash_insert(int *t, int size, int key) {
  // multiplicative hashing: the top log2(size) bits of key * (2^32 / golden ratio)
  unsigned h = ((unsigned)key * 2654435761u) >> (__clz(size) + 1);
  for (int probe = 0; probe < size; ++probe) {
    const int old = atomicCAS(&t[h], INT_MAX, key);
    if (old == INT_MAX || old == key) return;
    h = (h + 1) & (unsigned)(size - 1);
  }
}
// the keys of table t (size a multiple of blockDim.x, at most 16 slots per
// thread) packed into out[0..count), in slot order; out may alias t
__device__ int hash_compact(const int *t, int size, int *out) {
  const int chunk = size / (int)blockDim.x;
  const int b = threadIdx.x * chunk;
  int vals[16];
  int nv = 0;
  for (int i = 0; i < chunk; ++i) {
    const int v = t[b + i];
    if (v != INT_MAX) vals[nv++] = v;
  }
  int total;
  const int start = block_exclusive_scan(nv, &total);  // ends with a barrier: t is read
  for (int k = 0; k < nv; ++k) out[start + k] = vals[k];
  __syncthreads();
  return total;
}

// smallest power of two >= n (at least 32)
__device__ __forceinline__ int pow2_at_least(int n) {
  int p = 32;
  while (p < n) p <<= 1;
  return p;
}

__device__ __forceinline__ int bsearch_int(const int *a, int n, int key) {
  int lo = 0, hi = n - 1;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    int v = a[mid];
    if (v == key) return mid;
    if (v < key)
      lo = mid + 1;
    else
      hi = mid - 1;
  }
  return -1;
}

struct TileBuild {
  const int32_t *tile_start;
  const int32_t *perm, *iperm;
  const int32_t *tets;   // original numbering
  const int32_t *nbr;    // original numbering
  // pass 1 outputs
  int32_t *n_halo, *n_nodes;
  // pass 2 inputs/outputs
  const int64_t *hoff, *noff;
  int32_t *halo_tet;
  uint2 *halo_lconn;
  int32_t *tile_nodes;
  float4 *rec;   // per-tet records (tile order, 4 planes): lconn -> words 10,11; lnbr -> 12,13; slots -> 14,15
  int64_t rs;    // plane stride
  uint32_t *node_inc;  // per tile node: base of its slot group | own-slot count << 16
  int *max_slots;      // largest slot-array length over the tiles
  int key2_len;        // pass 2: power of two >= the largest node list (slot layout sort)
  unsigned long long *overflow;
};

// one CTA per tile; dynamic smem: halo candidates (kHaloCand padded) +
// node candidates (4*(kTileMax + kHaloCand) padded), and in pass 2 the slot
// layout tables (sized by the largest node list of pass 1: key2_len + 2 L +
// L / 32 + 4 ints)
constexpr int kHaloP = 2048;                        // >= kHaloCand, power of two
constexpr int kNodeP = 16384;                       // >= 4*(kTileMax + kHaloCand)
constexpr int kMaxTileNodes = 8000;                 // bounds the pass-2 tables (see below)
static_assert(kHaloP >= kHaloCand && kNodeP >= 4 * (kTileMax + kHaloCand), "tile build buffers too small");
// pass 2 tables at their largest: pow2(kMaxTileNodes) + 2 kMaxTileNodes + kMaxTileNodes / 32 + 4
static_assert(8192 >= kMaxTileNodes && 8192 + 2 * kMaxTileNodes + kMaxTileNodes / 32 + 4 <= 2 * kNodeP,
              "slot layout tables exceed the largest pass-2 shared memory");
constexpr int kBuildThreads = 1024;

__global__ void __launch_bounds__(kBuildThreads) k_tile_build(TileBuild B, int pass) {
  extern __shared__ int sm[];
  int *halo = sm;                 // kHaloP
  int *nodes = sm + kHaloP;       // kNodeP
  int *aux = nodes + kNodeP;      // slot layout tables (pass 2)
  const int tile = blockIdx.x;
  const int s = B.tile_start[tile], e = B.tile_start[tile + 1];
  const int n_own = e - s;
  // halo: the distinct neighbours outside [s, e), collected in a shared hash
  // set (in the node region, 4096 slots), compacted, then sorted
  hash_clear(nodes, kHaloHash);
  __syncthreads();
  for (int i = threadIdx.x; i < 4 * n_own; i += blockDim.x) {
    const int tnew = s + i / 4, a = i % 4;
    const int nb_old = B.nbr[4 * (int64_t)B.perm[tnew] + a];
    if (nb_old >= 0) {
      const int nb_new = B.iperm[nb_old];
      if (nb_new < s || nb_new >= e) hash_insert(nodes, kHaloHash, nb_new);
    }
  }
  __syncthreads();
  const int H = hash_compact(nodes, kHaloHash, halo);
  if (pass == 2) block_bitonic_sort(halo, pow2_at_least(H), H);
  // nodes of own and halo tets: hash set sized for the candidates, compacted
  // in place, sorted
  const int NT = min(kNodeP, max(kBuildThreads, pow2_at_least(8 * (n_own + H))));
  hash_clear(nodes, NT);
  __syncthreads();
  for (int i = threadIdx.x; i < 4 * (n_own + H); i += blockDim.x) {
    const int j = i / 4, a = i % 4;
    const int tnew = j < n_own ? s + j : halo[j - n_own];
    hash_insert(nodes, NT, B.tets[4 * (int64_t)B.perm[tnew] + a]);
  }
  __syncthreads();
  const int L = hash_compact(nodes, NT, nodes);
  if (pass == 2) block_bitonic_sort(nodes, pow2_at_least(L), L);
  if (pass == 1) {
    if (threadIdx.x == 0) {
      B.n_halo[tile] = H;
      B.n_nodes[tile] = L;
      if (L > kMaxTileNodes || n_own + H > 65535) atomicAdd(B.overflow, 1ull);
    }
    return;
  }
  const int64_t h0 = B.hoff[tile], n0 = B.noff[tile];
  // the tile's own slots sorted by (node, slot): the slots of each node in
  // the fixed order of the tets in the tile.  The keys live in the tail of
  // `nodes` past L (the halo list is still needed below).
  int *keys = nodes + ((L + 31) & ~31);
  const int KP = pow2_at_least(4 * n_own);  // >= 4 n_own slots, power of two
  for (int i = threadIdx.x; i < KP; i += blockDim.x) {
    int v = INT_MAX;
    if (i < 4 * n_own) {
      const int64_t to = B.perm[s + i / 4];
      const int l = bsearch_int(nodes, L, B.tets[4 * to + (i % 4)]);
      v = (l << 11) | i;
    }
    keys[i] = v;
  }
  __syncthreads();
  block_bitonic_sort(keys, KP, KP);
  // slot layout (see TileArgs): nodes ordered by own-slot count, largest
  // first (ties by node id), in groups of 32; group g starts at gbase[g] and
  // holds 32 x (count of its first node) positions
  int *key2 = aux;                  // pow2(L): (2047 - count) << 16 | ascending index
  int *start = aux + B.key2_len;    // L + 1: first key of each node (ascending index)
  int *jds = start + L + 1;         // L: position of each node in the count order
  int *gbase = jds + L;             // groups + 1
  const int ngroups = (L + 31) / 32;
  for (int l = threadIdx.x; l <= L; l += blockDim.x) {
    int lo = 0, hi = 4 * n_own;
    const int key = l << 11;        // number of keys below (l << 11)
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (keys[mid] < key)
        lo = mid + 1;
      else
        hi = mid;
    }
    start[l] = lo;
  }
  __syncthreads();
  for (int l = threadIdx.x; l < L; l += blockDim.x) key2[l] = ((2047 - (start[l + 1] - start[l])) << 16) | l;
  block_bitonic_sort(key2, pow2_at_least(L), L);
  for (int q = threadIdx.x; q < L; q += blockDim.x) jds[key2[q] & 0xFFFF] = q;
  if (threadIdx.x == 0) {
    int b = 0;
    for (int g = 0; g < ngroups; ++g) {
      gbase[g] = b;
      b += 32 * (2047 - (key2[32 * g] >> 16));
    }
    gbase[ngroups] = b;
    atomicMax(B.max_slots, b);
  }
  __syncthreads();
  for (int q = threadIdx.x; q < L; q += blockDim.x) {
    const int l = key2[q] & 0xFFFF, cnt = 2047 - (key2[q] >> 16);
    B.tile_nodes[n0 + q] = nodes[l];
    B.node_inc[n0 + q] = (uint32_t)gbase[q >> 5] | ((uint32_t)cnt << 16);
  }
  uint16_t *rpos = reinterpret_cast<uint16_t *>(B.rec + 3 * B.rs + s);
  for (int p = threadIdx.x; p < 4 * n_own; p += blockDim.x) {
    // slot i = 4j + a (tet j, vertex a) is the k-th slot of its node; its
    // position goes to record (s + j), 16-bit word 28 + a (words 14, 15)
    const int key = keys[p], l = key >> 11, i = key & 2047;
    const int k = p - start[l], q = jds[l];
    rpos[(i / 4) * 8 + 4 + (i % 4)] = (uint16_t)(gbase[q >> 5] + 32 * k + (((q & 31) + k) & 31));
  }
  for (int j = threadIdx.x; j < n_own + H; j += blockDim.x) {
    const int tnew = j < n_own ? s + j : halo[j - n_own];
    const int64_t to = B.perm[tnew];
    unsigned int l[4];
    for (int a = 0; a < 4; ++a) l[a] = (unsigned int)jds[bsearch_int(nodes, L, B.tets[4 * to + a])];
    const uint2 lc = make_uint2(l[0] | (l[1] << 16), l[2] | (l[3] << 16));
    if (j < n_own) {
      unsigned int *rw2 = reinterpret_cast<unsigned int *>(B.rec + 2 * B.rs + tnew);  // words 8-11
      unsigned int *rw3 = reinterpret_cast<unsigned int *>(B.rec + 3 * B.rs + tnew);  // words 12-15
      rw2[2] = lc.x;
      rw2[3] = lc.y;
      unsigned int nb[4];
      for (int a = 0; a < 4; ++a) {
        const int nb_old = B.nbr[4 * to + a];
        if (nb_old < 0) {
          nb[a] = kNoNbr;
        } else {
          const int nb_new = B.iperm[nb_old];
          nb[a] = (nb_new >= s && nb_new < e) ? (unsigned int)(nb_new - s)
                                                : (unsigned int)(n_own + bsearch_int(halo, H, nb_new));
        }
      }
      rw3[0] = nb[0] | (nb[1] << 16);
      rw3[1] = nb[2] | (nb[3] << 16);
    } else {
      B.halo_tet[h0 + (j - n_own)] = tnew;
      B.halo_lconn[h0 + (j - n_own)] = lc;
    }
  }
}

__global__ void k_max_i32(const int32_t *__restrict__ a, const int32_t *__restrict__ b, int64_t n, int *out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  atomicMax(&out[0], a[i]);
  atomicMax(&out[1], b[i]);
}

// ---------------------------------------------------------------------------
// the fused operator
// ---------------------------------------------------------------------------
template <class TU, class TY>
__global__ void __launch_bounds__(kTileThreads, 4)
    k_mf32_tiled(TileArgs A, const TU *__restrict__ u, TY *__restrict__ y, float lam, float mu, double *energy_out,
                 const int *done) {
  if (done && *done) return;
  extern __shared__ float4 smem[];
  TileRegs R;
  tile_load(A, blockIdx.x, R);
  tile_compute<TU, TY>(A, blockIdx.x, R, u, y, lam, mu, smem, energy_out);
}

// ---------------------------------------------------------------------------
// the fused operator, persistent form with prefetch
// ---------------------------------------------------------------------------
// Each CTA loops over tiles blockIdx.x, blockIdx.x + gridDim.x, ...  While it
// computes tile n, the inputs of the next tiles are already on their way
// into shared memory, so the tile's phases no longer wait on global loads:
//   * the own-tet records of tile n+1 (four contiguous planes) by bulk
//     copies, issued once the records of tile n are in registers;
//   * the index arrays of tile n+2 (node list, node slot info, halo ids,
//     halo connectivity; contiguous per tile) by bulk copies into one of two
//     index buffers, issued once tile n has finished with that buffer;
//   * the displacements of tile n+1 at its nodes, gathered by cp.async as
//     soon as its index buffer has landed (before tile n's strains).
// The halo tets' records are still read from global memory in the strain
// phase (their ids come from shared memory).  The index arrays are
// allocated with padding so that the copied ranges can start and end on
// 16-byte boundaries; each buffer records where the tile's entries begin.
struct PfLayout {
  int n_tiles;
  int capN, capH, capH2;  // entries per index-buffer array (nodes/info, halo ids, halo connectivity)
  int ibytes;             // bytes of one index buffer
  int capR;               // halo records per halo buffer plane
  int off_i, off_h, off_u, off_w;  // byte offsets: index buffers, halo records, displacements, work area
};

// index buffer: 8 ints of tile data, then node ids, node slot info, halo
// ids, halo connectivity
struct PfTile {
  int s, n_own, n0, L, h0, H, dn, dh;  // dn, dh: offsets of the tile's first node / halo entry
};

// tile ranges of one tile, read by the issuing thread a whole tile ahead
struct PfMeta {
  int s, e;
  int64_t n0, n1, h0, h1;
};

__device__ __forceinline__ PfMeta pf_meta(const TileArgs &A, int tile) {
  PfMeta m;
  m.s = A.tile_start[tile];
  m.e = A.tile_start[tile + 1];
  m.n0 = A.noff[tile];
  m.n1 = A.noff[tile + 1];
  m.h0 = A.hoff[tile];
  m.h1 = A.hoff[tile + 1];
  return m;
}

__device__ __forceinline__ int *pf_nodes(unsigned char *ib) { return reinterpret_cast<int *>(ib + 32); }
__device__ __forceinline__ uint32_t *pf_info(unsigned char *ib, const PfLayout &P) {
  return reinterpret_cast<uint32_t *>(ib + 32 + 4 * P.capN);
}
__device__ __forceinline__ int *pf_htet(unsigned char *ib, const PfLayout &P) {
  return reinterpret_cast<int *>(ib + 32 + 8 * P.capN);
}
__device__ __forceinline__ uint2 *pf_hlc(unsigned char *ib, const PfLayout &P) {
  return reinterpret_cast<uint2 *>(ib + 32 + 8 * P.capN + 4 * P.capH);
}

// Issuing a bulk copy stalls the issuing thread for a while (on the order
// of a hundred cycles each), so the copies of one tile are issued by lane 0
// of several warps, one copy each, instead of by one thread: the stalls
// overlap instead of adding up on one warp that the block then waits for.
// The barrier's expected byte count may be set before or after the copies
// complete (the transaction count of an mbarrier may go transiently
// negative; the phase completes when the arrival and all bytes are in).

// index arrays of a tile, part `part` of 4: 0 writes the buffer header,
// announces the bytes of all four copies and copies the node ids; 1 the node
// slot info; 2 the halo ids; 3 the halo connectivity
__device__ void pf_issue_index_part(const TileArgs &A, const PfLayout &P, const PfMeta &t, unsigned char *ib,
                                    uint64_t *bar, int part) {
  const int64_t na = t.n0 & ~int64_t(3), ne = (t.n1 + 3) & ~int64_t(3);
  const int64_t ha = t.h0 & ~int64_t(3), he = (t.h1 + 3) & ~int64_t(3);
  const int64_t la = t.h0 & ~int64_t(1), le = (t.h1 + 1) & ~int64_t(1);
  const uint32_t bn = (uint32_t)(ne - na) * 4u;
  const uint32_t bh = t.h1 > t.h0 ? (uint32_t)(he - ha) * 4u : 0u;
  const uint32_t bl = t.h1 > t.h0 ? (uint32_t)(le - la) * 8u : 0u;
  if (part == 0) {
    PfTile *m = reinterpret_cast<PfTile *>(ib);
    m->s = t.s;
    m->n_own = t.e - t.s;
    m->n0 = (int)t.n0;
    m->L = (int)(t.n1 - t.n0);
    m->h0 = (int)t.h0;
    m->H = (int)(t.h1 - t.h0);
    m->dn = (int)(t.n0 - na);
    m->dh = (int)(t.h0 - ha);
    mbar_arrive_expect_tx(bar, 2u * bn + bh + bl);
    bulk_load(pf_nodes(ib), A.tile_nodes + na, bn, bar);
  } else if (part == 1) {
    bulk_load(pf_info(ib, P), A.node_inc + na, bn, bar);
  } else if (part == 2) {
    if (bh) bulk_load(pf_htet(ib, P), A.halo_tet + ha, bh, bar);
  } else {
    if (bl) bulk_load(pf_hlc(ib, P), A.halo_lconn + la, bl, bar);
  }
}

// all four parts by one thread (start-up)
__device__ void pf_issue_index(const TileArgs &A, const PfLayout &P, const PfMeta &t, unsigned char *ib,
                               uint64_t *bar) {
  for (int k = 0; k < 4; ++k) pf_issue_index_part(A, P, t, ib, bar, k);
}

// record plane q of tets [s, s + n); plane 0 also announces all four planes.
// (An evict-first L2 policy on these copies cost 6 us per apply on the 2M-tet
// beam: neighbouring tiles read the same records as halo records from L2.)
__device__ __forceinline__ void pf_issue_record_plane(const TileArgs &A, int s, int n, float4 *rb, uint64_t *bar,
                                                      int q) {
  const uint32_t b = (uint32_t)n * 16u;
  if (q == 0) mbar_arrive_expect_tx(bar, 4u * b);
  bulk_load(rb + q * kTileMax, A.rec + q * A.rs + s, b, bar);
}

__device__ void pf_issue_records(const TileArgs &A, int s, int n, float4 *rb, uint64_t *bar) {
  for (int q = 0; q < 4; ++q) pf_issue_record_plane(A, s, n, rb, bar, q);
}

// all threads: gather u at the tile's nodes (its index buffer has landed)
template <class TU, int NT>
__device__ __forceinline__ void pf_issue_u(unsigned char *ib, const TU *u, TU *ub) {
  const PfTile *m = reinterpret_cast<const PfTile *>(ib);
  const int *nodes = pf_nodes(ib) + m->dn;
  for (int i = threadIdx.x; i < m->L; i += NT) {
    const TU *up = u + 3 * (int64_t)nodes[i];
#pragma unroll
    for (int c = 0; c < 3; ++c) cp_async<sizeof(TU)>(ub + 3 * i + c, up + c);
  }
}

// all threads: gather the first three record planes of the tile's halo tets
// (geometry and volume; their local connectivity is in the index buffer)
template <int NT>
__device__ __forceinline__ void pf_issue_halo(const TileArgs &A, const PfLayout &P, unsigned char *ib, float4 *hb) {
  const PfTile *m = reinterpret_cast<const PfTile *>(ib);
  const int *htet = pf_htet(ib, P) + m->dh;
  for (int h = threadIdx.x; h < m->H; h += NT) {
    const int64_t t = htet[h];
#pragma unroll
    for (int q = 0; q < 3; ++q) cp_async<16>(hb + q * P.capR + h, A.rec + q * A.rs + t);
  }
}

// after a wait that gave up: let this CTA's copies in flight land (bounded)
__device__ void pf_drain() {
  cp_async_wait_all();
  const uint64_t t0 = global_ns();
  while (global_ns() - t0 < 1000000ull) {
  }
}

// NT threads per CTA (256 in use), two CTAs per SM.  Per tile four block
// barriers: inputs in place (records in registers, displacements in shared
// memory), strains formed (and the next tile's index arrays landed), forces
// in their slots, nodal sums done.
template <class TU, class TY, int NT>
__global__ void __launch_bounds__(NT, 2)
    k_mf32_tiled_pf(TileArgs A, PfLayout P, const TU *__restrict__ u, TY *__restrict__ y, float lam, float mu,
                    double *energy_out, const int *done, int *err) {
  using Regs = TileRegsT<NT>;
  if (done && *done) return;
  extern __shared__ __align__(16) unsigned char sm_pf[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm_pf);  // [0] records, [1], [2] index buffers
  float4 *rb = reinterpret_cast<float4 *>(sm_pf + 32);  // 4 record planes of kTileMax
  unsigned char *ib0 = sm_pf + P.off_i;
  float4 *hb = reinterpret_cast<float4 *>(sm_pf + P.off_h);  // 3 halo record planes of capR
  TU *ub = reinterpret_cast<TU *>(sm_pf + P.off_u);
  float4 *W = reinterpret_cast<float4 *>(sm_pf + P.off_w);
  __shared__ float s_en[NT / 32];
  constexpr bool kRef = !std::is_same<TU, float>::value;  // see tile_compute
  int tile = blockIdx.x;
  if (tile >= P.n_tiles) return;
  int next = tile + gridDim.x;
  PfMeta meta2{};  // index-issuing threads: the tile after next
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < 3; ++k) mbar_init(&bar[k], 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const PfMeta m0 = pf_meta(A, tile);
    pf_issue_index(A, P, m0, ib0, &bar[1]);
    pf_issue_records(A, m0.s, m0.e - m0.s, rb, &bar[0]);
    if (next < P.n_tiles) pf_issue_index(A, P, pf_meta(A, next), ib0 + P.ibytes, &bar[2]);
  }
  bool failed = __syncthreads_or(!mbar_wait(&bar[1], 0));
  if (!failed) {
    pf_issue_u<TU, NT>(ib0, u, ub);
    pf_issue_halo<NT>(A, P, ib0, hb);
    cp_async_commit();
  }
  for (int n = 0; !failed && tile < P.n_tiles; ++n) {
    const int b = n & 1;
    unsigned char *ib = ib0 + b * P.ibytes;
    unsigned char *ibn = ib0 + (b ^ 1) * P.ibytes;
    const int next2 = next + gridDim.x;
    // lane 0 of warps 4..7 issue the index copies of the tile after next at
    // the end of this tile; their tile ranges are read now
    const int ipart = (threadIdx.x & 31) == 0 ? (int)(threadIdx.x >> 5) - 4 : -1;
    if (ipart >= 0 && ipart < 4 && next2 < P.n_tiles) meta2 = pf_meta(A, next2);
    const PfTile m = *reinterpret_cast<const PfTile *>(ib);
    TileView T;
    T.n_own = m.n_own;
    T.H = m.H;
    T.L = m.L;
    T.nt = m.n_own + m.H;
    T.ns = A.slot_stride;
    T.h0 = m.h0;
    T.n0 = 0;
    T.su = W;
    T.sfx = reinterpret_cast<float *>(W);
    T.swa = W + tile_slot_words(T.L, T.ns);
    T.swb = T.swa + T.nt;
    T.snode = pf_info(ib, P) + m.dn;
    // 1. inputs: records -> registers, displacements (and halo records) landed
    const bool rec_ok = mbar_wait(&bar[0], n & 1);
    Regs R;
#pragma unroll
    for (int r = 0; r < Regs::kPer; ++r) {
      const int j = threadIdx.x + r * NT;
      if (j < m.n_own) {
#pragma unroll
        for (int q = 0; q < 4; ++q) R.rr[r][q] = rb[q * kTileMax + j];
      }
    }
    // (each thread reads back the displacements and halo records it gathered
    // itself; the reference node of FP64 input was gathered by thread 0)
    cp_async_wait_all();
    if (kRef) __syncthreads();
    {
      const TU r0 = kRef ? ub[0] : TU(0), r1 = kRef ? ub[1] : TU(0), r2 = kRef ? ub[2] : TU(0);
      for (int i = threadIdx.x; i < T.L; i += NT)
        T.su[i] = make_float4((float)(ub[3 * i] - r0), (float)(ub[3 * i + 1] - r1), (float)(ub[3 * i + 2] - r2),
                              0.f);
    }
    if (__syncthreads_or(!rec_ok)) {
      failed = true;
      break;
    }
    if ((threadIdx.x & 31) == 0 && threadIdx.x < 128 && next < P.n_tiles) {  // the record buffer is free
      const PfTile *mn = reinterpret_cast<const PfTile *>(ibn);  // header written a tile ago
      fence_proxy_async_smem();
      pf_issue_record_plane(A, mn->s, mn->n_own, rb, &bar[0], threadIdx.x >> 5);
    }
    // 2. strains of the own tets (records in registers; the strains kept in
    // registers for the force phase) and the halo tets
    TileOwnWT<NT> Wn;
#pragma unroll
    for (int r = 0; r < Regs::kPer; ++r) {
      const int j = threadIdx.x + r * NT;
      if (j < T.n_own) {
        TetGeo G;
        uint2 lc;
        rec_unpack(R.rr[r], G, lc);
        strain_to(T.su, lc, G, Wn.w[r]);
        T.swa[j] = Wn.w[r][0];
        T.swb[j] = Wn.w[r][1];
      }
    }
    {
      const uint2 *hlc = pf_hlc(ib, P) + (m.h0 & 1);
      for (int h = threadIdx.x; h < T.H; h += NT) {
        const float4 q[4] = {hb[h], hb[P.capR + h], hb[2 * P.capR + h], make_float4(0.f, 0.f, 0.f, 0.f)};
        TetGeo G;
        uint2 lc;
        rec_unpack(q, G, lc);
        lc = hlc[h];
        float4 w2[2];
        strain_to(T.su, lc, G, w2);
        T.swa[T.n_own + h] = w2[0];
        T.swb[T.n_own + h] = w2[1];
      }
    }
    // the next tile's index arrays must have landed before its gathers
    const bool idx_ok = next < P.n_tiles ? mbar_wait(&bar[1 + (b ^ 1)], ((n + 1) >> 1) & 1) : true;
    if (__syncthreads_or(!idx_ok)) {
      failed = true;
      break;
    }
    if (next < P.n_tiles) {  // displacement and halo buffers are free
      pf_issue_u<TU, NT>(ibn, u, ub);
      pf_issue_halo<NT>(A, P, ibn, hb);
      cp_async_commit();
    }
    // 3. face-averaged stresses and the slot forces
    const float en = tile_forces<NT, true>(R, T, Wn, lam, mu);
    if (energy_out) {  // FP32 within the tile, FP64 across tiles
      float e = en;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
      if ((threadIdx.x & 31) == 0) s_en[threadIdx.x >> 5] = e;
    }
    __syncthreads();
    if (energy_out && threadIdx.x == 0) {
      float e = 0.f;
#pragma unroll
      for (int w = 0; w < NT / 32; ++w) e += s_en[w];
      atomicAdd(energy_out, (double)e);
    }
    // 4. nodal sums into y
    {
      const int *nodes = pf_nodes(ib) + m.dn;
      for (int i = threadIdx.x; i < T.L; i += NT) {
        float fx, fy, fz;
        if (!tile_node_force(T, i, fx, fy, fz)) continue;
        TY *yp = y + 3 * (int64_t)nodes[i];
        atomicAdd(yp, (TY)fx);
        atomicAdd(yp + 1, (TY)fy);
        atomicAdd(yp + 2, (TY)fz);
      }
    }
    __syncthreads();
    // index buffer b is free: the indices of the tile after next
    if (ipart >= 0 && ipart < 4 && next2 < P.n_tiles) {
      fence_proxy_async_smem();
      pf_issue_index_part(A, P, meta2, ib, &bar[1 + b], ipart);
    }
    tile = next;
    next = next2;
  }
  if (failed) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    pf_drain();
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int align_up(int x, int a) { return (x + a - 1) / a * a; }

// shared-memory layout and grid of the prefetching operator; it is used when
// two CTAs fit on an SM, else the one-CTA-per-tile kernel stays in use
static void setup_prefetch(Ctx &c) {
  TileData &t = c.tl;
  t.pf_capN = align_up(t.max_nodes + 6, 4);
  t.pf_capH = align_up(t.max_halo + 6, 4);
  t.pf_capH2 = align_up(t.max_halo + 2, 2);
  t.pf_capR = std::max(t.max_halo, 1);
  t.pf_ibytes = align_up(32 + 8 * t.pf_capN + 4 * t.pf_capH + 8 * t.pf_capH2, 16);
  t.pf_off_i = 32 + 4 * kTileMax * (int)sizeof(float4);
  t.pf_off_h = t.pf_off_i + 2 * t.pf_ibytes;
  t.pf_off_u = t.pf_off_h + 3 * t.pf_capR * (int)sizeof(float4);
  if (!t.err) {
    t.err = c.mem.get<int>(1);
    SFEM_CUDA(cudaMemsetAsync(t.err, 0, sizeof(int), c.stream));
  }
  int nsm = 0, dev = 0;
  SFEM_CUDA(cudaGetDevice(&dev));
  SFEM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  static size_t smem_set[2] = {0, 0};
  for (int v = 0; v < 2; ++v) {  // FP32 / FP64 input
    const int es = v ? 8 : 4;
    t.pf_off_w[v] = align_up(t.pf_off_u + 3 * t.max_nodes * es, 16);
    t.pf_smem[v] = (size_t)t.pf_off_w[v] + (size_t)tile_slot_words(t.max_nodes, t.slot_stride) * sizeof(float4) +
                   (size_t)(kTileMax + t.max_halo) * 2 * sizeof(float4);
    t.pf_grid[v] = 0;
    t.pf_threads[v] = 0;
    if (t.pf_smem[v] > 227 * 1024) continue;
    const void *k256 = v ? (const void *)k_mf32_tiled_pf<double, double, 256> : (const void *)k_mf32_tiled_pf<float, float, 256>;
    if (t.pf_smem[v] > smem_set[v]) {
      SFEM_CUDA(cudaFuncSetAttribute(k256, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t.pf_smem[v]));
      smem_set[v] = t.pf_smem[v];
    }
    // two CTAs of 256 threads per SM (512-thread CTAs measured 3.5 us slower
    // per apply on the 2M-tet beam)
    int per_sm = 0;
    SFEM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k256, 256, t.pf_smem[v]));
    if (per_sm < 2) continue;
    t.pf_threads[v] = 256;
    t.pf_grid[v] = (int)std::min<int64_t>(t.n_tiles, (int64_t)per_sm * nsm);
  }
}

// a wait of the prefetching operator gave up (reported once, then cleared)
void check_tile_error(Ctx &c) {
  if (!c.tl.err) return;
  int h = 0;
  SFEM_CUDA(cudaMemcpyAsync(&h, c.tl.err, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  SFEM_CUDA(cudaStreamSynchronize(c.stream));
  if (h) {
    SFEM_CUDA(cudaMemsetAsync(c.tl.err, 0, sizeof(int), c.stream));
    throw Error{SFEM_ECUDA, "the tiled operator's asynchronous copies did not complete in time"};
  }
}

void build_tiles(Ctx &c) {
  const int64_t n = c.n_tets;
  // bounding box and bin grid (mean bin holds about kTileTarget tets)
  unsigned long long *bb = c.mem.get<unsigned long long>(6);
  unsigned long long init[6];
  for (int k = 0; k < 3; ++k) {
    init[k] = ~0ull;
    init[3 + k] = 0ull;
  }
  SFEM_CUDA(cudaMemcpyAsync(bb, init, sizeof init, cudaMemcpyHostToDevice, c.stream));
  k_bbox<<<(unsigned)std::min<int64_t>(grid_for(c.n_nodes, 256), 4 * 152), 256, 0, c.stream>>>(c.xyz, c.n_nodes, bb, bb + 3);
  SFEM_CHECK_LAUNCH();
  unsigned long long hb[6];
  SFEM_CUDA(cudaMemcpyAsync(hb, bb, sizeof hb, cudaMemcpyDeviceToHost, c.stream));
  SFEM_CUDA(cudaStreamSynchronize(c.stream));
  c.mem.drop(bb);
  double lo[3], ext[3], boxvol = 1.0;
  for (int k = 0; k < 3; ++k) {
    lo[k] = from_ordered_bits(hb[k]);
    c.bbox_lo[k] = lo[k];
    c.bbox_hi[k] = from_ordered_bits(hb[3 + k]);
    ext[k] = std::max(c.bbox_hi[k] - lo[k], 1e-300);
    boxvol *= ext[k];
  }
  const double edge = std::cbrt(boxvol / (double)n * kTileTarget);
  BinGrid g;
  int64_t nbins = 1;
  for (int k = 0; k < 3; ++k) {
    g.nb[k] = (int)std::min<double>(std::max(1.0, std::ceil(ext[k] / edge)), 1 << 20);
    g.lo[k] = lo[k];
    g.inv[k] = g.nb[k] / ext[k];
    nbins *= g.nb[k];
  }
  SFEM_REQUIRE(nbins < (int64_t(1) << 30), SFEM_EINVAL, "tile grid too large");
  int32_t *key = c.mem.get<int32_t>(n);
  int32_t *hist = c.mem.get<int32_t>(nbins);
  SFEM_CUDA(cudaMemsetAsync(hist, 0, nbins * sizeof(int32_t), c.stream));
  k_bin_keys<<<grid_for(n, 256), 256, 0, c.stream>>>(c.xyz, c.tets, n, g, key, hist);
  SFEM_CHECK_LAUNCH();
  int64_t *bin_ptr = c.mem.get<int64_t>(nbins + 1);
  scan_counts(c, hist, nbins, bin_ptr);
  unsigned long long *cursor = c.mem.get<unsigned long long>(nbins);
  SFEM_CUDA(cudaMemcpyAsync(cursor, bin_ptr, nbins * sizeof(int64_t), cudaMemcpyDeviceToDevice, c.stream));
  c.tl.perm = c.mem.get<int32_t>(n);
  k_bin_scatter<<<grid_for(n, 256), 256, 0, c.stream>>>(key, n, cursor, c.tl.perm);
  SFEM_CHECK_LAUNCH();
  k_bin_tiles<<<grid_for(nbins, 256), 256, 0, c.stream>>>(bin_ptr, nbins, hist);  // hist reused: tiles per bin
  SFEM_CHECK_LAUNCH();
  int64_t *tile_base = c.mem.get<int64_t>(nbins + 1);
  c.tl.n_tiles = scan_counts(c, hist, nbins, tile_base);
  c.tl.tile_start = c.mem.get<int32_t>(c.tl.n_tiles + 1);
  k_tile_ranges<<<grid_for(nbins, 256), 256, 0, c.stream>>>(bin_ptr, tile_base, nbins, c.tl.n_tiles,
                                                            c.tl.tile_start);
  SFEM_CHECK_LAUNCH();
  c.mem.drop(key);
  c.mem.drop(cursor);
  c.mem.drop(bin_ptr);
  c.mem.drop(tile_base);

  // reordered operator data
  c.tl.iperm = c.mem.get<int32_t>(n);
  c.tl.rec = c.mem.get<float4>(4 * n);
  k_reorder<<<grid_for(n, 256), 256, 0, c.stream>>>(c.tl.perm, n, c.Gs32, c.vol, c.tl.rec, c.tl.iperm);
  SFEM_CHECK_LAUNCH();

  // per-tile tables, pass 1 (sizes)
  const int64_t nt = c.tl.n_tiles;
  int32_t *nh = hist;  // reuse (>= nt? no: allocate)
  nh = c.mem.get<int32_t>(nt);
  int32_t *nn = c.mem.get<int32_t>(nt);
  unsigned long long *ovf = c.mem.get<unsigned long long>(1);
  SFEM_CUDA(cudaMemsetAsync(ovf, 0, 8, c.stream));
  TileBuild B{};
  B.tile_start = c.tl.tile_start;
  B.perm = c.tl.perm;
  B.iperm = c.tl.iperm;
  B.tets = c.tets;
  B.nbr = c.nbr;
  B.n_halo = nh;
  B.n_nodes = nn;
  B.overflow = ovf;
  const size_t build_smem = (kHaloP + kNodeP) * sizeof(int);  // pass 1
  SFEM_CUDA(cudaFuncSetAttribute(k_tile_build, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)((kHaloP + 3 * kNodeP) * sizeof(int))));  // the largest pass 2 can ask
  k_tile_build<<<(unsigned)nt, kBuildThreads, build_smem, c.stream>>>(B, 1);
  SFEM_CHECK_LAUNCH();
  c.tl.hoff = c.mem.get<int64_t>(nt + 1);
  c.tl.noff = c.mem.get<int64_t>(nt + 1);
  const int64_t total_h = scan_counts(c, nh, nt, c.tl.hoff);
  const int64_t total_n = scan_counts(c, nn, nt, c.tl.noff);
  int *mx = c.mem.get<int>(3);  // largest halo, node list, slot array (pass 2)
  SFEM_CUDA(cudaMemsetAsync(mx, 0, 3 * sizeof(int), c.stream));
  k_max_i32<<<grid_for(nt, 256), 256, 0, c.stream>>>(nh, nn, nt, mx);
  SFEM_CHECK_LAUNCH();
  int hm[2];
  unsigned long long hovf = 0;
  SFEM_CUDA(cudaMemcpyAsync(hm, mx, sizeof hm, cudaMemcpyDeviceToHost, c.stream));
  SFEM_CUDA(cudaMemcpyAsync(&hovf, ovf, 8, cudaMemcpyDeviceToHost, c.stream));
  SFEM_CUDA(cudaStreamSynchronize(c.stream));
  SFEM_REQUIRE(hovf == 0, SFEM_EMESH, "tile tables exceed their local index ranges");
  c.tl.max_halo = hm[0];
  c.tl.max_nodes = hm[1];
  // (padded: the prefetching operator copies 16-byte aligned ranges)
  c.tl.halo_tet = c.mem.get<int32_t>(std::max<int64_t>(total_h, 1) + 4);
  c.tl.halo_lconn = c.mem.get<uint2>(std::max<int64_t>(total_h, 1) + 2);
  c.tl.tile_nodes = c.mem.get<int32_t>(total_n + 4);
  c.tl.node_inc = c.mem.get<uint32_t>(total_n + 4);
  B.hoff = c.tl.hoff;
  B.noff = c.tl.noff;
  B.halo_tet = c.tl.halo_tet;
  B.halo_lconn = c.tl.halo_lconn;
  B.tile_nodes = c.tl.tile_nodes;
  B.node_inc = c.tl.node_inc;
  B.rec = c.tl.rec;
  B.rs = n;
  B.max_slots = mx + 2;
  B.key2_len = 32;
  while (B.key2_len < c.tl.max_nodes) B.key2_len <<= 1;
  const size_t build_smem2 =
      (size_t)(kHaloP + kNodeP + B.key2_len + 2 * c.tl.max_nodes + c.tl.max_nodes / 32 + 4) * sizeof(int);
  k_tile_build<<<(unsigned)nt, kBuildThreads, build_smem2, c.stream>>>(B, 2);
  SFEM_CHECK_LAUNCH();
  int hslots = 0;
  SFEM_CUDA(cudaMemcpyAsync(&hslots, mx + 2, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  SFEM_CUDA(cudaStreamSynchronize(c.stream));
  c.tl.slot_stride = std::max(hslots, 32);  // a multiple of 32 (groups of 32 positions)
  c.mem.drop(nh);
  c.mem.drop(nn);
  c.mem.drop(ovf);
  c.mem.drop(mx);
  c.mem.drop(hist);
  c.tl.smem = (size_t)tile_slot_words(c.tl.max_nodes, c.tl.slot_stride) * sizeof(float4) +
              (size_t)(kTileMax + c.tl.max_halo) * 2 * sizeof(float4) + (size_t)c.tl.max_nodes * sizeof(uint32_t);
  c.tl.smem = (c.tl.smem + 15) & ~size_t(15);
  SFEM_REQUIRE(c.tl.smem <= 220 * 1024, SFEM_EMESH, "tile working set exceeds shared memory");
  c.tl.total_halo = total_h;
  c.tl.total_nodes = total_n;
  setup_prefetch(c);
  // opt in to the dynamic shared memory this mesh needs (never lowered, so
  // contexts of smaller meshes keep working)
  static size_t smem_set = 48 * 1024;
  static bool carveout_set = false;
  if (!carveout_set) {  // all of the unified L1/shared storage as shared memory: 4 tiles per SM
    SFEM_CUDA(cudaFuncSetAttribute(k_mf32_tiled<float, float>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                   cudaSharedmemCarveoutMaxShared));
    SFEM_CUDA(cudaFuncSetAttribute(k_mf32_tiled<double, double>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                   cudaSharedmemCarveoutMaxShared));
    carveout_set = true;
  }
  if (c.tl.smem > smem_set) {
    SFEM_CUDA(cudaFuncSetAttribute(k_mf32_tiled<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)c.tl.smem));
    SFEM_CUDA(cudaFuncSetAttribute(k_mf32_tiled<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)c.tl.smem));
    smem_set = c.tl.smem;
  }
  c.tl.ready = true;
}

template <class TU, class TY>
void launch_mf32_tiled(Ctx &c, cudaStream_t st, const TU *u, TY *y, double *energy_out, const int *done) {
  TileArgs A{c.tl.tile_start, c.tl.hoff, c.tl.noff, c.tl.halo_tet, c.tl.halo_lconn, c.tl.tile_nodes,
             c.tl.node_inc, c.tl.rec, c.n_tets, c.tl.slot_stride};
  const int v = sizeof(TU) == 8 ? 1 : 0;
  if (c.tl.pf_grid[v] > 0) {
    const PfLayout P{(int)c.tl.n_tiles, c.tl.pf_capN,  c.tl.pf_capH,  c.tl.pf_capH2,  c.tl.pf_ibytes,
                     c.tl.pf_capR,      c.tl.pf_off_i, c.tl.pf_off_h, c.tl.pf_off_u, c.tl.pf_off_w[v]};
    k_mf32_tiled_pf<TU, TY, 256><<<(unsigned)c.tl.pf_grid[v], 256, c.tl.pf_smem[v], st>>>(
        A, P, u, y, (float)c.lam, (float)c.mu, energy_out, done, c.tl.err);
  } else {
    k_mf32_tiled<TU, TY><<<(unsigned)c.tl.n_tiles, kTileThreads, c.tl.smem, st>>>(A, u, y, (float)c.lam,
                                                                                 (float)c.mu, energy_out, done);
  }
  SFEM_CHECK_LAUNCH();
}

template void launch_mf32_tiled<float, float>(Ctx &, cudaStream_t, const float *, float *, double *, const int *);
template void launch_mf32_tiled<double, double>(Ctx &, cudaStream_t, const double *, double *, double *,
                                                const int *);

}  // namespace sfem

extern "C" int sfem_tile_info(sfem_ctx *h, int64_t *out, int n) {
  using namespace sfem;
  try {
    SFEM_REQUIRE(h && h->c.vol && out && n >= 1, SFEM_EINVAL, "bad arguments");
    const TileData &t = h->c.tl;
    SFEM_REQUIRE(t.ready, SFEM_EINVAL, "the tiled operator is not set up");
    const int64_t v[10] = {t.n_tiles,     t.max_halo,      t.max_nodes,           t.slot_stride, t.total_halo,
                           t.total_nodes, (int64_t)t.smem, (int64_t)t.pf_smem[0], t.pf_grid[0], t.pf_threads[0]};
    for (int i = 0; i < n && i < 10; ++i) out[i] = v[i];
  } catch (const Error &err) {
    set_last_error(err.msg);
    return err.status;
  }
  return SFEM_OK;
}
