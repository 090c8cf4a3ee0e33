// Mesh setup of the FS-FEM-T4 library: FP64 geometry, tet/face topology,
// smoothing-domain weights, loads, Dirichlet mask, Jacobi diagonal.
//
// Geometry follows Eq. 10 (tet volume, taken in absolute value) and Eq. 1
// (linear shape functions, whose gradients are the rows of inv(J)).  The
// face tables carry the information of Face_in / Face_out (Section 3.2,
// Fig. 7, Algorithm 1) but are derived from the tets: node->tet incidence,
// then for every tet face the other tet holding its three nodes.

#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <atomic>
#include <mutex>

#include "face.cuh"
#include "sfem_internal.cuh"

namespace sfem {

// ---------------------------------------------------------------------------
// last error (per thread)
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;
void set_last_error(const std::string &msg) { g_last_error = msg; }

static std::atomic<int64_t> g_launches{0};
static thread_local bool g_capturing = false;
void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
bool capturing() { return g_capturing; }
void set_capturing(bool on) { g_capturing = on; }

// ---------------------------------------------------------------------------
// allocator
// ---------------------------------------------------------------------------
void *Allocator::raw(size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  void *p = nullptr;
  if (alloc) {
    p = alloc(bytes, (void *)stream, user);
  } else {
    if (cudaMallocAsync(&p, bytes, stream) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
  }
  if (!p) throw Error{SFEM_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed"};
  if ((reinterpret_cast<uintptr_t>(p) & 15) != 0)
    throw Error{SFEM_ENOMEM, "allocator returned a pointer that is not 16-byte aligned"};
  blocks.push_back({p, bytes});
  return p;
}

void Allocator::drop(void *p) {
  for (size_t i = 0; i < blocks.size(); ++i)
    if (blocks[i].p == p) {
      if (free)
        free(p, blocks[i].n, (void *)stream, user);
      else
        cudaFreeAsync(p, stream);
      blocks.erase(blocks.begin() + i);
      return;
    }
}

void Allocator::release_all() {
  for (auto &b : blocks) {
    if (free)
      free(b.p, b.n, (void *)stream, user);
    else
      cudaFreeAsync(b.p, stream);
  }
  blocks.clear();
}

// ---------------------------------------------------------------------------
// exclusive scan (counts -> offsets), two levels of block scans
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class TIn>
__global__ void k_scan_tiles(const TIn *in, int64_t n, int64_t *out, int64_t *tile_sums) {
  __shared__ int64_t warp_tot[32];
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    int64_t idx = base + i;
    v[i] = idx < n ? (int64_t)in[idx] : 0;
    s += v[i];
  }
  // inclusive warp scan of the thread sums
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    int64_t wt = warp_tot[lane];
    int64_t wi = wt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    warp_tot[lane] = wi - wt;  // exclusive prefix of warps
    if (lane == 31) tile_sums[blockIdx.x] = wi;
  }
  __syncthreads();
  int64_t run = warp_tot[wid] + incl - s;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    int64_t idx = base + i;
    if (idx < n) out[idx] = run;
    run += v[i];
  }
}

__global__ void k_scan_add(int64_t *out, int64_t n, const int64_t *tile_off) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += tile_off[i / kScanTile];
}

__global__ void k_write_total(int64_t *out, int64_t n, const int64_t *tile_sums, const int64_t *tile_off,
                              int64_t ntiles) {
  out[n] = tile_off[ntiles - 1] + tile_sums[ntiles - 1];
}

template <class TIn>
static void scan_rec(Ctx &c, const TIn *in, int64_t n, int64_t *out) {
  // out has n+1 entries; out[n] = total
  int64_t ntiles = (n + kScanTile - 1) / kScanTile;
  if (ntiles == 0) {
    SFEM_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), c.stream));
    return;
  }
  int64_t *sums = c.mem.get<int64_t>(ntiles);
  int64_t *offs = c.mem.get<int64_t>(ntiles + 1);
  k_scan_tiles<TIn><<<(unsigned)ntiles, kScanThreads, 0, c.stream>>>(in, n, out, sums);
  SFEM_CHECK_LAUNCH();
  if (ntiles == 1) {
    SFEM_CUDA(cudaMemsetAsync(offs, 0, sizeof(int64_t), c.stream));
  } else {
    scan_rec<int64_t>(c, sums, ntiles, offs);
    k_scan_add<<<grid_for(n, 256), 256, 0, c.stream>>>(out, n, offs);
    SFEM_CHECK_LAUNCH();
  }
  k_write_total<<<1, 1, 0, c.stream>>>(out, n, sums, offs, ntiles);
  SFEM_CHECK_LAUNCH();
  c.mem.drop(sums);
  c.mem.drop(offs);
}

int64_t scan_counts(Ctx &c, const int32_t *counts, int64_t n, int64_t *out) {
  scan_rec<int32_t>(c, counts, n, out);
  int64_t total = 0;
  SFEM_CUDA(cudaMemcpyAsync(&total, out + n, sizeof(int64_t), cudaMemcpyDeviceToHost, c.stream));
  SFEM_CUDA(cudaStreamSynchronize(c.stream));
  return total;
}

// ---------------------------------------------------------------------------
// geometry (FP64)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// quality and volume extrema of the tet handled by each lane, reduced over
// the warp before one atomic per warp (positive doubles order like their
// bit patterns); every lane of the warp must call it
__device__ __forceinline__ void warp_geometry_stats(DevStatus *st, bool valid, double q, double V) {
  unsigned long long qb = valid ? (unsigned long long)__double_as_longlong(q) : ~0ull;
  unsigned long long vlo = valid ? (unsigned long long)__double_as_longlong(V) : ~0ull;
  unsigned long long vhi = valid ? (unsigned long long)__double_as_longlong(V) : 0ull;
  qb = warp_min_u64(qb);
  vlo = warp_min_u64(vlo);
  vhi = warp_max_u64(vhi);
  if ((threadIdx.x & 31) == 0 && qb != ~0ull) {
    atomicMin(&st->minq_bits, qb);
    atomicMin(&st->minv_bits, vlo);
    atomicMax(&st->maxv_bits, vhi);
  }
}

// Per tet: V = |det J| / 6 (Eq. 10), gradients grad N_a (Eq. 1) as rows of
// inv(J) with J = [x1-x0, x2-x0, x3-x0]; grad N_0 = -(sum of the others).
// Launched with whole warps (block size a multiple of 32).
__global__ void k_geometry(const double *__restrict__ xyz, const int32_t *__restrict__ tets,
                           int64_t n_tets, int64_t n_nodes, double *__restrict__ vol,
                           double *__restrict__ grad, DevStatus *st) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool valid = false;
  double q = 0.0, V = 0.0;
  if (e < n_tets) {
    const int4 t = reinterpret_cast<const int4 *>(tets)[e];
    const int v[4] = {t.x, t.y, t.z, t.w};
    bool ok = true;
    for (int a = 0; a < 4; ++a) ok = ok && v[a] >= 0 && v[a] < n_nodes;
    double *ge = grad + e * 12;
    double X[4][3], det = 0.0, l3 = 0.0;
    double c23[3] = {}, c31[3] = {}, c12[3] = {};
    if (ok) {
      for (int a = 0; a < 4; ++a)
        for (int i = 0; i < 3; ++i) X[a][i] = xyz[3 * (int64_t)v[a] + i];
      double d1[3], d2[3], d3[3];
      for (int i = 0; i < 3; ++i) {
        d1[i] = X[1][i] - X[0][i];
        d2[i] = X[2][i] - X[0][i];
        d3[i] = X[3][i] - X[0][i];
      }
      c23[0] = d2[1] * d3[2] - d2[2] * d3[1], c23[1] = d2[2] * d3[0] - d2[0] * d3[2],
      c23[2] = d2[0] * d3[1] - d2[1] * d3[0];
      c31[0] = d3[1] * d1[2] - d3[2] * d1[1], c31[1] = d3[2] * d1[0] - d3[0] * d1[2],
      c31[2] = d3[0] * d1[1] - d3[1] * d1[0];
      c12[0] = d1[1] * d2[2] - d1[2] * d2[1], c12[1] = d1[2] * d2[0] - d1[0] * d2[2],
      c12[2] = d1[0] * d2[1] - d1[1] * d2[0];
      det = d1[0] * c23[0] + d1[1] * c23[1] + d1[2] * c23[2];
      double l2 = 0.0;
      for (int a = 0; a < 4; ++a)
        for (int b = a + 1; b < 4; ++b)
          for (int i = 0; i < 3; ++i) {
            const double d = X[a][i] - X[b][i];
            l2 += d * d;
          }
      l2 /= 6.0;
      l3 = l2 * sqrt(l2);
      V = fabs(det) / 6.0;
      valid = isfinite(det) && isfinite(l3) && V > 1e-14 * l3;
    } else {
      atomicAdd(&st->bad_index, 1ull);
    }
    if (ok && !valid) atomicAdd(&st->bad_tets, 1ull);
    if (!valid) {
      vol[e] = 0.0;
      for (int k = 0; k < 12; ++k) ge[k] = 0.0;
    } else {
      q = 6.0 * sqrt(2.0) * V / l3;
      if (q < 1e-3) atomicAdd(&st->slivers, 1ull);
      const double inv = 1.0 / det;
      double g[4][3];
      for (int i = 0; i < 3; ++i) {
        g[1][i] = c23[i] * inv;
        g[2][i] = c31[i] * inv;
        g[3][i] = c12[i] * inv;
        g[0][i] = -(g[1][i] + g[2][i] + g[3][i]);
      }
      vol[e] = V;
      for (int a = 0; a < 4; ++a)
        for (int i = 0; i < 3; ++i) ge[3 * a + i] = g[a][i];
    }
  }
  warp_geometry_stats(st, valid, q, V);
}

// ---------------------------------------------------------------------------
// node -> tet incidence
// ---------------------------------------------------------------------------
__global__ void k_inc_count(const int32_t *__restrict__ tets, int64_t n_tets, int64_t n_nodes,
                            int32_t *cnt) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 4 * n_tets) return;
  int v = tets[i];
  if (v >= 0 && v < n_nodes) atomicAdd(&cnt[v], 1);
}

__global__ void k_inc_fill(const int32_t *__restrict__ tets, int64_t n_tets, int64_t n_nodes,
                           unsigned long long *cursor, int32_t *n2t) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 4 * n_tets) return;
  int v = tets[i];
  if (v >= 0 && v < n_nodes) {
    unsigned long long pos = atomicAdd(&cursor[v], 1ull);
    n2t[pos] = (int32_t)(i >> 2);
  }
}

// sort each node's tet list ascending (insertion sort: lists are short)
__global__ void k_inc_sort(const int64_t *__restrict__ ptr, int32_t *n2t, int64_t n_nodes, DevStatus *st) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n_nodes) return;
  int64_t b = ptr[v], e = ptr[v + 1];
  int64_t len = e - b;
  atomicMax(&st->max_inc, (unsigned long long)len);
  if (len > kMaxInc) atomicAdd(&st->too_many_inc, 1ull);
  for (int64_t i = b + 1; i < e; ++i) {
    int32_t x = n2t[i];
    int64_t j = i - 1;
    while (j >= b && n2t[j] > x) {
      n2t[j + 1] = n2t[j];
      --j;
    }
    n2t[j + 1] = x;
  }
}

// For face a of tet e (the face opposite local vertex a), find the other
// tet holding its three nodes by scanning the incidence list of the face
// node with the shortest list.  More than one such tet is a mesh error.
__global__ void k_neighbors(const int32_t *__restrict__ tets, int64_t n_tets,
                            const int64_t *__restrict__ ptr, const int32_t *__restrict__ n2t,
                            int32_t *nbr, int32_t *nbr_slot, DevStatus *st) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 4 * n_tets) return;
  int64_t e = i >> 2;
  int a = (int)(i & 3);
  int4 t = reinterpret_cast<const int4 *>(tets)[e];
  int v[4] = {t.x, t.y, t.z, t.w};
  int f[3], k = 0;
  for (int b = 0; b < 4; ++b)
    if (b != a) f[k++] = v[b];
  // pick the face node with the shortest incidence list
  int best = 0;
  int64_t blen = ptr[f[0] + 1] - ptr[f[0]];
  for (int j = 1; j < 3; ++j) {
    int64_t l = ptr[f[j] + 1] - ptr[f[j]];
    if (l < blen) {
      blen = l;
      best = j;
    }
  }
  int o1 = f[(best + 1) % 3], o2 = f[(best + 2) % 3];
  int found = -1, slot = -1, cnt = 0;
  for (int64_t p = ptr[f[best]]; p < ptr[f[best] + 1]; ++p) {
    int32_t t2 = n2t[p];
    if (t2 == e) continue;
    int4 u = reinterpret_cast<const int4 *>(tets)[t2];
    int w[4] = {u.x, u.y, u.z, u.w};
    bool h1 = false, h2 = false;
    for (int b = 0; b < 4; ++b) {
      h1 = h1 || w[b] == o1;
      h2 = h2 || w[b] == o2;
    }
    if (h1 && h2) {
      ++cnt;
      found = t2;
      for (int b = 0; b < 4; ++b)
        if (w[b] != f[0] && w[b] != f[1] && w[b] != f[2]) slot = b;
    }
  }
  if (cnt > 1) {
    atomicAdd(&st->bad_faces, 1ull);
    found = -1;
    slot = -1;
  }
  nbr[i] = found;
  nbr_slot[i] = slot;
}

// A tet owns its face a when the face is exterior or the neighbour id is larger.
__global__ void k_face_count(const int32_t *__restrict__ nbr, int64_t n_tets, int32_t *cnt,
                             unsigned long long *n_bnd) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_tets) return;
  int c = 0, b = 0;
  for (int a = 0; a < 4; ++a) {
    int n = nbr[4 * e + a];
    if (n < 0) ++b;
    if (n < 0 || e < n) ++c;
  }
  cnt[e] = c;
  if (b) atomicAdd(n_bnd, (unsigned long long)b);
}

__global__ void k_face_fill(const int32_t *__restrict__ nbr, const int32_t *__restrict__ nbr_slot,
                            int64_t n_tets, const int64_t *__restrict__ fptr, int32_t *face_tet,
                            int32_t *face_slot) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_tets) return;
  int64_t f = fptr[e];
  for (int a = 0; a < 4; ++a) {
    int n = nbr[4 * e + a];
    if (n < 0 || e < n) {
      face_tet[2 * f] = (int32_t)e;
      face_tet[2 * f + 1] = n;
      face_slot[2 * f] = a;
      face_slot[2 * f + 1] = n < 0 ? -1 : nbr_slot[4 * e + a];
      ++f;
    }
  }
}

// Smoothing-domain data.  Omega_k is the union of the sub-tets (face +
// centroid of each adjacent tet), each of volume V_e/4 (Fig. 1), so
// V_k = (V_i + V_j)/4 and the smoothed strain of face k is the volume
// average (V_i eps_i + V_j eps_j) / (V_i + V_j) (Eq. 2-3).  Stored per tet:
// Gs = V_e * grad N_1..3 (planar layout) and kap[a] = 1/(4 (V_e + V_nbr))
// (1/(4 V_e) on exterior faces), in FP64 and rounded once to FP32.
__global__ void k_domain(const double *__restrict__ vol, const double *__restrict__ grad,
                         const int32_t *__restrict__ nbr, int64_t n_tets, double *Gs64, double *kap64,
                         float *Gs32, float *kap32) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_tets) return;
  double V = vol[e];
  for (int k = 0; k < 9; ++k) {
    double g = V * grad[12 * e + 3 + k];
    Gs64[k * n_tets + e] = g;
    Gs32[k * n_tets + e] = (float)g;
  }
  for (int a = 0; a < 4; ++a) {
    int n = nbr[4 * e + a];
    double k = n >= 0 ? 1.0 / (4.0 * (V + vol[n])) : 1.0 / (4.0 * V);
    if (!(V > 0.0)) k = 0.0;
    kap64[4 * e + a] = k;
    kap32[4 * e + a] = (float)k;
  }
}

__global__ void k_face_vk(const int32_t *__restrict__ face_tet, const double *__restrict__ vol,
                          int64_t n_faces, double *Vk) {
  int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n_faces) return;
  int t0 = face_tet[2 * f], t1 = face_tet[2 * f + 1];
  Vk[f] = (vol[t0] + (t1 >= 0 ? vol[t1] : 0.0)) * 0.25;
}

// Nodal loads: each triangle gives t * A / 3 to each of its nodes, A by Eq. 11.
__global__ void k_loads(const double *__restrict__ xyz, int64_t n_nodes, const int32_t *__restrict__ tris,
                        const double *__restrict__ trac, int64_t n_tri, int nrhs, int64_t ndof, double *f,
                        DevStatus *st) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_tri * nrhs) return;
  int64_t r = i / n_tri, t = i % n_tri;
  int v0 = tris[3 * t], v1 = tris[3 * t + 1], v2 = tris[3 * t + 2];
  if (v0 < 0 || v0 >= n_nodes || v1 < 0 || v1 >= n_nodes || v2 < 0 || v2 >= n_nodes) {
    if (r == 0) atomicAdd(&st->bad_tri, 1ull);
    return;
  }
  double a[3], b[3];
  for (int k = 0; k < 3; ++k) {
    a[k] = xyz[3 * (int64_t)v1 + k] - xyz[3 * (int64_t)v0 + k];
    b[k] = xyz[3 * (int64_t)v2 + k] - xyz[3 * (int64_t)v0 + k];
  }
  double cx = a[1] * b[2] - a[2] * b[1], cy = a[2] * b[0] - a[0] * b[2], cz = a[0] * b[1] - a[1] * b[0];
  double A = 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
  const double *tv = trac + 3 * (r * n_tri + t);
  double *fr = f + r * ndof;
  int vs[3] = {v0, v1, v2};
  for (int j = 0; j < 3; ++j)
    for (int k = 0; k < 3; ++k) atomicAdd(&fr[3 * (int64_t)vs[j] + k], tv[k] * A / 3.0);
}

__global__ void k_dirichlet(const int32_t *__restrict__ dofs, const double *__restrict__ vals, int64_t n_dir,
                            int64_t ndof, uint8_t *dmask, double *g, DevStatus *st) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_dir) return;
  int d = dofs[i];
  if (d < 0 || d >= ndof) {
    atomicAdd(&st->bad_dir, 1ull);
    return;
  }
  dmask[d] = 0;
  g[d] = vals ? vals[i] : 0.0;
}

// Diagonal of K from the face matrices: block (I,I) of V_k Bbar^T c Bbar is
// V_k [(lam + mu) b b^T + mu |b|^2 I] for isotropic c (Eq. 4, Eq. 9).
__global__ void k_face_diag(int64_t n_faces, const int32_t *__restrict__ tets, const int32_t *__restrict__ face_tet,
                            const int32_t *__restrict__ face_slot, const double *__restrict__ vol,
                            const double *__restrict__ grad, double lam, double mu, double *diag) {
  int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n_faces) return;
  FaceStencil s;
  face_stencil(f, tets, face_tet, face_slot, vol, grad, s);
  for (int i = 0; i < s.nn; ++i) {
    double bb = s.b[i][0] * s.b[i][0] + s.b[i][1] * s.b[i][1] + s.b[i][2] * s.b[i][2];
    for (int c = 0; c < 3; ++c)
      atomicAdd(&diag[3 * (int64_t)s.node[i] + c], s.Vk * ((lam + mu) * s.b[i][c] * s.b[i][c] + mu * bb));
  }
}

__global__ void k_face_nodes(int64_t n_faces, const int32_t *__restrict__ tets, const int32_t *__restrict__ face_tet,
                             const int32_t *__restrict__ face_slot, const double *__restrict__ vol,
                             const double *__restrict__ grad, int32_t *nodes) {
  int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n_faces) return;
  FaceStencil s;
  face_stencil(f, tets, face_tet, face_slot, vol, grad, s);
  for (int i = 0; i < 5; ++i) nodes[5 * f + i] = s.node[i];
}

__global__ void k_dinv(const double *__restrict__ diag, const uint8_t *__restrict__ dmask, int64_t ndof,
                       double *dinv64, float *dinv32) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ndof) return;
  double d = diag[i];
  double v = (dmask[i] && d > 0.0) ? 1.0 / d : 0.0;
  dinv64[i] = v;
  dinv32[i] = (float)v;
}

// b = P (f - K g) + (I - P) g for one load case, and its squared norm
__global__ void k_rhs(const double *__restrict__ f, const double *__restrict__ Kg, const double *__restrict__ g,
                      const uint8_t *__restrict__ dmask, int64_t ndof, double *b) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ndof) return;
  b[i] = dmask[i] ? f[i] - Kg[i] : g[i];
}

void compute_diag(Ctx &c) {
  SFEM_CUDA(cudaMemsetAsync(c.diag, 0, c.ndof * sizeof(double), c.stream));
  k_face_diag<<<grid_for(c.n_faces, 128), 128, 0, c.stream>>>(c.n_faces, c.tets, c.face_tet, c.face_slot, c.vol,
                                                               c.grad, c.lam, c.mu, c.diag);
  SFEM_CHECK_LAUNCH();
  k_dinv<<<grid_for(c.ndof, 256), 256, 0, c.stream>>>(c.diag, c.dmask, c.ndof, c.dinv64, c.dinv32);
  SFEM_CHECK_LAUNCH();
}

static double bits_to_double(unsigned long long b) {
  double d;
  memcpy(&d, &b, sizeof d);
  return d;
}

// compute b for load case r into a device buffer (ndof)
static void build_rhs(Ctx &c, int r, double *b, double *Kg) {
  if (c.g_zero)
    SFEM_CUDA(cudaMemsetAsync(Kg, 0, c.ndof * sizeof(double), c.stream));  // K 0 = 0
  else
    apply_mf64(c, c.g, Kg, 1, nullptr);
  k_rhs<<<grid_for(c.ndof, 256), 256, 0, c.stream>>>(c.f + (int64_t)r * c.ndof, Kg, c.g, c.dmask, c.ndof, b);
  SFEM_CHECK_LAUNCH();
}

static void setup(Ctx &c, const double *xyz, const int32_t *tets, const int32_t *dir_dofs, const double *dir_vals,
                  const int32_t *trac_tris, const double *trac, bool on_device) {
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaEvent_t ev0, ev1;
  SFEM_CUDA(cudaEventCreate(&ev0));
  SFEM_CUDA(cudaEventCreate(&ev1));
  SFEM_CUDA(cudaEventRecord(ev0, c.stream));

  c.xyz = c.mem.get<double>(3 * c.n_nodes);
  c.tets = c.mem.get<int32_t>(4 * c.n_tets);
  SFEM_CUDA(cudaMemcpyAsync(c.xyz, xyz, 3 * c.n_nodes * sizeof(double), kind, c.stream));
  SFEM_CUDA(cudaMemcpyAsync(c.tets, tets, 4 * c.n_tets * sizeof(int32_t), kind, c.stream));

  c.dstat = c.mem.get<DevStatus>(1);
  DevStatus init{};
  double big = INFINITY;
  memcpy(&init.minq_bits, &big, 8);
  memcpy(&init.minv_bits, &big, 8);
  SFEM_CUDA(cudaMemcpyAsync(c.dstat, &init, sizeof init, cudaMemcpyHostToDevice, c.stream));

  // a1: geometry
  c.vol = c.mem.get<double>(c.n_tets);
  c.grad = c.mem.get<double>(12 * c.n_tets);
  k_geometry<<<grid_for(c.n_tets, 128), 128, 0, c.stream>>>(c.xyz, c.tets, c.n_tets, c.n_nodes, c.vol, c.grad,
                                                            c.dstat);
  SFEM_CHECK_LAUNCH();

  // a2: node->tet incidence, neighbours, faces
  int32_t *cnt = c.mem.get<int32_t>(std::max<int64_t>(c.n_nodes, c.n_tets));
  SFEM_CUDA(cudaMemsetAsync(cnt, 0, c.n_nodes * sizeof(int32_t), c.stream));
  k_inc_count<<<grid_for(4 * c.n_tets, 256), 256, 0, c.stream>>>(c.tets, c.n_tets, c.n_nodes, cnt);
  SFEM_CHECK_LAUNCH();
  c.n2t_ptr = c.mem.get<int64_t>(c.n_nodes + 1);
  int64_t ninc = scan_counts(c, cnt, c.n_nodes, c.n2t_ptr);
  c.n2t = c.mem.get<int32_t>(std::max<int64_t>(ninc, 1));
  unsigned long long *cursor = c.mem.get<unsigned long long>(c.n_nodes + 1);
  SFEM_CUDA(cudaMemcpyAsync(cursor, c.n2t_ptr, c.n_nodes * sizeof(int64_t), cudaMemcpyDeviceToDevice, c.stream));
  k_inc_fill<<<grid_for(4 * c.n_tets, 256), 256, 0, c.stream>>>(c.tets, c.n_tets, c.n_nodes, cursor, c.n2t);
  SFEM_CHECK_LAUNCH();
  k_inc_sort<<<grid_for(c.n_nodes, 128), 128, 0, c.stream>>>(c.n2t_ptr, c.n2t, c.n_nodes, c.dstat);
  SFEM_CHECK_LAUNCH();

  // stop early on index errors: later kernels index nodes without checks
  SFEM_CUDA(cudaMemcpyAsync(&c.hstat, c.dstat, sizeof(DevStatus), cudaMemcpyDeviceToHost, c.stream));
  SFEM_CUDA(cudaStreamSynchronize(c.stream));
  if (c.hstat.bad_index) throw Error{SFEM_EMESH, "tet node id out of range"};

  c.nbr = c.mem.get<int32_t>(4 * c.n_tets);
  c.nbr_slot = c.mem.get<int32_t>(4 * c.n_tets);
  k_neighbors<<<grid_for(4 * c.n_tets, 128), 128, 0, c.stream>>>(c.tets, c.n_tets, c.n2t_ptr, c.n2t, c.nbr,
                                                                 c.nbr_slot, c.dstat);
  SFEM_CHECK_LAUNCH();
  unsigned long long *nb_dev = c.mem.get<unsigned long long>(1);
  SFEM_CUDA(cudaMemsetAsync(nb_dev, 0, 8, c.stream));
  k_face_count<<<grid_for(c.n_tets, 256), 256, 0, c.stream>>>(c.nbr, c.n_tets, cnt, nb_dev);
  SFEM_CHECK_LAUNCH();
  int64_t *fptr = c.mem.get<int64_t>(c.n_tets + 1);
  c.n_faces = scan_counts(c, cnt, c.n_tets, fptr);
  unsigned long long nb = 0;
  SFEM_CUDA(cudaMemcpyAsync(&nb, nb_dev, 8, cudaMemcpyDeviceToHost, c.stream));
  SFEM_CUDA(cudaStreamSynchronize(c.stream));
  c.n_bnd = (int64_t)nb;
  c.n_int = c.n_faces - c.n_bnd;
  c.face_tet = c.mem.get<int32_t>(2 * c.n_faces);
  c.face_slot = c.mem.get<int32_t>(2 * c.n_faces);
  k_face_fill<<<grid_for(c.n_tets, 256), 256, 0, c.stream>>>(c.nbr, c.nbr_slot, c.n_tets, fptr, c.face_tet,
                                                            c.face_slot);
  SFEM_CHECK_LAUNCH();

  // a3: smoothing-domain data
  c.Gs64 = c.mem.get<double>(9 * c.n_tets);
  c.kap64 = c.mem.get<double>(4 * c.n_tets);
  c.Gs32 = c.mem.get<float>(9 * c.n_tets);
  c.kap32 = c.mem.get<float>(4 * c.n_tets);
  k_domain<<<grid_for(c.n_tets, 128), 128, 0, c.stream>>>(c.vol, c.grad, c.nbr, c.n_tets, c.Gs64, c.kap64, c.Gs32,
                                                          c.kap32);
  SFEM_CHECK_LAUNCH();
  c.Vk = c.mem.get<double>(c.n_faces);
  k_face_vk<<<grid_for(c.n_faces, 256), 256, 0, c.stream>>>(c.face_tet, c.vol, c.n_faces, c.Vk);
  SFEM_CHECK_LAUNCH();

  // a5: loads and boundary conditions
  c.f = c.mem.get<double>((int64_t)c.nrhs * c.ndof);
  SFEM_CUDA(cudaMemsetAsync(c.f, 0, (int64_t)c.nrhs * c.ndof * sizeof(double), c.stream));
  if (c.n_tri > 0) {
    int32_t *tris_d = c.mem.get<int32_t>(3 * c.n_tri);
    double *trac_d = c.mem.get<double>(3 * c.n_tri * c.nrhs);
    SFEM_CUDA(cudaMemcpyAsync(tris_d, trac_tris, 3 * c.n_tri * sizeof(int32_t), kind, c.stream));
    SFEM_CUDA(cudaMemcpyAsync(trac_d, trac, 3 * c.n_tri * c.nrhs * sizeof(double), kind, c.stream));
    k_loads<<<grid_for(c.n_tri * c.nrhs, 128), 128, 0, c.stream>>>(c.xyz, c.n_nodes, tris_d, trac_d, c.n_tri,
                                                                   c.nrhs, c.ndof, c.f, c.dstat);
    SFEM_CHECK_LAUNCH();
  }
  c.dmask = c.mem.get<uint8_t>(c.ndof);
  c.g = c.mem.get<double>(c.ndof);
  SFEM_CUDA(cudaMemsetAsync(c.dmask, 1, c.ndof, c.stream));
  SFEM_CUDA(cudaMemsetAsync(c.g, 0, c.ndof * sizeof(double), c.stream));
  if (c.n_dir > 0) {
    c.dir_dofs = c.mem.get<int32_t>(c.n_dir);
    SFEM_CUDA(cudaMemcpyAsync(c.dir_dofs, dir_dofs, c.n_dir * sizeof(int32_t), kind, c.stream));
    c.dir_vals = c.mem.get<double>(c.n_dir);
    if (dir_vals)
      SFEM_CUDA(cudaMemcpyAsync(c.dir_vals, dir_vals, c.n_dir * sizeof(double), kind, c.stream));
    else
      SFEM_CUDA(cudaMemsetAsync(c.dir_vals, 0, c.n_dir * sizeof(double), c.stream));
    k_dirichlet<<<grid_for(c.n_dir, 256), 256, 0, c.stream>>>(c.dir_dofs, c.dir_vals, c.n_dir, c.ndof, c.dmask,
                                                              c.g, c.dstat);
    SFEM_CHECK_LAUNCH();
  }
  c.diag = c.mem.get<double>(c.ndof);
  c.dinv64 = c.mem.get<double>(c.ndof);
  c.dinv32 = c.mem.get<float>(c.ndof);
  compute_diag(c);

  // solver scratch
  c.red_blocks = reduction_blocks();
  int64_t nred = std::max<int64_t>((int64_t)c.red_blocks, (c.n_tets + 127) / 128 + 1);
  c.red_partial = c.mem.get<double>(4 * nred);
  c.scal = c.mem.get<SolveScalars>(4);
  SFEM_CUDA(cudaMemsetAsync(c.scal, 0, 4 * sizeof(SolveScalars), c.stream));
  c.tickets = c.mem.get<unsigned int>(64);
  SFEM_CUDA(cudaMemsetAsync(c.tickets, 0, 64 * sizeof(unsigned int), c.stream));
  SFEM_CUDA(cudaStreamCreateWithFlags(&c.cap_stream, cudaStreamNonBlocking));

  SFEM_CUDA(cudaMemcpyAsync(&c.hstat, c.dstat, sizeof(DevStatus), cudaMemcpyDeviceToHost, c.stream));
  SFEM_CUDA(cudaStreamSynchronize(c.stream));
  if (c.hstat.bad_tets || c.hstat.bad_faces || c.hstat.bad_dir || c.hstat.bad_tri) {
    throw Error{SFEM_EMESH, "invalid mesh: " + std::to_string(c.hstat.bad_tets) + " degenerate tets, " +
                                std::to_string(c.hstat.bad_faces) + " over-shared faces, " +
                                std::to_string(c.hstat.bad_dir) + " bad Dirichlet DOFs, " +
                                std::to_string(c.hstat.bad_tri) + " bad traction triangles"};
  }

  // tiles of the single-pass FP32 operator
  build_tiles(c);

  // ||b|| per load case
  c.g_zero = c.n_dir == 0 || device_norm2(c, c.g, c.ndof) == 0.0;
  double *b = c.mem.get<double>(c.ndof);
  double *Kg = c.mem.get<double>(c.ndof);
  c.bnorm.assign(c.nrhs, 0.0);
  for (int r = 0; r < c.nrhs; ++r) {
    build_rhs(c, r, b, Kg);
    c.bnorm[r] = std::sqrt(device_norm2(c, b, c.ndof));
  }
  c.mem.drop(b);
  c.mem.drop(Kg);
  c.mem.drop(cnt);
  c.mem.drop(cursor);
  c.mem.drop(fptr);
  c.mem.drop(nb_dev);

  SFEM_CUDA(cudaEventRecord(ev1, c.stream));
  SFEM_CUDA(cudaEventSynchronize(ev1));
  float ms = 0.f;
  SFEM_CUDA(cudaEventElapsedTime(&ms, ev0, ev1));
  c.setup_ms = ms;
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
}

}  // namespace sfem

using namespace sfem;

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------
#define SFEM_API_BEGIN try {
#define SFEM_API_END                              \
  }                                               \
  catch (const ::sfem::Error &err) {              \
    ::sfem::set_last_error(err.msg);              \
    return err.status;                            \
  }                                               \
  catch (const std::exception &ex) {              \
    ::sfem::set_last_error(ex.what());            \
    return SFEM_EINVAL;                           \
  }                                               \
  return SFEM_OK;

extern "C" int sfem_mesh_setup(sfem_ctx **out, const double *xyz, int64_t n_nodes, const int32_t *tets,
                               int64_t n_tets, double E, double nu, const int32_t *dir_dofs,
                               const double *dir_vals, int64_t n_dir, const int32_t *trac_tris,
                               const double *trac, int64_t n_tri, const sfem_opts *opts, void *stream) {
  sfem_ctx *h = nullptr;
  try {
    SFEM_REQUIRE(out, SFEM_EINVAL, "out is NULL");
    *out = nullptr;
    SFEM_REQUIRE(xyz && tets, SFEM_EINVAL, "xyz and tets must not be NULL");
    SFEM_REQUIRE(n_nodes >= 4 && n_tets >= 1, SFEM_EINVAL, "need n_nodes >= 4 and n_tets >= 1");
    SFEM_REQUIRE(n_nodes < (int64_t(1) << 31) / 3 && n_tets < (int64_t(1) << 31) / 4, SFEM_EINVAL,
                 "mesh too large for 32-bit DOF and slot indices");
    SFEM_REQUIRE(E > 0.0 && std::isfinite(E), SFEM_EINVAL, "E must be positive");
    SFEM_REQUIRE(nu > -1.0 && nu < 0.5, SFEM_EINVAL, "nu must lie in (-1, 0.5)");
    SFEM_REQUIRE(n_dir >= 0 && (n_dir == 0 || dir_dofs), SFEM_EINVAL, "dir_dofs is NULL");
    SFEM_REQUIRE(n_tri >= 0 && (n_tri == 0 || (trac_tris && trac)), SFEM_EINVAL, "traction arrays are NULL");
    if (opts)
      for (int r : opts->reserved) SFEM_REQUIRE(r == 0, SFEM_EINVAL, "reserved options must be zero");
    h = new sfem_ctx();
    Ctx &c = h->c;
    SFEM_CUDA(cudaGetDevice(&c.device));
    c.stream = (cudaStream_t)stream;
    c.mem.stream = c.stream;
    if (opts) {
      c.mem.alloc = opts->alloc;
      c.mem.free = opts->free;
      c.mem.user = opts->alloc_user;
      SFEM_REQUIRE((opts->alloc == nullptr) == (opts->free == nullptr), SFEM_EINVAL,
                   "alloc and free hooks must be given together");
    }
    c.nrhs = (opts && opts->nrhs > 0) ? opts->nrhs : 1;
    c.n_nodes = n_nodes;
    c.n_tets = n_tets;
    c.ndof = 3 * n_nodes;
    c.n_dir = n_dir;
    c.n_tri = n_tri;
    c.E = E;
    c.nu = nu;
    c.lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    c.mu = E / (2.0 * (1.0 + nu));
    *out = h;  // returned even on SFEM_EMESH so that sfem_get_info can report counts
    setup(c, xyz, tets, dir_dofs, dir_vals, trac_tris, trac, opts && opts->inputs_on_device);
  } catch (const Error &err) {
    set_last_error(err.msg);
    if (h && err.status != SFEM_EMESH) {
      sfem_destroy(h);
      *out = nullptr;
    }
    return err.status;
  } catch (const std::exception &ex) {
    set_last_error(ex.what());
    if (h) sfem_destroy(h);
    if (out) *out = nullptr;
    return SFEM_EINVAL;
  }
  return SFEM_OK;
}

extern "C" void sfem_destroy(sfem_ctx *h) {
  if (!h) return;
  Ctx &c = h->c;
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != c.device) cudaSetDevice(c.device);
  c.mem.release_all();
  cudaStreamSynchronize(c.stream);
  if (c.h_scal) cudaFreeHost(c.h_scal);
  if (c.cap_stream) cudaStreamDestroy(c.cap_stream);
  cudaStreamSynchronize(c.stream);
  if (dev >= 0 && dev != c.device) cudaSetDevice(dev);
  delete h;
}

extern "C" const char *sfem_strerror(int s) {
  switch (s) {
    case SFEM_OK: return "ok";
    case SFEM_EINVAL: return "invalid argument";
    case SFEM_EMESH: return "invalid mesh";
    case SFEM_ENOMEM: return "out of device memory";
    case SFEM_ENOCONV: return "no convergence within the iteration limit";
    case SFEM_EBREAKDOWN: return "conjugate-gradient breakdown";
    case SFEM_ECUDA: return "CUDA error";
    case SFEM_ETIMEOUT: return "device-side wait timed out";
    default: return "unknown status";
  }
}

extern "C" const char *sfem_last_error(void) { return g_last_error.c_str(); }
extern "C" int sfem_version(void) { return SFEM_API_VERSION; }
extern "C" int64_t sfem_launch_count(void) { return g_launches.load(); }

extern "C" int sfem_get_info(const sfem_ctx *h, sfem_mesh_info *info) {
  if (!h || !info) return SFEM_EINVAL;
  const Ctx &c = h->c;
  memset(info, 0, sizeof *info);
  info->n_nodes = c.n_nodes;
  info->n_tets = c.n_tets;
  info->ndof = c.ndof;
  info->n_faces = c.n_faces;
  info->n_interior = c.n_int;
  info->n_boundary = c.n_bnd;
  info->n_dir = c.n_dir;
  info->nrhs = c.nrhs;
  info->nnz = c.assembled ? c.csr.nnz : 0;
  info->n_slivers = (int64_t)c.hstat.slivers;
  info->n_bad_tets = (int64_t)c.hstat.bad_tets + (int64_t)c.hstat.bad_index;
  info->n_bad_faces = (int64_t)c.hstat.bad_faces;
  info->max_tets_per_node = (int64_t)c.hstat.max_inc;
  info->min_quality = bits_to_double(c.hstat.minq_bits);
  info->min_volume = bits_to_double(c.hstat.minv_bits);
  info->max_volume = bits_to_double(c.hstat.maxv_bits);
  info->setup_ms = c.setup_ms;
  return SFEM_OK;
}

static int copy_out(Ctx &c, void *dst, const void *src, size_t bytes) {
  SFEM_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c.stream));
  SFEM_CUDA(cudaStreamSynchronize(c.stream));
  return SFEM_OK;
}

extern "C" int sfem_get_geometry(sfem_ctx *h, double *vol, double *grad) {
  SFEM_API_BEGIN
  SFEM_REQUIRE(h && h->c.vol, SFEM_EINVAL, "context not set up");
  Ctx &c = h->c;
  if (vol) copy_out(c, vol, c.vol, c.n_tets * sizeof(double));
  if (grad) copy_out(c, grad, c.grad, 12 * c.n_tets * sizeof(double));
  SFEM_API_END
}

extern "C" int sfem_get_neighbors(sfem_ctx *h, int32_t *nbr) {
  SFEM_API_BEGIN
  SFEM_REQUIRE(h && h->c.nbr && nbr, SFEM_EINVAL, "context not set up or nbr NULL");
  copy_out(h->c, nbr, h->c.nbr, 4 * h->c.n_tets * sizeof(int32_t));
  SFEM_API_END
}

extern "C" int sfem_get_faces(sfem_ctx *h, int32_t *nodes, int32_t *tets, double *Vk) {
  SFEM_API_BEGIN
  SFEM_REQUIRE(h && h->c.face_tet, SFEM_EINVAL, "context not set up");
  Ctx &c = h->c;
  if (nodes) {
    int32_t *d = c.mem.get<int32_t>(5 * c.n_faces);
    k_face_nodes<<<grid_for(c.n_faces, 128), 128, 0, c.stream>>>(c.n_faces, c.tets, c.face_tet, c.face_slot, c.vol,
                                                                 c.grad, d);
    SFEM_CHECK_LAUNCH();
    copy_out(c, nodes, d, 5 * c.n_faces * sizeof(int32_t));
    c.mem.drop(d);
  }
  if (tets) copy_out(c, tets, c.face_tet, 2 * c.n_faces * sizeof(int32_t));
  if (Vk) copy_out(c, Vk, c.Vk, c.n_faces * sizeof(double));
  SFEM_API_END
}

extern "C" int sfem_get_rhs(sfem_ctx *h, double *b, int rhs) {
  SFEM_API_BEGIN
  SFEM_REQUIRE(h && h->c.f && b, SFEM_EINVAL, "context not set up or b NULL");
  Ctx &c = h->c;
  SFEM_REQUIRE(rhs >= 0 && rhs < c.nrhs, SFEM_EINVAL, "rhs out of range");
  double *bd = c.mem.get<double>(c.ndof);
  double *Kg = c.mem.get<double>(c.ndof);
  build_rhs(c, rhs, bd, Kg);
  copy_out(c, b, bd, c.ndof * sizeof(double));
  c.mem.drop(bd);
  c.mem.drop(Kg);
  SFEM_API_END
}

extern "C" int sfem_get_diag(sfem_ctx *h, double *diag) {
  SFEM_API_BEGIN
  SFEM_REQUIRE(h && h->c.diag && diag, SFEM_EINVAL, "context not set up or diag NULL");
  Ctx &c = h->c;
  // diagonal of A = P K P + (I - P): K_ii on free DOFs, 1 on prescribed ones
  std::vector<double> d(c.ndof);
  std::vector<uint8_t> m(c.ndof);
  copy_out(c, d.data(), c.diag, c.ndof * sizeof(double));
  copy_out(c, m.data(), c.dmask, c.ndof);
  for (int64_t i = 0; i < c.ndof; ++i) diag[i] = m[i] ? d[i] : 1.0;
  SFEM_API_END
}
