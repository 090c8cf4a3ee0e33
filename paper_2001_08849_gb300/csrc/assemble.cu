// CSR assembly of the smoothed stiffness K = sum_k V_k Bbar_k^T c Bbar_k
// (Eq. 9), FP64.
//
// The paper fills COO triplets (N_e*144 + N_i*225 of them, Eq. 12) and lets
// sparse() sum duplicates into CSC (Section 3.3, STEP 4-5).  Here the CSR
// pattern is built first and the face matrices are added in place:
//   1. node graph: node I couples with J when both lie in the stencil of a
//      face, i.e. J is a node of a tet e containing I or the far node of a
//      neighbour of such an e (one warp per node, sorted unique list by
//      repeated warp-min over the candidates staged in shared memory);
//   2. scalar CSR: rows 3I+r hold columns 3J+c for J in the node list, in
//      ascending order (canonical layout, every stencil pair present);
//   3. values: per face, the 3x3 blocks
//      V_k [lam b_I b_J^T + mu b_J b_I^T + mu (b_I . b_J) I]
//      (isotropic c with the Voigt rows of Eq. 4) added with FP64 atomics.

#include <cuda_runtime.h>

#include <climits>

#include "face.cuh"
#include "sfem_internal.cuh"

namespace sfem {

constexpr int kAdjWarps = 4;
constexpr int kAdjCand = kMaxInc * 8;

__global__ void __launch_bounds__(32 * kAdjWarps)
    k_node_adj(int64_t n_nodes, const int64_t *__restrict__ n2t_ptr, const int32_t *__restrict__ n2t,
               const int32_t *__restrict__ tets, const int32_t *__restrict__ nbr,
               const int32_t *__restrict__ nbr_slot, const int64_t *__restrict__ nptr, int32_t *__restrict__ deg,
               int32_t *__restrict__ nadj) {
  __shared__ int cand[kAdjWarps][kAdjCand];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int64_t nw = (int64_t)gridDim.x * kAdjWarps;
  for (int64_t I = (int64_t)blockIdx.x * kAdjWarps + wl; I < n_nodes; I += nw) {
    const int64_t b = n2t_ptr[I];
    int len = (int)(n2t_ptr[I + 1] - b);
    if (len > kMaxInc) len = kMaxInc;  // rejected on the host before this kernel runs
    const int nc = 8 * len;
    for (int i = lane; i < nc; i += 32) {
      const int e = n2t[b + i / 8];
      const int j = i % 8;
      int v;
      if (j < 4) {
        v = tets[4 * (int64_t)e + j];
      } else {
        const int nb = nbr[4 * (int64_t)e + (j - 4)];
        v = nb >= 0 ? tets[4 * (int64_t)nb + nbr_slot[4 * (int64_t)e + (j - 4)]] : -1;
      }
      cand[wl][i] = v;
    }
    __syncwarp();
    int last = -1, k = 0;
    const int64_t out = nptr ? nptr[I] : 0;
    while (true) {
      int m = INT_MAX;
      for (int i = lane; i < nc; i += 32) {
        const int v = cand[wl][i];
        if (v > last && v < m) m = v;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (m == INT_MAX) break;
      if (nadj && lane == 0) nadj[out + k] = m;
      ++k;
      last = m;
    }
    if (deg && lane == 0) deg[I] = k;
    __syncwarp();
  }
}

// scalar CSR pattern from the node graph: row 3I+r starts at
// 9 nptr[I] + 3 r deg(I) and lists 3J+c for the sorted neighbours J.
__global__ void k_csr_pattern(int64_t n_nodes, const int64_t *__restrict__ nptr, const int32_t *__restrict__ nadj,
                              int64_t *__restrict__ row_ptr, int32_t *__restrict__ col) {
  const int lane = threadIdx.x & 31;
  const int64_t I = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (I >= n_nodes) return;
  const int64_t b = nptr[I];
  const int d = (int)(nptr[I + 1] - b);
  if (lane < 3) row_ptr[3 * I + lane] = 9 * b + 3 * (int64_t)lane * d;
  if (I == n_nodes - 1 && lane == 0) row_ptr[3 * n_nodes] = 9 * nptr[n_nodes];
  for (int i = lane; i < 3 * d; i += 32) {
    const int J = nadj[b + i / 3];
    const int c = i % 3;
    const int v = 3 * J + c;
    for (int r = 0; r < 3; ++r) col[9 * b + 3 * (int64_t)r * d + i] = v;
  }
}

__device__ __forceinline__ int find_sorted(const int32_t *__restrict__ a, int n, int key) {
  int lo = 0, hi = n - 1;
  while (lo <= hi) {
    const int mid = (lo + hi) >> 1;
    const int v = a[mid];
    if (v == key) return mid;
    if (v < key)
      lo = mid + 1;
    else
      hi = mid - 1;
  }
  return -1;
}

__global__ void k_csr_values(int64_t n_faces, const int32_t *__restrict__ tets, const int32_t *__restrict__ face_tet,
                             const int32_t *__restrict__ face_slot, const double *__restrict__ vol,
                             const double *__restrict__ grad, double lam, double mu,
                             const int64_t *__restrict__ nptr, const int32_t *__restrict__ nadj,
                             double *__restrict__ val, unsigned long long *missing) {
  const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n_faces) return;
  FaceStencil s;
  face_stencil(f, tets, face_tet, face_slot, vol, grad, s);
  for (int i = 0; i < s.nn; ++i) {
    const int I = s.node[i];
    const int64_t b = nptr[I];
    const int d = (int)(nptr[I + 1] - b);
    const double *bi = s.b[i];
    for (int j = 0; j < s.nn; ++j) {
      const int pos = find_sorted(nadj + b, d, s.node[j]);
      if (pos < 0) {
        atomicAdd(missing, 1ull);
        continue;
      }
      const double *bj = s.b[j];
      const double dot = bi[0] * bj[0] + bi[1] * bj[1] + bi[2] * bj[2];
      for (int r = 0; r < 3; ++r) {
        double *row = val + 9 * b + 3 * (int64_t)r * d + 3 * (int64_t)pos;
        for (int cc = 0; cc < 3; ++cc) {
          const double k = s.Vk * (lam * bi[r] * bj[cc] + mu * bj[r] * bi[cc] + (r == cc ? mu * dot : 0.0));
          atomicAdd(row + cc, k);
        }
      }
    }
  }
}

}  // namespace sfem

using namespace sfem;

extern "C" int sfem_assemble(sfem_ctx *h, sfem_csr *out) {
  try {
    SFEM_REQUIRE(h && h->c.vol, SFEM_EINVAL, "context not set up");
    Ctx &c = h->c;
    if (!c.assembled) {
      SFEM_REQUIRE(c.hstat.too_many_inc == 0, SFEM_EMESH,
                   "a node lies in more than " + std::to_string(kMaxInc) + " tets");
      Csr &m = c.csr;
      int32_t *deg = c.mem.get<int32_t>(c.n_nodes);
      const int adj_blocks = grid_for(c.n_nodes, kAdjWarps);
      k_node_adj<<<adj_blocks, 32 * kAdjWarps, 0, c.stream>>>(c.n_nodes, c.n2t_ptr, c.n2t, c.tets, c.nbr,
                                                              c.nbr_slot, nullptr, deg, nullptr);
      SFEM_CHECK_LAUNCH();
      m.nptr = c.mem.get<int64_t>(c.n_nodes + 1);
      const int64_t nblk = scan_counts(c, deg, c.n_nodes, m.nptr);
      m.nadj = c.mem.get<int32_t>(nblk);
      k_node_adj<<<adj_blocks, 32 * kAdjWarps, 0, c.stream>>>(c.n_nodes, c.n2t_ptr, c.n2t, c.tets, c.nbr,
                                                              c.nbr_slot, m.nptr, nullptr, m.nadj);
      SFEM_CHECK_LAUNCH();
      c.mem.drop(deg);
      m.n_rows = c.ndof;
      m.nnz = 9 * nblk;
      SFEM_REQUIRE(m.nnz < (int64_t(1) << 40), SFEM_EINVAL, "too many non-zeros");
      m.row_ptr = c.mem.get<int64_t>(c.ndof + 1);
      m.col = c.mem.get<int32_t>(m.nnz);
      m.val = c.mem.get<double>(m.nnz);
      k_csr_pattern<<<grid_for(32 * c.n_nodes, 256), 256, 0, c.stream>>>(c.n_nodes, m.nptr, m.nadj, m.row_ptr,
                                                                         m.col);
      SFEM_CHECK_LAUNCH();
      SFEM_CUDA(cudaMemsetAsync(m.val, 0, m.nnz * sizeof(double), c.stream));
      unsigned long long *missing = c.mem.get<unsigned long long>(1);
      SFEM_CUDA(cudaMemsetAsync(missing, 0, 8, c.stream));
      k_csr_values<<<grid_for(c.n_faces, 128), 128, 0, c.stream>>>(c.n_faces, c.tets, c.face_tet, c.face_slot,
                                                                   c.vol, c.grad, c.lam, c.mu, m.nptr, m.nadj,
                                                                   m.val, missing);
      SFEM_CHECK_LAUNCH();
      unsigned long long hmiss = 0;
      SFEM_CUDA(cudaMemcpyAsync(&hmiss, missing, 8, cudaMemcpyDeviceToHost, c.stream));
      SFEM_CUDA(cudaStreamSynchronize(c.stream));
      c.mem.drop(missing);
      SFEM_REQUIRE(hmiss == 0, SFEM_EMESH, "face stencil pair missing from the node graph");
      c.assembled = true;
    }
    if (out) {
      out->n_rows = c.csr.n_rows;
      out->nnz = c.csr.nnz;
      out->row_ptr = c.csr.row_ptr;
      out->col = c.csr.col;
      out->val = c.csr.val;
    }
  } catch (const Error &err) {
    set_last_error(err.msg);
    return err.status;
  }
  return SFEM_OK;
}
